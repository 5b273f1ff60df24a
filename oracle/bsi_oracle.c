/*
 * bsi_oracle.c -- FP64 CPU oracle for cubic B-spline interpolation (BSI).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product path.  It shares
 * nothing with the CUDA library.  "Slow and obviously correct" is the design:
 * every output is Eq. 1 (Sec. 2.1) or its transpose written out per voxel, the
 * basis evaluated from its polynomial at every voxel, no look-up table, no
 * separable factorisation, no tiling.
 *
 * Readings of the paper that this file encodes (the paper is silent on each):
 *  - B_0..B_3 are the standard uniform cubic B-spline blending functions; the
 *    paper cites them as "scalar B-spline coefficients" without printing them
 *    (Sec. 2.1).  B_0 pairs with the lowest index i.
 *  - Voxel coordinates are integer indices and the spacing is in voxels
 *    (Sec. 2.1: "spacing (in voxels)").
 *  - i = floor(x/dx) - 1 is negative near the origin, so the stored grid has a
 *    one-point border: stored column = i + 1 + l.
 *  - Layout is x fastest, channel-last, channel order (x, y, z).
 *
 * Pinned by tests/test_oracle_pins.py against partition of unity, affine
 * reproduction, knot values, a brute-force global sum over the centred cubic
 * B-spline, scipy's tensor-product B-spline, and the adjoint dot-product
 * identity.  ORACLE_MUTANT (default 0) plants one known mistake for the test
 * that checks those pins catch it; builds for every other use leave it at 0.
 */
#include "bsi_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* ------------------------------------------------------------------------- */
/* Cubic B-spline blending functions at fractional offset t in [0,1).          */
/* ------------------------------------------------------------------------- */
static void oracle_basis(double t, double B[4]) {
    const double t2 = t * t;
    const double t3 = t2 * t;
    const double s = 1.0 - t;
    B[0] = s * s * s / 6.0;
    B[1] = (3.0 * t3 - 6.0 * t2 + 4.0) / 6.0;
#if ORACLE_MUTANT == 3 /* dropped constant term in B_2 */
    B[2] = (-3.0 * t3 + 3.0 * t2 + 3.0 * t) / 6.0;
#else
    B[2] = (-3.0 * t3 + 3.0 * t2 + 3.0 * t + 1.0) / 6.0;
#endif
    B[3] = t3 / 6.0;
#if ORACLE_MUTANT == 1 /* basis paired with the indices in reverse order */
    {
        double a = B[0], b = B[1];
        B[0] = B[3]; B[1] = B[2]; B[2] = b; B[3] = a;
    }
#endif
}

/* Cell and fractional offset of one axis, as Eq. 1 defines them:
 * i = floor(x/d) - 1 (returned as the paper's i), u = x/d - floor(x/d). */
static void oracle_axis(int64_t x, int d, int64_t* i, double* u) {
    const double q = (double)x / (double)d;
    const double f = floor(q);
    *i = (int64_t)f - 1;
    *u = q - f;
#if ORACLE_MUTANT == 2 /* wrong sign of the fractional offset */
    *u = 1.0 - *u;
    if (*u >= 1.0) *u = 0.0;
#endif
}

static inline double oracle_load(const void* p, int in_f32, int64_t idx) {
    return in_f32 ? (double)((const float*)p)[idx] : ((const double*)p)[idx];
}

typedef struct {
    int64_t X, Y, Z;
    int dx, dy, dz;
    int64_t nx, ny, nz;
} oracle_geom;

static int oracle_make_geom(oracle_geom* g, int64_t X, int64_t Y, int64_t Z, int dx, int dy,
                            int dz) {
    if (X < 0 || Y < 0 || Z < 0 || dx < 1 || dy < 1 || dz < 1) return -1;
    g->X = X; g->Y = Y; g->Z = Z;
    g->dx = dx; g->dy = dy; g->dz = dz;
    g->nx = (X + dx - 1) / dx + 3;
    g->ny = (Y + dy - 1) / dy + 3;
    g->nz = (Z + dz - 1) / dz + 3;
    return 0;
}

/* Eq. 1 at one voxel: the triple sum over l, m, n in the paper's order. */
static void oracle_eval(const oracle_geom* g, const void* phi, int in_f32, int64_t x, int64_t y,
                        int64_t z, double out[3]) {
    int64_t i, j, k;
    double u, v, w;
    oracle_axis(x, g->dx, &i, &u);
    oracle_axis(y, g->dy, &j, &v);
    oracle_axis(z, g->dz, &k, &w);
#if ORACLE_MUTANT == 4 /* transposed operand: the y offset drives the x weights */
    {
        double t = u; u = v; v = t;
    }
#endif
    double Bu[4], Bv[4], Bw[4];
    oracle_basis(u, Bu);
    oracle_basis(v, Bv);
    oracle_basis(w, Bw);
    out[0] = out[1] = out[2] = 0.0;
    for (int l = 0; l < 4; ++l)
        for (int m = 0; m < 4; ++m)
            for (int n = 0; n < 4; ++n) {
                const double wt = Bu[l] * Bv[m] * Bw[n];
#if ORACLE_MUTANT == 5 /* transposed index: l and m swapped in the grid read */
                const int64_t col = i + 1 + m, row = j + 1 + l;
#else
                const int64_t col = i + 1 + l, row = j + 1 + m;
#endif
                const int64_t pl = k + 1 + n;
                const int64_t idx = ((pl * g->ny + row) * g->nx + col) * 3;
                for (int c = 0; c < 3; ++c) {
#if ORACLE_MUTANT == 6 /* channels crossed */
                    out[c] += wt * oracle_load(phi, in_f32, idx + (c + 1) % 3);
#else
                    out[c] += wt * oracle_load(phi, in_f32, idx + c);
#endif
                }
            }
}

/* ------------------------------------------------------------------------- */
/* A minimal static-partition parallel-for over [0, n).                         */
/* ------------------------------------------------------------------------- */
typedef void (*oracle_body)(void* ctx, int64_t begin, int64_t end, int tid);

typedef struct {
    oracle_body body;
    void* ctx;
    int64_t begin, end;
    int tid;
} oracle_job;

static void* oracle_job_run(void* a) {
    oracle_job* j = (oracle_job*)a;
    j->body(j->ctx, j->begin, j->end, j->tid);
    return NULL;
}

int bsi_oracle_threads(int nthreads) {
    if (nthreads > 0) return nthreads;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* Runs body over nt contiguous chunks of [0, n); chunk t gets tid t. */
static void oracle_parallel(int64_t n, int nt, oracle_body body, void* ctx) {
    if (nt < 1) nt = 1;
    if ((int64_t)nt > n) nt = n > 0 ? (int)n : 1;
    oracle_job* jobs = (oracle_job*)calloc((size_t)nt, sizeof(oracle_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nt, sizeof(pthread_t));
    for (int t = 0; t < nt; ++t) {
        jobs[t].body = body;
        jobs[t].ctx = ctx;
        jobs[t].begin = n * t / nt;
        jobs[t].end = n * (t + 1) / nt;
        jobs[t].tid = t;
    }
    for (int t = 1; t < nt; ++t) pthread_create(&th[t], NULL, oracle_job_run, &jobs[t]);
    oracle_job_run(&jobs[0]);
    for (int t = 1; t < nt; ++t) pthread_join(th[t], NULL);
    free(jobs);
    free(th);
}

/* ------------------------------------------------------------------------- */
/* Forward                                                                     */
/* ------------------------------------------------------------------------- */
typedef struct {
    const oracle_geom* g;
    const void* phi;
    int in_f32;
    double* field;
} fwd_ctx;

static void fwd_rows(void* c, int64_t b, int64_t e, int tid) {
    (void)tid;
    fwd_ctx* f = (fwd_ctx*)c;
    const oracle_geom* g = f->g;
    for (int64_t row = b; row < e; ++row) { /* row = z*Y + y */
        const int64_t z = row / g->Y, y = row % g->Y;
        for (int64_t x = 0; x < g->X; ++x)
            oracle_eval(g, f->phi, f->in_f32, x, y, z, f->field + (row * g->X + x) * 3);
    }
}

int bsi_oracle_forward(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz, const void* phi,
                       int in_f32, double* field, int nthreads) {
    oracle_geom g;
    if (oracle_make_geom(&g, X, Y, Z, dx, dy, dz)) return -1;
    if (!phi || (!field && X * Y * Z > 0)) return -1;
    fwd_ctx c = {&g, phi, in_f32, field};
    oracle_parallel(Y * Z, bsi_oracle_threads(nthreads), fwd_rows, &c);
    return 0;
}

typedef struct {
    const oracle_geom* g;
    const void* phi;
    int in_f32;
    const int64_t* xyz;
    double* out;
    int bad;
} pts_ctx;

static void fwd_pts(void* c, int64_t b, int64_t e, int tid) {
    (void)tid;
    pts_ctx* p = (pts_ctx*)c;
    const oracle_geom* g = p->g;
    for (int64_t q = b; q < e; ++q) {
        const int64_t x = p->xyz[3 * q], y = p->xyz[3 * q + 1], z = p->xyz[3 * q + 2];
        if (x < 0 || y < 0 || z < 0 || x >= g->X || y >= g->Y || z >= g->Z) {
            p->bad = 1;
            continue;
        }
        oracle_eval(g, p->phi, p->in_f32, x, y, z, p->out + 3 * q);
    }
}

int bsi_oracle_forward_points(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz,
                              const void* phi, int in_f32, const int64_t* xyz, int64_t npts,
                              double* out, int nthreads) {
    oracle_geom g;
    if (oracle_make_geom(&g, X, Y, Z, dx, dy, dz)) return -1;
    if (npts < 0 || (npts > 0 && (!phi || !xyz || !out))) return -1;
    pts_ctx c = {&g, phi, in_f32, xyz, out, 0};
    oracle_parallel(npts, bsi_oracle_threads(nthreads), fwd_pts, &c);
    return c.bad ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint: the literal transpose of Eq. 1 as a scatter-add over voxels.       */
/* Each thread owns a z-range of voxels and a private FP64 accumulator over    */
/* the grid planes that range touches; accumulators are summed afterwards in   */
/* thread order, so the result depends only on the thread count.              */
/* ------------------------------------------------------------------------- */
typedef struct {
    const oracle_geom* g;
    const void* grad;
    int in_f32;
    int nt;
    double** acc;      /* per thread: planes [plane0[t], plane0[t]+nplanes[t]) */
    int64_t* plane0;
    int64_t* nplanes;
} adj_ctx;

static void adj_slab(void* c, int64_t zb, int64_t ze, int tid) {
    adj_ctx* a = (adj_ctx*)c;
    const oracle_geom* g = a->g;
    if (ze <= zb) return;
    /* stored planes touched by voxels z in [zb, ze): (k+1)+n, k = floor(z/dz)-1 */
    const int64_t p0 = zb / g->dz, p1 = (ze - 1) / g->dz + 3;
    const int64_t np = p1 - p0 + 1;
    const int64_t plane = g->ny * g->nx * 3;
    double* acc = (double*)calloc((size_t)(np * plane), sizeof(double));
    a->acc[tid] = acc;
    a->plane0[tid] = p0;
    a->nplanes[tid] = np;
    for (int64_t z = zb; z < ze; ++z)
        for (int64_t y = 0; y < g->Y; ++y)
            for (int64_t x = 0; x < g->X; ++x) {
                int64_t i, j, k;
                double u, v, w, Bu[4], Bv[4], Bw[4], G[3];
                oracle_axis(x, g->dx, &i, &u);
                oracle_axis(y, g->dy, &j, &v);
                oracle_axis(z, g->dz, &k, &w);
                oracle_basis(u, Bu);
                oracle_basis(v, Bv);
                oracle_basis(w, Bw);
                const int64_t vi = ((z * g->Y + y) * g->X + x) * 3;
                for (int c2 = 0; c2 < 3; ++c2) G[c2] = oracle_load(a->grad, a->in_f32, vi + c2);
                for (int l = 0; l < 4; ++l)
                    for (int m = 0; m < 4; ++m)
#if ORACLE_MUTANT == 8 /* adjoint drops the last z term */
                        for (int n = 0; n < 3; ++n) {
#else
                        for (int n = 0; n < 4; ++n) {
#endif
                            const double wt = Bu[l] * Bv[m] * Bw[n];
#if ORACLE_MUTANT == 7 /* adjoint scatters to the mirrored x neighbour */
                            const int64_t col = i + 1 + (3 - l);
#else
                            const int64_t col = i + 1 + l;
#endif
                            const int64_t idx =
                                (((k + 1 + n - p0) * g->ny + (j + 1 + m)) * g->nx + col) * 3;
                            for (int c2 = 0; c2 < 3; ++c2) acc[idx + c2] += wt * G[c2];
                        }
            }
}

int bsi_oracle_adjoint(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz, const void* grad,
                       int in_f32, double* dphi, int nthreads) {
    oracle_geom g;
    if (oracle_make_geom(&g, X, Y, Z, dx, dy, dz)) return -1;
    if (!dphi || (!grad && X * Y * Z > 0)) return -1;
    const int64_t plane = g.ny * g.nx * 3;
    memset(dphi, 0, (size_t)(g.nz * plane) * sizeof(double));
    if (X * Y * Z == 0) return 0;
    int nt = bsi_oracle_threads(nthreads);
    if ((int64_t)nt > Z) nt = (int)Z;
    adj_ctx a;
    a.g = &g;
    a.grad = grad;
    a.in_f32 = in_f32;
    a.nt = nt;
    a.acc = (double**)calloc((size_t)nt, sizeof(double*));
    a.plane0 = (int64_t*)calloc((size_t)nt, sizeof(int64_t));
    a.nplanes = (int64_t*)calloc((size_t)nt, sizeof(int64_t));
    oracle_parallel(Z, nt, adj_slab, &a);
    for (int t = 0; t < nt; ++t) {
        if (!a.acc[t]) continue;
        double* dst = dphi + a.plane0[t] * plane;
        const int64_t n = a.nplanes[t] * plane;
        for (int64_t q = 0; q < n; ++q) dst[q] += a.acc[t][q];
        free(a.acc[t]);
    }
    free(a.acc);
    free(a.plane0);
    free(a.nplanes);
    return 0;
}

typedef struct {
    const oracle_geom* g;
    const void* grad;
    int in_f32;
    const int64_t* gxyz;
    double* out;
    int bad;
} adj_pts_ctx;

/* One stored control point: the voxels of its support are those whose cell
 * f = floor(x/dx) satisfies f <= gx <= f + 3, i.e. x in [(gx-3)dx, (gx+1)dx). */
static void adj_pts(void* c, int64_t b, int64_t e, int tid) {
    (void)tid;
    adj_pts_ctx* p = (adj_pts_ctx*)c;
    const oracle_geom* g = p->g;
    for (int64_t q = b; q < e; ++q) {
        const int64_t gx = p->gxyz[3 * q], gy = p->gxyz[3 * q + 1], gz = p->gxyz[3 * q + 2];
        double* o = p->out + 3 * q;
        o[0] = o[1] = o[2] = 0.0;
        if (gx < 0 || gy < 0 || gz < 0 || gx >= g->nx || gy >= g->ny || gz >= g->nz) {
            p->bad = 1;
            continue;
        }
        int64_t x0 = (gx - 3) * g->dx, x1 = (gx + 1) * g->dx;
        int64_t y0 = (gy - 3) * g->dy, y1 = (gy + 1) * g->dy;
        int64_t z0 = (gz - 3) * g->dz, z1 = (gz + 1) * g->dz;
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (z0 < 0) z0 = 0;
        if (x1 > g->X) x1 = g->X;
        if (y1 > g->Y) y1 = g->Y;
        if (z1 > g->Z) z1 = g->Z;
        for (int64_t z = z0; z < z1; ++z)
            for (int64_t y = y0; y < y1; ++y)
                for (int64_t x = x0; x < x1; ++x) {
                    int64_t i, j, k;
                    double u, v, w, Bu[4], Bv[4], Bw[4];
                    oracle_axis(x, g->dx, &i, &u);
                    oracle_axis(y, g->dy, &j, &v);
                    oracle_axis(z, g->dz, &k, &w);
                    oracle_basis(u, Bu);
                    oracle_basis(v, Bv);
                    oracle_basis(w, Bw);
                    const int l = (int)(gx - (i + 1)), m = (int)(gy - (j + 1)),
                              n = (int)(gz - (k + 1));
                    const double wt = Bu[l] * Bv[m] * Bw[n];
                    const int64_t vi = ((z * g->Y + y) * g->X + x) * 3;
                    for (int c2 = 0; c2 < 3; ++c2)
                        o[c2] += wt * oracle_load(p->grad, p->in_f32, vi + c2);
                }
    }
}

int bsi_oracle_adjoint_points(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz,
                              const void* grad, int in_f32, const int64_t* gxyz, int64_t npts,
                              double* out, int nthreads) {
    oracle_geom g;
    if (oracle_make_geom(&g, X, Y, Z, dx, dy, dz)) return -1;
    if (npts < 0 || (npts > 0 && (!gxyz || !out || (!grad && X * Y * Z > 0)))) return -1;
    adj_pts_ctx c = {&g, grad, in_f32, gxyz, out, 0};
    oracle_parallel(npts, bsi_oracle_threads(nthreads), adj_pts, &c);
    return c.bad ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Resampling of a floating image by the BSI displacement field.              */
/*                                                                             */
/* The step of FFD that follows BSI, which the paper proposes to merge with    */
/* it (Sec. 8): the floating image F [fZ][fY][fX] is sampled at p = x + T(x),  */
/* T from Eq. 1 at voxel x, in voxel units.  F~ below is the trilinear         */
/* interpolant of F extended by zeros outside it: with i = floor(p_x),         */
/* a = p_x - i (likewise j, b and k, c),                                       */
/*   F~(p) = sum over s, t, r in {0, 1} of                                     */
/*           (s ? a : 1 - a) (t ? b : 1 - b) (r ? c : 1 - c) F(i+s, j+t, k+r),  */
/* F taken as 0 at indices outside the image.  Its gradient is the derivative  */
/* of that sum in a, b and c (one-sided from above at integer positions,       */
/* where floor() puts them).                                                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    const void* F;
    int in_f32;
    int64_t fX, fY, fZ;
} oracle_image;

static double oracle_tap(const oracle_image* im, int64_t i, int64_t j, int64_t k) {
#if ORACLE_MUTANT == 11 /* edge values repeated outside the image instead of zeros */
    i = i < 0 ? 0 : (i >= im->fX ? im->fX - 1 : i);
    j = j < 0 ? 0 : (j >= im->fY ? im->fY - 1 : j);
    k = k < 0 ? 0 : (k >= im->fZ ? im->fZ - 1 : k);
#endif
    if (i < 0 || j < 0 || k < 0 || i >= im->fX || j >= im->fY || k >= im->fZ) return 0.0;
    return oracle_load(im->F, im->in_f32, (k * im->fY + j) * im->fX + i);
}

/* F~(p) and, when grad is not NULL, its gradient (d/dp_x, d/dp_y, d/dp_z). */
static double oracle_trilinear(const oracle_image* im, double px, double py, double pz,
                               double* grad) {
    const double fi = floor(px), fj = floor(py), fk = floor(pz);
    const double a = px - fi, b = py - fj, c = pz - fk;
    const int64_t i = (int64_t)fi, j = (int64_t)fj, k = (int64_t)fk;
    double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int s = 0; s < 2; ++s)
        for (int t = 0; t < 2; ++t)
            for (int r = 0; r < 2; ++r) {
                const double f = oracle_tap(im, i + s, j + t, k + r);
#if ORACLE_MUTANT == 9 /* x weights of the two taps exchanged */
                const double wx = s ? 1.0 - a : a;
#else
                const double wx = s ? a : 1.0 - a;
#endif
                const double wy = t ? b : 1.0 - b, wz = r ? c : 1.0 - c;
                v += wx * wy * wz * f;
                gx += (s ? 1.0 : -1.0) * wy * wz * f;
                gy += wx * (t ? 1.0 : -1.0) * wz * f;
#if ORACLE_MUTANT == 10 /* sign of the z derivative flipped */
                gz -= wx * wy * (r ? 1.0 : -1.0) * f;
#else
                gz += wx * wy * (r ? 1.0 : -1.0) * f;
#endif
            }
    if (grad) {
        grad[0] = gx;
        grad[1] = gy;
        grad[2] = gz;
    }
    return v;
}

typedef struct {
    const oracle_geom* g;
    const void* phi;
    int in_f32;
    oracle_image im;
    const void* dW;     /* gradient mode: dL/dwarped [Z][Y][X], else NULL */
    int dw_f32;
    double* out;        /* warped [Z][Y][X], or G [Z][Y][X][3] in gradient mode */
} rs_ctx;

static void rs_rows(void* c, int64_t b, int64_t e, int tid) {
    (void)tid;
    rs_ctx* r = (rs_ctx*)c;
    const oracle_geom* g = r->g;
    for (int64_t row = b; row < e; ++row) { /* row = z*Y + y */
        const int64_t z = row / g->Y, y = row % g->Y;
        for (int64_t x = 0; x < g->X; ++x) {
            double T[3], grad[3];
            oracle_eval(g, r->phi, r->in_f32, x, y, z, T);
            const int64_t v = row * g->X + x;
            if (!r->dW) {
                r->out[v] = oracle_trilinear(&r->im, (double)x + T[0], (double)y + T[1],
                                             (double)z + T[2], NULL);
            } else {
                (void)oracle_trilinear(&r->im, (double)x + T[0], (double)y + T[1], (double)z + T[2],
                                       grad);
                const double w = oracle_load(r->dW, r->dw_f32, v);
                for (int ch = 0; ch < 3; ++ch) r->out[3 * v + ch] = w * grad[ch];
            }
        }
    }
}

int bsi_oracle_resample(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz, const void* phi,
                        int in_f32, const void* F, int f_f32, int64_t fX, int64_t fY, int64_t fZ,
                        double* warped, int nthreads) {
    oracle_geom g;
    if (oracle_make_geom(&g, X, Y, Z, dx, dy, dz)) return -1;
    if (fX < 0 || fY < 0 || fZ < 0 || !phi || (X * Y * Z > 0 && !warped) || (fX * fY * fZ > 0 && !F))
        return -1;
    rs_ctx c = {&g, phi, in_f32, {F, f_f32, fX, fY, fZ}, NULL, 0, warped};
    oracle_parallel(Y * Z, bsi_oracle_threads(nthreads), rs_rows, &c);
    return 0;
}

int bsi_oracle_resample_grad(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz,
                             const void* phi, int in_f32, const void* F, int f_f32, int64_t fX,
                             int64_t fY, int64_t fZ, const void* dW, int dw_f32, double* G,
                             int nthreads) {
    oracle_geom g;
    if (oracle_make_geom(&g, X, Y, Z, dx, dy, dz)) return -1;
    if (fX < 0 || fY < 0 || fZ < 0 || !phi || (X * Y * Z > 0 && (!G || !dW)) ||
        (fX * fY * fZ > 0 && !F))
        return -1;
    rs_ctx c = {&g, phi, in_f32, {F, f_f32, fX, fY, fZ}, dW, dw_f32, G};
    oracle_parallel(Y * Z, bsi_oracle_threads(nthreads), rs_rows, &c);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Non-integer, non-aligned spacing (the paper's future work, Sec. 8: grids   */
/* not aligned to the voxel grid, weights computed on the fly).               */
/*                                                                             */
/* Per axis the spacing is num/den voxels and the lattice is shifted by       */
/* off/den voxels: u_x = (x * den + off) / num, cell f = floor(u_x), offset   */
/* u = u_x - f, and Eq. 1 reads the stored columns f .. f + 3 (one border     */
/* point below, as for integer spacing).  With den = 1, off = 0 this is the    */
/* integer-spacing oracle above.  Grid dims: floor(((N - 1) den + off) / num)  */
/* + 4 per axis.                                                               */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t X, Y, Z;
    int64_t num[3], den[3], off[3];
    int64_t n[3];
} oracle_rgeom;

static int64_t oracle_rdim(int64_t N, int64_t num, int64_t den, int64_t off) {
    return N > 0 ? ((N - 1) * den + off) / num + 4 : 4;
}

static void oracle_raxis(int64_t x, int64_t num, int64_t den, int64_t off, int64_t* f, double* u) {
#if ORACLE_MUTANT == 12 /* lattice shift applied with the wrong sign */
    const double q = (double)(x * den + (off ? num - off : 0)) / (double)num;
#else
    const double q = (double)(x * den + off) / (double)num;
#endif
    const double fl = floor(q);
    *f = (int64_t)fl;
    *u = q - fl;
}

int bsi_oracle_forward_rational(int64_t X, int64_t Y, int64_t Z, const int64_t num[3], const int64_t den[3],
                                const int64_t off[3], const void* phi, int in_f32, double* field) {
    if (X < 0 || Y < 0 || Z < 0 || !num || !den || !off || !phi || (X * Y * Z > 0 && !field)) return -1;
    oracle_rgeom g;
    g.X = X; g.Y = Y; g.Z = Z;
    const int64_t N[3] = {X, Y, Z};
    for (int a = 0; a < 3; ++a) {
        if (num[a] < 1 || den[a] < 1 || off[a] < 0 || off[a] >= num[a]) return -1;
        g.num[a] = num[a]; g.den[a] = den[a]; g.off[a] = off[a];
        g.n[a] = oracle_rdim(N[a], num[a], den[a], off[a]);
    }
    for (int64_t z = 0; z < Z; ++z)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t x = 0; x < X; ++x) {
                int64_t fi, fj, fk;
                double u, v, w, Bu[4], Bv[4], Bw[4];
                oracle_raxis(x, g.num[0], g.den[0], g.off[0], &fi, &u);
                oracle_raxis(y, g.num[1], g.den[1], g.off[1], &fj, &v);
                oracle_raxis(z, g.num[2], g.den[2], g.off[2], &fk, &w);
                oracle_basis(u, Bu);
                oracle_basis(v, Bv);
                oracle_basis(w, Bw);
                double* out = field + ((z * Y + y) * X + x) * 3;
                out[0] = out[1] = out[2] = 0.0;
                for (int l = 0; l < 4; ++l)
                    for (int m = 0; m < 4; ++m)
                        for (int n = 0; n < 4; ++n) {
                            const double wt = Bu[l] * Bv[m] * Bw[n];
                            const int64_t idx = (((fk + n) * g.n[1] + (fj + m)) * g.n[0] + (fi + l)) * 3;
                            for (int c = 0; c < 3; ++c) out[c] += wt * oracle_load(phi, in_f32, idx + c);
                        }
            }
    return 0;
}

/* Transpose of bsi_oracle_forward_rational: every voxel scatters W(x, g) grad[x]
 * onto its 4 x 4 x 4 stored control points, in voxel order, in FP64. */
int bsi_oracle_adjoint_rational(int64_t X, int64_t Y, int64_t Z, const int64_t num[3], const int64_t den[3],
                                const int64_t off[3], const void* grad, int in_f32, double* dphi) {
    if (X < 0 || Y < 0 || Z < 0 || !num || !den || !off || !dphi || (X * Y * Z > 0 && !grad)) return -1;
    int64_t n[3];
    const int64_t N[3] = {X, Y, Z};
    for (int a = 0; a < 3; ++a) {
        if (num[a] < 1 || den[a] < 1 || off[a] < 0 || off[a] >= num[a]) return -1;
        n[a] = oracle_rdim(N[a], num[a], den[a], off[a]);
    }
    memset(dphi, 0, (size_t)(n[0] * n[1] * n[2] * 3) * sizeof(double));
    for (int64_t z = 0; z < Z; ++z)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t x = 0; x < X; ++x) {
                int64_t fi, fj, fk;
                double u, v, w, Bu[4], Bv[4], Bw[4], G[3];
                oracle_raxis(x, num[0], den[0], off[0], &fi, &u);
                oracle_raxis(y, num[1], den[1], off[1], &fj, &v);
                oracle_raxis(z, num[2], den[2], off[2], &fk, &w);
                if (fi < 0 || fj < 0 || fk < 0 || fi + 3 >= n[0] || fj + 3 >= n[1] || fk + 3 >= n[2])
                    return -1;   /* a neighbourhood outside the grid: the cell arithmetic is wrong */
                oracle_basis(u, Bu);
                oracle_basis(v, Bv);
                oracle_basis(w, Bw);
                const int64_t vi = ((z * Y + y) * X + x) * 3;
                for (int c = 0; c < 3; ++c) G[c] = oracle_load(grad, in_f32, vi + c);
                for (int l = 0; l < 4; ++l)
                    for (int m = 0; m < 4; ++m)
                        for (int k = 0; k < 4; ++k) {
                            const double wt = Bu[l] * Bv[m] * Bw[k];
#if ORACLE_MUTANT == 13 /* non-integer spacing adjoint: scatters to the mirrored x neighbour */
                            const int64_t col = fi + (3 - l);
#else
                            const int64_t col = fi + l;
#endif
                            const int64_t idx = (((fk + k) * n[1] + (fj + m)) * n[0] + col) * 3;
                            for (int c = 0; c < 3; ++c) dphi[idx + c] += wt * G[c];
                        }
            }
    return 0;
}

/* The voxels of one stored index g's support on one axis: those whose cell f
 * has f <= g <= f + 3; their weight is B_{g - f}(u).  Returns the count. */
static int64_t oracle_rsupport(int64_t g, int64_t N, int64_t num, int64_t den, int64_t off, int64_t* xs,
                               double* ws) {
    int64_t cnt = 0;
    for (int64_t x = 0; x < N; ++x) {
        int64_t f;
        double u, B[4];
        oracle_raxis(x, num, den, off, &f, &u);
        if (f > g || f + 3 < g) continue;
        oracle_basis(u, B);
        xs[cnt] = x;
        ws[cnt] = B[g - f];
        ++cnt;
    }
    return cnt;
}

int bsi_oracle_adjoint_rational_points(int64_t X, int64_t Y, int64_t Z, const int64_t num[3],
                                       const int64_t den[3], const int64_t off[3], const void* grad,
                                       int in_f32, const int64_t* gxyz, int64_t npts, double* out) {
    if (X < 0 || Y < 0 || Z < 0 || !num || !den || !off || npts < 0 ||
        (npts > 0 && (!grad || !gxyz || !out)))
        return -1;
    int64_t n[3];
    const int64_t N[3] = {X, Y, Z};
    for (int a = 0; a < 3; ++a) {
        if (num[a] < 1 || den[a] < 1 || off[a] < 0 || off[a] >= num[a]) return -1;
        n[a] = oracle_rdim(N[a], num[a], den[a], off[a]);
    }
    int64_t* xs[3];
    double* ws[3];
    for (int a = 0; a < 3; ++a) {
        xs[a] = (int64_t*)malloc((size_t)(N[a] + 1) * sizeof(int64_t));
        ws[a] = (double*)malloc((size_t)(N[a] + 1) * sizeof(double));
    }
    int rc = 0;
    for (int64_t q = 0; q < npts && !rc; ++q) {
        int64_t cnt[3];
        for (int a = 0; a < 3; ++a) {
            const int64_t g = gxyz[3 * q + a];
            if (g < 0 || g >= n[a]) { rc = -1; break; }
            cnt[a] = oracle_rsupport(g, N[a], num[a], den[a], off[a], xs[a], ws[a]);
        }
        if (rc) break;
        double* o = out + 3 * q;
        o[0] = o[1] = o[2] = 0.0;
        for (int64_t c2 = 0; c2 < cnt[2]; ++c2)
            for (int64_t c1 = 0; c1 < cnt[1]; ++c1)
                for (int64_t c0 = 0; c0 < cnt[0]; ++c0) {
                    const double wt = ws[0][c0] * ws[1][c1] * ws[2][c2];
                    const int64_t vi = ((xs[2][c2] * Y + xs[1][c1]) * X + xs[0][c0]) * 3;
                    for (int c = 0; c < 3; ++c) o[c] += wt * oracle_load(grad, in_f32, vi + c);
                }
    }
    for (int a = 0; a < 3; ++a) {
        free(xs[a]);
        free(ws[a]);
    }
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Point-wise versions of the resampling and the non-integer spacing, for     */
/* checking full-size results on sampled voxels.                             */
/* ------------------------------------------------------------------------- */
int bsi_oracle_resample_points(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz, const void* phi,
                               int in_f32, const void* F, int f_f32, int64_t fX, int64_t fY, int64_t fZ,
                               const int64_t* xyz, int64_t npts, double* value, double* grad) {
    oracle_geom g;
    if (oracle_make_geom(&g, X, Y, Z, dx, dy, dz)) return -1;
    if (fX < 0 || fY < 0 || fZ < 0 || npts < 0 || (npts > 0 && (!phi || !xyz || !value)) ||
        (fX * fY * fZ > 0 && !F))
        return -1;
    const oracle_image im = {F, f_f32, fX, fY, fZ};
    for (int64_t q = 0; q < npts; ++q) {
        const int64_t x = xyz[3 * q], y = xyz[3 * q + 1], z = xyz[3 * q + 2];
        if (x < 0 || y < 0 || z < 0 || x >= X || y >= Y || z >= Z) return -1;
        double T[3];
        oracle_eval(&g, phi, in_f32, x, y, z, T);
        value[q] = oracle_trilinear(&im, (double)x + T[0], (double)y + T[1], (double)z + T[2],
                                    grad ? grad + 3 * q : NULL);
    }
    return 0;
}

int bsi_oracle_forward_rational_points(int64_t X, int64_t Y, int64_t Z, const int64_t num[3],
                                       const int64_t den[3], const int64_t off[3], const void* phi,
                                       int in_f32, const int64_t* xyz, int64_t npts, double* out) {
    if (X < 0 || Y < 0 || Z < 0 || !num || !den || !off || npts < 0 || (npts > 0 && (!phi || !xyz || !out)))
        return -1;
    int64_t n[3];
    const int64_t N[3] = {X, Y, Z};
    for (int a = 0; a < 3; ++a) {
        if (num[a] < 1 || den[a] < 1 || off[a] < 0 || off[a] >= num[a]) return -1;
        n[a] = oracle_rdim(N[a], num[a], den[a], off[a]);
    }
    for (int64_t q = 0; q < npts; ++q) {
        const int64_t x = xyz[3 * q], y = xyz[3 * q + 1], z = xyz[3 * q + 2];
        if (x < 0 || y < 0 || z < 0 || x >= X || y >= Y || z >= Z) return -1;
        int64_t fi, fj, fk;
        double u, v, w, Bu[4], Bv[4], Bw[4];
        oracle_raxis(x, num[0], den[0], off[0], &fi, &u);
        oracle_raxis(y, num[1], den[1], off[1], &fj, &v);
        oracle_raxis(z, num[2], den[2], off[2], &fk, &w);
        oracle_basis(u, Bu);
        oracle_basis(v, Bv);
        oracle_basis(w, Bw);
        double* o = out + 3 * q;
        o[0] = o[1] = o[2] = 0.0;
        for (int l = 0; l < 4; ++l)
            for (int m = 0; m < 4; ++m)
                for (int k = 0; k < 4; ++k) {
                    const double wt = Bu[l] * Bv[m] * Bw[k];
                    const int64_t idx = (((fk + k) * n[1] + (fj + m)) * n[0] + (fi + l)) * 3;
                    for (int c = 0; c < 3; ++c) o[c] += wt * oracle_load(phi, in_f32, idx + c);
                }
    }
    return 0;
}
