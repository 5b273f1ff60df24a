/*
 * bsi_oracle.h -- FP64 CPU oracle for cubic B-spline interpolation (BSI) of a
 * free-form-deformation control grid into a dense 3-channel displacement field.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this library: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no source, header, table or helper with the CUDA
 * library under paper_2004_05962_gb300/csrc.
 *
 * What it computes (Eq. 1, Sec. 2.1 "B-spline interpolation theory"):
 *
 *   T(x,y,z) = sum_{l=0..3} sum_{m=0..3} sum_{n=0..3}
 *                 B_l(u) B_m(v) B_n(w) phi_{i+l, j+m, k+n}
 *   i = floor(x/dx) - 1,  u = x/dx - floor(x/dx)   (likewise j,v and k,w)
 *
 * with x,y,z integer voxel indices and dx,dy,dz the integer control-point
 * spacing in voxels.  The stored control grid carries a one-point border, so
 * the paper's index i+l is stored at column i+1+l; grid dims are
 * nx = ceil(X/dx)+3 (likewise ny, nz) and every read is in range.
 *
 * Layouts (x fastest, channel-last, channel order x,y,z):
 *   phi   [nz][ny][nx][3]
 *   field [Z][Y][X][3]
 *
 * Input arrays are FP64 (in_f32 == 0) or FP32 (in_f32 != 0, promoted to FP64
 * on read); all arithmetic and every output is FP64.
 *
 * nthreads <= 0 means "all online host cores"; the count used is returned by
 * bsi_oracle_threads().  Functions return 0 on success, -1 on bad arguments.
 */
#ifndef BSI_ORACLE_H
#define BSI_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of threads the oracle uses for a request of nthreads (<= 0: all cores). */
int bsi_oracle_threads(int nthreads);

/* Dense forward field: Eq. 1 evaluated literally at every voxel. */
int bsi_oracle_forward(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz,
                       const void* phi, int in_f32, double* field, int nthreads);

/* Eq. 1 at npts voxels given as (x,y,z) triples in xyz[3*npts]; out[3*npts]. */
int bsi_oracle_forward_points(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz,
                              const void* phi, int in_f32, const int64_t* xyz,
                              int64_t npts, double* out, int nthreads);

/* Adjoint (transpose of Eq. 1): dphi[g][c] = sum_x W(x,g) grad[x][c], where
 * W(x,g) is the Eq. 1 weight that control point g carries at voxel x.  Written
 * as the literal scatter-add over voxels; dphi is overwritten. */
int bsi_oracle_adjoint(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz,
                       const void* grad, int in_f32, double* dphi, int nthreads);

/* The same transpose at npts control points given as stored-grid (gx,gy,gz)
 * triples: for each point, the sum over the voxels of its support. */
int bsi_oracle_adjoint_points(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz,
                              const void* grad, int in_f32, const int64_t* gxyz,
                              int64_t npts, double* out, int nthreads);

/* Resampling of a floating image F [fZ][fY][fX] by the Eq. 1 displacement
 * (the FFD step that follows BSI; Sec. 8 proposes merging it with BSI):
 *   warped[z][y][x] = F~(x + T_x, y + T_y, z + T_z),
 * F~ the trilinear interpolant of F extended by zeros outside the image, in
 * voxel units. */
int bsi_oracle_resample(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz,
                        const void* phi, int in_f32, const void* F, int f_f32,
                        int64_t fX, int64_t fY, int64_t fZ, double* warped, int nthreads);

/* Voxel gradient of a loss L(warped) through the resampling:
 *   G[z][y][x][c] = dW[z][y][x] * dF~/dp_c (x + T(x)),  dW = dL/dwarped,
 * the derivative of the trilinear sum, one-sided from above at integer
 * positions.  dL/dphi is then the adjoint (transpose of Eq. 1) of G. */
int bsi_oracle_resample_grad(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz,
                             const void* phi, int in_f32, const void* F, int f_f32,
                             int64_t fX, int64_t fY, int64_t fZ, const void* dW, int dw_f32,
                             double* G, int nthreads);

/* Non-integer, non-aligned spacing (Sec. 8's future work): per axis a spacing
 * of num/den voxels and a lattice shift of off/den voxels (0 <= off < num):
 * u_x = (x den + off) / num, cell floor(u_x), offset u_x - floor(u_x); grid
 * dims floor(((N-1) den + off) / num) + 4 per axis.  Arrays num, den, off are
 * (x, y, z).  Single-threaded; den = 1, off = 0 gives bsi_oracle_forward. */
int bsi_oracle_forward_rational(int64_t X, int64_t Y, int64_t Z, const int64_t num[3],
                                const int64_t den[3], const int64_t off[3], const void* phi,
                                int in_f32, double* field);

/* Transpose of bsi_oracle_forward_rational (the gradient with respect to the
 * grid): dphi[nz][ny][nx][3] = sum over voxels of W(x, g) grad[x], FP64, in
 * voxel order.  Single-threaded.  The _points form sums, for each of npts
 * stored control points gxyz[3*npts] = (gx, gy, gz), over the voxels of its
 * support (out[3*npts]). */
int bsi_oracle_adjoint_rational(int64_t X, int64_t Y, int64_t Z, const int64_t num[3],
                                const int64_t den[3], const int64_t off[3], const void* grad,
                                int in_f32, double* dphi);
int bsi_oracle_adjoint_rational_points(int64_t X, int64_t Y, int64_t Z, const int64_t num[3],
                                       const int64_t den[3], const int64_t off[3], const void* grad,
                                       int in_f32, const int64_t* gxyz, int64_t npts, double* out);

/* Point-wise forms (for sampled checks of full-size results): the resampled
 * value (and, if grad is not NULL, the interpolant's gradient, 3 per point) at
 * npts voxels xyz[3*npts] = (x, y, z); Eq. 1 with non-integer spacing at npts
 * voxels (out[3*npts]). */
int bsi_oracle_resample_points(int64_t X, int64_t Y, int64_t Z, int dx, int dy, int dz,
                               const void* phi, int in_f32, const void* F, int f_f32,
                               int64_t fX, int64_t fY, int64_t fZ, const int64_t* xyz,
                               int64_t npts, double* value, double* grad);
int bsi_oracle_forward_rational_points(int64_t X, int64_t Y, int64_t Z, const int64_t num[3],
                                       const int64_t den[3], const int64_t off[3], const void* phi,
                                       int in_f32, const int64_t* xyz, int64_t npts, double* out);

#ifdef __cplusplus
}
#endif

#endif /* BSI_ORACLE_H */
