// bsi_kernels.cuh -- sm_103a kernels for cubic B-spline interpolation (BSI).
//
// Forward (Eq. 1, Sec. 2.1), evaluated by sum factorisation: for a tile the
// 4x4x4 neighbourhood is contracted along z, then y, then x, so a voxel costs
// 12 FMAs (4 taps x 3 channels) plus the z and y stages shared by the tiles of
// a warp, instead of the 255 (direct) or 126 (trilinear rewrite) operations
// per channel counted in App. B.
//
// Each warp owns a strip of tiles (see bsi_geometry.h).  Lane l keeps the 4x4
// column of control displacements at grid column cell0 + l in registers (the
// register reuse of Sec. 3.2.2, one column per lane instead of one 4x4x4 cube
// per thread), contracts it along z and y, and takes the three x-neighbour
// columns from lanes l+1..l+3 with shuffles.  Rows are staged in a per-warp
// shared-memory buffer and written with 16-byte coalesced stores -- the paper
// found its one-thread-per-tile stores uncoalesced and bandwidth-limiting
// (Sec. 5.2.1); here every row segment leaves the SM as contiguous 16-byte
// chunks.
//
// Adjoint (transpose of Eq. 1): the same strip walked in the opposite
// direction -- x-transpose per lane, column gather with shuffles, y and z
// accumulation in registers -- into per-unit partial sums, reduced afterwards
// in a fixed order (no atomics, bitwise reproducible).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bsi_geometry.h"
#include "bsi_weights.cuh"

namespace bsi {

constexpr int kWarpsPerCta = 8;                  // at most; fewer when staging buffers are large
constexpr int kThreads = kWarpsPerCta * kLanes;
constexpr int kSmemBudget = 200 * 1024;          // dynamic shared memory per CTA we allow

// Warps per CTA such that each warp's two staging buffers fit the budget.
inline int warps_per_cta(int buf_bytes) {
    int w = kSmemBudget / (2 * buf_bytes);
    return w < 1 ? 1 : (w > kWarpsPerCta ? kWarpsPerCta : w);
}
constexpr unsigned kFull = 0xffffffffu;

// Kernel error bits (checked builds only).
enum : unsigned {
    kErrPhiRead = 1u,
    kErrFieldWrite = 2u,
    kErrStage = 4u,
    kErrGradRead = 8u,
    kErrPartWrite = 16u,
    kErrPartRead = 32u,
    kErrDphiWrite = 64u,
};

#ifdef BSI_CHECKED
#define BSI_GUARD(cond, bit, err)        \
    if (!(cond)) {                       \
        atomicOr((err), (bit));          \
    } else
#else
#define BSI_GUARD(cond, bit, err)
#endif

// ------------------------------------------------------------------ copies

// Stores nbytes from shared s to global g; s and g are congruent mod 16.  The
// 16-byte-aligned body goes out as one coalesced uint4 per lane per step;
// the unaligned head and tail (< 16 bytes each) as ES-byte elements.
template <int ES>
__device__ __forceinline__ void copy_out(const unsigned char* s, unsigned char* g, int nbytes,
                                         int lane) {
    const int mis = (int)((uintptr_t)g & 15);
    int head = mis ? 16 - mis : 0;
    if (head > nbytes) head = nbytes;
    const int nbody = (nbytes - head) >> 4;
    const int tail = nbytes - head - (nbody << 4);
    const uint4* sb = reinterpret_cast<const uint4*>(s + head);
    uint4* gb = reinterpret_cast<uint4*>(g + head);
    for (int i = lane; i < nbody; i += kLanes) __stcs(gb + i, sb[i]);
    const int nh = head / ES, nt = tail / ES;
    int off = -1;
    if (lane < nh) off = lane * ES;
    else if (lane < nh + nt) off = head + (nbody << 4) + (lane - nh) * ES;
    if (off >= 0) {
        if (ES == 4) *reinterpret_cast<uint32_t*>(g + off) = *reinterpret_cast<const uint32_t*>(s + off);
        else *reinterpret_cast<uint16_t*>(g + off) = *reinterpret_cast<const uint16_t*>(s + off);
    }
}

// Loads nbytes (multiple of 4) from global g into shared s; congruent mod 16.
__device__ __forceinline__ void copy_in(unsigned char* s, const unsigned char* g, int nbytes,
                                        int lane) {
    const int mis = (int)((uintptr_t)g & 15);
    int head = mis ? 16 - mis : 0;
    if (head > nbytes) head = nbytes;
    const int nbody = (nbytes - head) >> 4;
    const int tail = nbytes - head - (nbody << 4);
    const uint4* gb = reinterpret_cast<const uint4*>(g + head);
    uint4* sb = reinterpret_cast<uint4*>(s + head);
    for (int i = lane; i < nbody; i += kLanes) sb[i] = gb[i];
    const int nh = head >> 2, nt = tail >> 2;
    int off = -1;
    if (lane < nh) off = lane * 4;
    else if (lane < nh + nt) off = head + (nbody << 4) + (lane - nh) * 4;
    if (off >= 0)
        *reinterpret_cast<uint32_t*>(s + off) = *reinterpret_cast<const uint32_t*>(g + off);
}

template <bool BF16>
__device__ __forceinline__ void put_elem(unsigned char* s, int e, float v) {
    if (BF16) reinterpret_cast<__nv_bfloat16*>(s)[e] = __float2bfloat16_rn(v);
    else reinterpret_cast<float*>(s)[e] = v;
}

// ------------------------------------------------------------------ forward

// One forward unit: tile-plane kz, tile-row jy, x-group xg.  DX > 0 is a
// compile-time x-spacing (fully unrolled inner loop, weights as constant
// operands); DX == 0 reads the spacing at run time.
template <int DX, bool BF16>
__device__ __forceinline__ void forward_unit(const WeightTable& lut, const InstDesc& d,
                                             long long ul, unsigned char* stage, int buf_bytes,
                                             int lane, int& par, unsigned* err) {
    constexpr int ES = BF16 ? 2 : 4;
    const int dx = DX > 0 ? DX : d.dx;
    const FwdUnit u = fwd_unit(d, ul);
    const int col = u.cell0 + lane;

    // 4 (z) x 4 (y) neighbourhood column of control displacements, 3 channels.
    float ph[4][4][3];
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            float a = 0.f, b = 0.f, c = 0.f;
            if (col < d.nx) {
                const long long e = phi_elem(d, u.kz + n, u.jy + m, col);
                BSI_GUARD(e >= 0 && e + 3 <= 3LL * d.nx * d.ny * d.nz, kErrPhiRead, err) {
                    const float* p = d.phi + e;
                    a = __ldg(p);
                    b = __ldg(p + 1);
                    c = __ldg(p + 2);
                }
            }
            ph[n][m][0] = a;
            ph[n][m][1] = b;
            ph[n][m][2] = c;
        }

    const int z0 = u.kz * d.dz, zn = imin(d.dz, d.Z - z0);
    const int y0 = u.jy * d.dy, yn = imin(d.dy, d.Y - y0);
    const float* wz = lut.w + weight_base(d.dz);
    const float* wy = lut.w + weight_base(d.dy);
    const float* wx = lut.w + weight_base(dx);
    const int xl = lane * dx;             // first strip voxel of this lane's tile
    const bool emits = lane < u.ncell;
    const int nbytes = u.nvox * 3 * ES;

    for (int rz = 0; rz < zn; ++rz) {
        const float a0 = wz[4 * rz], a1 = wz[4 * rz + 1], a2 = wz[4 * rz + 2], a3 = wz[4 * rz + 3];
        float pz[4][3];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                pz[m][c] = fmaf(a3, ph[3][m][c], fmaf(a2, ph[2][m][c], fmaf(a1, ph[1][m][c], a0 * ph[0][m][c])));

        for (int ry = 0; ry < yn; ++ry) {
            const float b0 = wy[4 * ry], b1 = wy[4 * ry + 1], b2 = wy[4 * ry + 2], b3 = wy[4 * ry + 3];
            float p0[3], p1[3], p2[3], p3[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                p0[c] = fmaf(b3, pz[3][c], fmaf(b2, pz[2][c], fmaf(b1, pz[1][c], b0 * pz[0][c])));
                p1[c] = __shfl_down_sync(kFull, p0[c], 1);
                p2[c] = __shfl_down_sync(kFull, p0[c], 2);
                p3[c] = __shfl_down_sync(kFull, p0[c], 3);
            }

            const long long e0 = field_elem(d, z0 + rz, y0 + ry, u.x0);
            unsigned char* g = static_cast<unsigned char*>(d.field) + e0 * ES;
            const int shift = (int)((uintptr_t)g & 15);
            unsigned char* sbuf = stage + par * buf_bytes + shift;
            par ^= 1;
            BSI_GUARD(shift + nbytes <= buf_bytes, kErrStage, err) {
                if (emits) {
                    if (DX > 0) {
#pragma unroll
                        for (int r = 0; r < (DX > 0 ? DX : 1); ++r) {
                            if (xl + r < u.nvox) {
                                const float w0 = wx[4 * r], w1 = wx[4 * r + 1], w2 = wx[4 * r + 2], w3 = wx[4 * r + 3];
#pragma unroll
                                for (int c = 0; c < 3; ++c)
                                    put_elem<BF16>(sbuf, (xl + r) * 3 + c,
                                                   fmaf(w3, p3[c], fmaf(w2, p2[c], fmaf(w1, p1[c], w0 * p0[c]))));
                            }
                        }
                    } else {
                        const int rn = imin(dx, u.nvox - xl);
                        for (int r = 0; r < rn; ++r) {
                            const float w0 = wx[4 * r], w1 = wx[4 * r + 1], w2 = wx[4 * r + 2], w3 = wx[4 * r + 3];
#pragma unroll
                            for (int c = 0; c < 3; ++c)
                                put_elem<BF16>(sbuf, (xl + r) * 3 + c,
                                               fmaf(w3, p3[c], fmaf(w2, p2[c], fmaf(w1, p1[c], w0 * p0[c]))));
                        }
                    }
                }
            }
            __syncwarp();
            BSI_GUARD(e0 >= 0 && e0 + 3LL * u.nvox <= 3LL * d.X * d.Y * d.Z && shift + nbytes <= buf_bytes,
                      kErrFieldWrite, err) {
                copy_out<ES>(sbuf, g, nbytes, lane);
            }
        }
    }
}

// ------------------------------------------------------------------ adjoint

// Writes one completed grid plane of a unit's partial sums (lanes 3..31 hold
// the 29 complete columns).
__device__ __forceinline__ void flush_plane(const InstDesc& d, long long ul, int pz, const AdjUnit& u,
                                            int lane, const float (&h)[4][3], float* part,
                                            long long ws_floats, unsigned* err) {
    const int j = lane - kHalo;
    if (j >= 0 && u.col0 + j < d.nx) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const long long e = part_elem(d, ul, pz, m, j);
            BSI_GUARD(e >= 0 && e + 3 <= ws_floats, kErrPartWrite, err) {
                part[e] = h[m][0];
                part[e + 1] = h[m][1];
                part[e + 2] = h[m][2];
            }
        }
    }
}

template <int DX>
__device__ __forceinline__ void adjoint_unit(const WeightTable& lut, const InstDesc& d, long long ul,
                                             unsigned char* stage, int buf_bytes, int lane, int& par,
                                             float* part, long long ws_floats, unsigned* err) {
    const int dx = DX > 0 ? DX : d.dx;
    const AdjUnit u = adj_unit(d, ul);
    const int cell = u.col0 - kHalo + lane;
    const int nv = (cell >= 0 && cell < d.ncx) ? imin(dx, d.X - cell * dx) : 0;
    const int xl = cell * dx - u.xs;      // strip-local first voxel of this lane's tile
    const int y0 = u.jy * d.dy, yn = imin(d.dy, d.Y - y0);
    const float* wz = lut.w + weight_base(d.dz);
    const float* wy = lut.w + weight_base(d.dy);
    const float* wx = lut.w + weight_base(dx);
    const int nbytes = u.nvox * 12;

    float hz[4][4][3];
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c) hz[n][m][c] = 0.f;

    for (int kz = u.kz0; kz < u.kz1; ++kz) {
        const int z0 = kz * d.dz, zn = imin(d.dz, d.Z - z0);
        for (int rz = 0; rz < zn; ++rz) {
            float hy[4][3];
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int c = 0; c < 3; ++c) hy[m][c] = 0.f;

            for (int ry = 0; ry < yn; ++ry) {
                const long long e0 = field_elem(d, z0 + rz, y0 + ry, u.xs);
                const unsigned char* g = reinterpret_cast<const unsigned char*>(d.grad + e0);
                const int shift = (int)((uintptr_t)g & 15);
                unsigned char* sbuf = stage + par * buf_bytes + shift;
                par ^= 1;
                BSI_GUARD(e0 >= 0 && e0 + 3LL * u.nvox <= 3LL * d.X * d.Y * d.Z && shift + nbytes <= buf_bytes,
                          kErrGradRead, err) {
                    copy_in(sbuf, g, nbytes, lane);
                }
                __syncwarp();
                const float* sv = reinterpret_cast<const float*>(sbuf);
                float q[4][3];
#pragma unroll
                for (int l = 0; l < 4; ++l)
#pragma unroll
                    for (int c = 0; c < 3; ++c) q[l][c] = 0.f;
                if (DX > 0) {
#pragma unroll
                    for (int r = 0; r < (DX > 0 ? DX : 1); ++r) {
                        if (r < nv) {
                            const float g0 = sv[(xl + r) * 3], g1 = sv[(xl + r) * 3 + 1], g2 = sv[(xl + r) * 3 + 2];
#pragma unroll
                            for (int l = 0; l < 4; ++l) {
                                const float w = wx[4 * r + l];
                                q[l][0] = fmaf(w, g0, q[l][0]);
                                q[l][1] = fmaf(w, g1, q[l][1]);
                                q[l][2] = fmaf(w, g2, q[l][2]);
                            }
                        }
                    }
                } else {
                    for (int r = 0; r < nv; ++r) {
                        const float g0 = sv[(xl + r) * 3], g1 = sv[(xl + r) * 3 + 1], g2 = sv[(xl + r) * 3 + 2];
#pragma unroll
                        for (int l = 0; l < 4; ++l) {
                            const float w = wx[4 * r + l];
                            q[l][0] = fmaf(w, g0, q[l][0]);
                            q[l][1] = fmaf(w, g1, q[l][1]);
                            q[l][2] = fmaf(w, g2, q[l][2]);
                        }
                    }
                }
                // column sum: column of lane l collects q[k] of the tile k lanes below
                const float b0 = wy[4 * ry], b1 = wy[4 * ry + 1], b2 = wy[4 * ry + 2], b3 = wy[4 * ry + 3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float h = q[0][c] + __shfl_up_sync(kFull, q[1][c], 1) +
                                    __shfl_up_sync(kFull, q[2][c], 2) + __shfl_up_sync(kFull, q[3][c], 3);
                    hy[0][c] = fmaf(b0, h, hy[0][c]);
                    hy[1][c] = fmaf(b1, h, hy[1][c]);
                    hy[2][c] = fmaf(b2, h, hy[2][c]);
                    hy[3][c] = fmaf(b3, h, hy[3][c]);
                }
            }
            const float a0 = wz[4 * rz], a1 = wz[4 * rz + 1], a2 = wz[4 * rz + 2], a3 = wz[4 * rz + 3];
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    hz[0][m][c] = fmaf(a0, hy[m][c], hz[0][m][c]);
                    hz[1][m][c] = fmaf(a1, hy[m][c], hz[1][m][c]);
                    hz[2][m][c] = fmaf(a2, hy[m][c], hz[2][m][c]);
                    hz[3][m][c] = fmaf(a3, hy[m][c], hz[3][m][c]);
                }
        }
        // grid plane kz + 0 is complete for this unit; roll the window by one plane
        flush_plane(d, ul, kz - u.kz0, u, lane, hz[0], part, ws_floats, err);
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int c = 0; c < 3; ++c) hz[n][m][c] = hz[n + 1][m][c];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c) hz[3][m][c] = 0.f;
    }
    const int nk = u.kz1 - u.kz0;
#pragma unroll
    for (int n = 0; n < 3; ++n) flush_plane(d, ul, nk + n, u, lane, hz[n], part, ws_floats, err);
}

}  // namespace bsi
