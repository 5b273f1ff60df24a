// bsi_resample.cu -- BSI fused with the resampling of a floating image (the
// FFD step that follows BSI; Sec. 7 proposes merging it with BSI), and the
// voxel gradient of that resampling for the adjoint.
//
// A warp walks the forward's strips (forward_unit's decomposition and z / y /
// x contraction of Eq. 1), but each voxel's displacement T never leaves the
// SM: it becomes the sample position p = x + T of the floating image F, read
// with the trilinear interpolant extended by zeros outside F.
//   value mode    : warped(x) = F~(p)                       4 B per voxel out
//   gradient mode : G(x) = dL/dwarped(x) * grad F~(p)       12 B per voxel out
// Output rows are staged in shared memory and leave as TMA bulk copies, as in
// the forward.  The displacement field itself (12 B per voxel) is never
// written: the traffic is the image reads (mostly L1/L2 hits: samples lie near
// their voxel) and the output.
#include "bsi_kernels.cuh"
#include "bsi_launch.h"

namespace bsi {

static __device__ unsigned g_err;

// F~ at (x + tx, y + ty, z + tz) and, in GRAD mode, its gradient in grad[3].
// The integer part of the position is x + floor(t) and its fraction t - floor(t)
// (exact in FP32), so large voxel coordinates cost no precision.  Taps outside
// F get weight 0 and read an in-range element instead (no predicated loads).
template <bool GRAD>
__device__ __forceinline__ float sample_floating(const InstDesc& d, int x, int y, int z, float tx, float ty,
                                                 float tz, float* grad) {
    constexpr float kFar = 2097152.f;   // 2^21 voxels: past every image on either side
    tx = fminf(fmaxf(tx, -kFar), kFar);
    ty = fminf(fmaxf(ty, -kFar), kFar);
    tz = fminf(fmaxf(tz, -kFar), kFar);
    const float fx = floorf(tx), fy = floorf(ty), fz = floorf(tz);
    const float a = tx - fx, b = ty - fy, c = tz - fz;
    const int i = x + (int)fx, j = y + (int)fy, k = z + (int)fz;
    const bool xi0 = (unsigned)i < (unsigned)d.fX, xi1 = (unsigned)(i + 1) < (unsigned)d.fX;
    const bool yj0 = (unsigned)j < (unsigned)d.fY, yj1 = (unsigned)(j + 1) < (unsigned)d.fY;
    const bool zk0 = (unsigned)k < (unsigned)d.fZ, zk1 = (unsigned)(k + 1) < (unsigned)d.fZ;
    const int i0 = xi0 ? i : 0, i1 = xi1 ? i + 1 : 0;
    const int j0 = yj0 ? j : 0, j1 = yj1 ? j + 1 : 0;
    const int k0 = zk0 ? k : 0, k1 = zk1 ? k + 1 : 0;
    const float ex0 = xi0 ? 1.f : 0.f, ex1 = xi1 ? 1.f : 0.f;
    const float ey0 = yj0 ? 1.f : 0.f, ey1 = yj1 ? 1.f : 0.f;
    const float ez0 = zk0 ? 1.f : 0.f, ez1 = zk1 ? 1.f : 0.f;
    const float* F = d.image;
    const float* r00 = F + ((long long)k0 * d.fY + j0) * d.fX;   // (z tap 0, y tap 0)
    const float* r01 = F + ((long long)k0 * d.fY + j1) * d.fX;   // (0, 1)
    const float* r10 = F + ((long long)k1 * d.fY + j0) * d.fX;   // (1, 0)
    const float* r11 = F + ((long long)k1 * d.fY + j1) * d.fX;   // (1, 1)
    const float f000 = __ldg(r00 + i0), f100 = __ldg(r00 + i1);
    const float f010 = __ldg(r01 + i0), f110 = __ldg(r01 + i1);
    const float f001 = __ldg(r10 + i0), f101 = __ldg(r10 + i1);
    const float f011 = __ldg(r11 + i0), f111 = __ldg(r11 + i1);
    // x, then y, then z (weights of taps outside F are 0)
    const float wx0 = ex0 * (1.f - a), wx1 = ex1 * a;
    const float v00 = fmaf(wx1, f100, wx0 * f000), v10 = fmaf(wx1, f110, wx0 * f010);
    const float v01 = fmaf(wx1, f101, wx0 * f001), v11 = fmaf(wx1, f111, wx0 * f011);
    const float wy0 = ey0 * (1.f - b), wy1 = ey1 * b;
    const float v0 = fmaf(wy1, v10, wy0 * v00), v1 = fmaf(wy1, v11, wy0 * v01);
    const float wz0 = ez0 * (1.f - c), wz1 = ez1 * c;
    if (GRAD) {
        // d/da: the x pass differentiated; d/db, d/dc: the y, z passes differentiated
        const float d00 = fmaf(ex1, f100, -ex0 * f000), d10 = fmaf(ex1, f110, -ex0 * f010);
        const float d01 = fmaf(ex1, f101, -ex0 * f001), d11 = fmaf(ex1, f111, -ex0 * f011);
        const float gx0 = fmaf(wy1, d10, wy0 * d00), gx1 = fmaf(wy1, d11, wy0 * d01);
        grad[0] = fmaf(wz1, gx1, wz0 * gx0);
        const float gy0 = fmaf(ey1, v10, -ey0 * v00), gy1 = fmaf(ey1, v11, -ey0 * v01);
        grad[1] = fmaf(wz1, gy1, wz0 * gy0);
        grad[2] = fmaf(ez1, v1, -ez0 * v0);
    }
    return fmaf(wz1, v1, wz0 * v0);
}

// Voxel r of a lane's tile (weights at wo): T by the x-stage of Eq. 1, then the
// sample (value mode) or the scaled gradient (gradient mode), staged at sv.
template <bool GRAD>
__device__ __forceinline__ void resample_voxel(const InstDesc& d, uint32_t sv, int wo, int x, int y, int z,
                                               const float (&p0)[3], const float (&p1)[3], const float (&p2)[3],
                                               const float (&p3)[3], bool in_row) {
    const float w0 = c_lut.w[wo], w1 = c_lut.w[wo + 1], w2 = c_lut.w[wo + 2], w3 = c_lut.w[wo + 3];
    float T[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) T[c] = fmaf(w3, p3[c], fmaf(w2, p2[c], fmaf(w1, p1[c], w0 * p0[c])));
    if (!GRAD) {
        sts_f32(sv, sample_floating<false>(d, x, y, z, T[0], T[1], T[2], nullptr));
    } else {
        float g[3];
        (void)sample_floating<true>(d, x, y, z, T[0], T[1], T[2], g);
        // voxels past the row end are staged but never copied out: no dL/dwarped read
        const float w = in_row ? __ldg(d.gwarp + ((long long)z * d.Y + y) * d.X + x) : 0.f;
        sts_f32(sv, w * g[0]);
        sts_f32(sv + 4, w * g[1]);
        sts_f32(sv + 8, w * g[2]);
    }
}

// One unit (tile-plane kz, tile-row jy, x-group xg) of the resampling; the
// forward_unit walk with the per-voxel epilogue above.
template <int DX, bool GRAD>
__device__ __forceinline__ void resample_unit(const InstDesc& d, long long ul, unsigned char* stage, int buf_bytes,
                                              int lane, int& ring, unsigned* err) {
    constexpr int OB = GRAD ? 12 : 4;   // output bytes per voxel
    const int dx = DX > 0 ? DX : d.dx;
    const FwdUnit u = fwd_unit(d, ul);
    const int col = u.cell0 + lane;

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
    const int wzb = weight_base(d.dz), wyb = weight_base(d.dy), wxb = weight_base(dx);
    const int xl = lane * dx;                 // first strip voxel of this lane's tile
    const int rn = lane < u.ncell ? imin(dx, u.nvox - xl) : 0;
    const int xb = u.x0 + xl;                 // its volume x
    const int nbytes = u.nvox * OB;
    const long long row_pitch = (long long)d.X * OB;
    const long long plane_pitch = row_pitch * d.Y;
    unsigned char* gplane = static_cast<unsigned char*>(d.field) + (((long long)z0 * d.Y + y0) * d.X + u.x0) * OB;

    for (int rz = 0; rz < zn; ++rz, gplane += plane_pitch) {
        const float a0 = c_lut.w[wzb + 4 * rz], a1 = c_lut.w[wzb + 4 * rz + 1];
        const float a2 = c_lut.w[wzb + 4 * rz + 2], a3 = c_lut.w[wzb + 4 * rz + 3];
        float pz[4][3];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                pz[m][c] = fmaf(a3, ph[3][m][c], fmaf(a2, ph[2][m][c], fmaf(a1, ph[1][m][c], a0 * ph[0][m][c])));

        unsigned char* g = gplane;
        for (int ry = 0; ry < yn; ++ry, g += row_pitch) {
            const float b0 = c_lut.w[wyb + 4 * ry], b1 = c_lut.w[wyb + 4 * ry + 1];
            const float b2 = c_lut.w[wyb + 4 * ry + 2], b3 = c_lut.w[wyb + 4 * ry + 3];
            float p0[3], p1[3], p2[3], p3[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                p0[c] = fmaf(b3, pz[3][c], fmaf(b2, pz[2][c], fmaf(b1, pz[1][c], b0 * pz[0][c])));
                p1[c] = __shfl_down_sync(kFull, p0[c], 1);
                p2[c] = __shfl_down_sync(kFull, p0[c], 2);
                p3[c] = __shfl_down_sync(kFull, p0[c], 3);
            }
            const int y = y0 + ry, z = z0 + rz;
            const int shift = (int)(reinterpret_cast<uintptr_t>(g) & 15);
            unsigned char* sb = stage + ring * buf_bytes + shift;
            ring = ring == kStoreStages - 1 ? 0 : ring + 1;
            BSI_GUARD(shift + (DX > 0 ? OB * kLanes * DX : nbytes) <= buf_bytes, kErrStage, err) {
                const uint32_t sv = smem_u32(sb) + (uint32_t)(OB * xl);
                if (DX > 0) {
                    // every lane stages all DX voxels (past the row end for cut and
                    // halo tiles: inside the buffer, never copied out); their samples
                    // read in-range image elements only
                    constexpr int DXS = DX > 0 ? DX : 1;
#pragma unroll
                    for (int r = 0; r < DXS; ++r)
                        resample_voxel<GRAD>(d, sv + OB * r, weight_base(DXS) + 4 * r, xb + r, y, z, p0, p1, p2, p3,
                                             r < rn);
                } else {
                    for (int r = 0; r < rn; ++r)
                        resample_voxel<GRAD>(d, sv + OB * r, wxb + 4 * r, xb + r, y, z, p0, p1, p2, p3, true);
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            BSI_GUARD((g - static_cast<unsigned char*>(d.field)) / OB + u.nvox <= (long long)d.X * d.Y * d.Z &&
                          g >= static_cast<unsigned char*>(d.field) && shift + nbytes <= buf_bytes,
                      kErrFieldWrite, err) {
                store_row<4>(sb, g, shift, nbytes, lane);
            }
            __syncwarp();
        }
    }
}

// Gradient mode keeps the neighbourhood, T, the taps and the gradient live at
// once: one 8-warp CTA per SM with up to 255 registers (at 128 it spilled).
template <bool GRAD, bool GENERIC>
__global__ void __launch_bounds__(kMaxWarpsPerCta * kLanes, GRAD ? 1 : 2)
    bsi_resample_kernel(const __grid_constant__ Batch<1> b) {
    extern __shared__ __align__(16) unsigned char rsmem[];
    const int lane = threadIdx.x & (kLanes - 1);
    const int warp = threadIdx.x >> 5;
    unsigned char* stage = rsmem + (size_t)warp * fwd_warp_smem(b.buf_bytes);
    const int wpc = blockDim.x >> 5;
    int ring = 0;
    const InstDesc& d = b.inst[0];
    for (long long r = 0;; ++r) {
        const long long ul = slot_unit(r, blockIdx.x, warp, gridDim.x, wpc, b.total_units, false);
        if (ul < 0) break;
        if (GENERIC) {
            resample_unit<0, GRAD>(d, ul, stage, b.buf_bytes, lane, ring, &g_err);
        } else {
            switch (d.dx) {
                case 1: resample_unit<1, GRAD>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 2: resample_unit<2, GRAD>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 3: resample_unit<3, GRAD>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 4: resample_unit<4, GRAD>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 5: resample_unit<5, GRAD>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 6: resample_unit<6, GRAD>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 7: resample_unit<7, GRAD>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                default: resample_unit<8, GRAD>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
            }
        }
    }
    if (lane == 0) bulk_wait_all<0>();
    __syncwarp();
}

template <bool GRAD, bool GENERIC>
static cudaError_t launch_rs_t(const Batch<1>& b, cudaStream_t s, LaunchInfo* info) {
    auto kern = bsi_resample_kernel<GRAD, GENERIC>;
    const int wpc = warps_per_cta(fwd_warp_smem(b.buf_bytes), b.warps_req);
    const int threads = wpc * kLanes;
    const int smem = wpc * fwd_warp_smem(b.buf_bytes);
    KernelFacts f;
    cudaError_t e = kernel_facts(reinterpret_cast<const void*>(kern), threads, smem, &f);
    if (e != cudaSuccess) return e;
    const long long want = cdiv(b.total_units, wpc);
    const long long cap = (long long)f.sms * f.ctas_per_sm;
    const int grid = (int)(want < cap ? want : cap);
    if (info) *info = LaunchInfo{grid, threads, smem, f.ctas_per_sm};
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, threads, smem, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_resample(const Batch<1>& b, bool grad, bool generic, cudaStream_t s, LaunchInfo* info) {
    if (grad) return generic ? launch_rs_t<true, true>(b, s, info) : launch_rs_t<true, false>(b, s, info);
    return generic ? launch_rs_t<false, true>(b, s, info) : launch_rs_t<false, false>(b, s, info);
}

cudaError_t resample_err_read_clear(unsigned* out, cudaStream_t s) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_err, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_err);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(p, 0, sizeof(unsigned), s);
}

}  // namespace bsi
