// bsi_resample.cu -- BSI fused with the resampling of a floating image (the
// FFD step that follows BSI; Sec. 8 proposes merging it with BSI), and the
// voxel gradient of that resampling for the adjoint.
//
// A warp walks the forward's strips (forward_unit's decomposition and z / y /
// x contraction of Eq. 1), but each voxel's displacement T never leaves the
// SM: it becomes the sample position p = x + T of the floating image F, read
// with the trilinear interpolant extended by zeros outside F.
//   value mode    : warped(x) = F~(p)                       4 B per voxel out
//   gradient mode : G(x) = dL/dwarped(x) * grad F~(p)       12 B per voxel out
// Per row, every lane stages T of its tile in shared memory (the forward's
// staging layout); the warp then walks the row with consecutive lanes on
// consecutive voxels, so one gather instruction of the warp reads neighbouring
// image elements (a lane per tile put them dx voxels apart: ~27 L1 sectors per
// request, measured, against ~5), and its outputs are coalesced streaming
// stores.  The displacement field itself (12 B per voxel) is never written:
// the traffic is the image reads (mostly L1/L2 hits: samples lie near their
// voxel) and the output.
#include "bsi_kernels.cuh"
#include "bsi_launch.h"

namespace bsi {

static __device__ unsigned g_err;

// Each warp keeps its lanes' 4 x 4 control points in shared memory, ahead of its
// staging row, as [48][32] floats (a lane reads only its own column: no bank
// conflicts).  In registers they held 48 per thread and capped the kernel at two
// CTAs per SM; moved out, three fit, and the extra warps hide the gathers'
// latency (value mode -17%, gradient mode -23% on a 512x512x300 volume).
constexpr int kPhFloats = 48 * kLanes;
constexpr int kPhBytes = kPhFloats * 4;
__device__ __forceinline__ int ph_index(int n, int m, int c, int lane) { return ((n * 4 + m) * 3 + c) * kLanes + lane; }

// F~ at (x + tx, y + ty, z + tz) and, in GRAD mode, its gradient in grad[3].
// The integer part of the position is x + floor(t) and its fraction t - floor(t)
// (exact in FP32), so large voxel coordinates cost no precision.  Taps outside
// F get weight 0 and read an in-range element instead (no predicated loads).
// Element offsets are 32-bit: the host admits floating images of fewer than
// 2^32 elements.
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
    const unsigned uX = (unsigned)d.fX, uY = (unsigned)d.fY;
    const unsigned r00 = ((unsigned)k0 * uY + (unsigned)j0) * uX;   // (z tap 0, y tap 0)
    const unsigned r01 = ((unsigned)k0 * uY + (unsigned)j1) * uX;   // (0, 1)
    const unsigned r10 = ((unsigned)k1 * uY + (unsigned)j0) * uX;   // (1, 0)
    const unsigned r11 = ((unsigned)k1 * uY + (unsigned)j1) * uX;   // (1, 1)
    const float f000 = __ldg(F + (r00 + i0)), f100 = __ldg(F + (r00 + i1));
    const float f010 = __ldg(F + (r01 + i0)), f110 = __ldg(F + (r01 + i1));
    const float f001 = __ldg(F + (r10 + i0)), f101 = __ldg(F + (r10 + i1));
    const float f011 = __ldg(F + (r11 + i0)), f111 = __ldg(F + (r11 + i1));
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

// One unit (tile-plane kz, tile-row jy, x-group xg) of the resampling: the
// forward_unit walk, then per row the sample of every strip voxel v by lane
// v mod 32.  stage is the warp's staging buffer (16-byte aligned), preceded by
// its kPhBytes of control points.
template <int DX, bool GRAD>
__device__ __forceinline__ void resample_unit(const InstDesc& d, long long ul, unsigned char* stage, int buf_bytes,
                                              int lane, unsigned* err) {
    const int dx = DX > 0 ? DX : d.dx;
    const FwdUnit u = fwd_unit(d, ul);
    const int col = u.cell0 + lane;

    float* ph = reinterpret_cast<float*>(stage - kPhBytes);
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
            ph[ph_index(n, m, 0, lane)] = a;
            ph[ph_index(n, m, 1, lane)] = b;
            ph[ph_index(n, m, 2, lane)] = c;
        }

    const int z0 = u.kz * d.dz, zn = imin(d.dz, d.Z - z0);
    const int y0 = u.jy * d.dy, yn = imin(d.dy, d.Y - y0);
    const int wzb = weight_base(d.dz), wyb = weight_base(d.dy), wxb = weight_base(dx);
    const int xl = lane * dx;                 // first strip voxel of this lane's tile
    const int rn = lane < u.ncell ? imin(dx, u.nvox - xl) : 0;
    const uint32_t s0 = smem_u32(stage);
    const uint32_t sv = s0 + 12u * (uint32_t)xl;
    BSI_GUARD((DX > 0 ? 12 * kLanes * DX : 12 * u.nvox) <= buf_bytes && (s0 & 15) == 0, kErrStage, err) {}

    for (int rz = 0; rz < zn; ++rz) {
        const float a0 = c_lut.w[wzb + 4 * rz], a1 = c_lut.w[wzb + 4 * rz + 1];
        const float a2 = c_lut.w[wzb + 4 * rz + 2], a3 = c_lut.w[wzb + 4 * rz + 3];
        float pz[4][3];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                pz[m][c] = fmaf(a3, ph[ph_index(3, m, c, lane)],
                                fmaf(a2, ph[ph_index(2, m, c, lane)],
                                     fmaf(a1, ph[ph_index(1, m, c, lane)], a0 * ph[ph_index(0, m, c, lane)])));

        for (int ry = 0; ry < yn; ++ry) {
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
            // T of the lane's tile into the staging row (voxel v of the strip at 12 v)
            if (DX > 0) {
                constexpr int DXS = DX > 0 ? DX : 1;
                constexpr int VW = tile_vec<DXS>();
                emit_tile<DXS, VW, false, 3>(sv, p0, p1, p2, p3);   // every lane, past the row end too
            } else {
                for (int r = 0; r < rn; ++r) emit_voxel<false, 3>(sv + 12u * r, wxb + 4 * r, p0, p1, p2, p3);
            }
            __syncwarp();
            const int y = y0 + ry, z = z0 + rz;
            const long long rowv = ((long long)z * d.Y + y) * d.X + u.x0;   // voxel index of strip voxel 0
            auto sample_voxel = [&](int v) {
                const uint32_t a = s0 + 12u * (uint32_t)v;
                const float tx = lds_f32(a), ty = lds_f32(a + 4), tz = lds_f32(a + 8);
                const long long o = rowv + v;
                BSI_GUARD(o >= 0 && o < (long long)d.X * d.Y * d.Z, kErrFieldWrite, err) {
                    if (!GRAD) {
                        __stcs(static_cast<float*>(d.field) + o,
                               sample_floating<false>(d, u.x0 + v, y, z, tx, ty, tz, nullptr));
                    } else {
                        float g[3];
                        (void)sample_floating<true>(d, u.x0 + v, y, z, tx, ty, tz, g);
                        const float w = __ldg(d.gwarp + o);
                        float* G = static_cast<float*>(d.field) + 3 * o;
                        __stcs(G, w * g[0]);
                        __stcs(G + 1, w * g[1]);
                        __stcs(G + 2, w * g[2]);
                    }
                }
            };
            // value mode: two voxels per lane in flight (measured 13% faster); the
            // gradient mode's larger live state made that 23% slower
            if (!GRAD) {
#pragma unroll 2
                for (int v = lane; v < u.nvox; v += kLanes) sample_voxel(v);
            } else {
                for (int v = lane; v < u.nvox; v += kLanes) sample_voxel(v);
            }
            __syncwarp();   // every lane has read the staging row before the next one is written
        }
    }
}

template <bool GRAD, bool GENERIC>
__global__ void __launch_bounds__(kMaxWarpsPerCta * kLanes, GRAD ? 2 : 3)
    bsi_resample_kernel(const __grid_constant__ Batch<1> b) {
    extern __shared__ __align__(16) unsigned char rsmem[];
    const int lane = threadIdx.x & (kLanes - 1);
    const int warp = threadIdx.x >> 5;
    unsigned char* stage = rsmem + (size_t)warp * (b.buf_bytes + kPhBytes) + kPhBytes;
    const int wpc = blockDim.x >> 5;
    const InstDesc& d = b.inst[0];
    for (long long r = 0;; ++r) {
        const long long ul = slot_unit(r, blockIdx.x, warp, gridDim.x, wpc, b.total_units, false);
        if (ul < 0) break;
        if (GENERIC) {
            resample_unit<0, GRAD>(d, ul, stage, b.buf_bytes, lane, &g_err);
        } else {
            switch (d.dx) {
                case 1: resample_unit<1, GRAD>(d, ul, stage, b.buf_bytes, lane, &g_err); break;
                case 2: resample_unit<2, GRAD>(d, ul, stage, b.buf_bytes, lane, &g_err); break;
                case 3: resample_unit<3, GRAD>(d, ul, stage, b.buf_bytes, lane, &g_err); break;
                case 4: resample_unit<4, GRAD>(d, ul, stage, b.buf_bytes, lane, &g_err); break;
                case 5: resample_unit<5, GRAD>(d, ul, stage, b.buf_bytes, lane, &g_err); break;
                case 6: resample_unit<6, GRAD>(d, ul, stage, b.buf_bytes, lane, &g_err); break;
                case 7: resample_unit<7, GRAD>(d, ul, stage, b.buf_bytes, lane, &g_err); break;
                default: resample_unit<8, GRAD>(d, ul, stage, b.buf_bytes, lane, &g_err); break;
            }
        }
    }
}

template <bool GRAD, bool GENERIC>
static cudaError_t launch_rs_t(const Batch<1>& b, cudaStream_t s, LaunchInfo* info) {
    auto kern = bsi_resample_kernel<GRAD, GENERIC>;
    const int wpc = warps_per_cta(b.buf_bytes + kPhBytes, b.warps_req);   // control points + a staging row per warp
    const int threads = wpc * kLanes;
    const int smem = wpc * (b.buf_bytes + kPhBytes);
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
