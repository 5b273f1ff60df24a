// bsi_rational.cu -- Eq. 1 for control grids that are not aligned to the voxel
// grid: per axis a spacing of num/den voxels and a lattice shift of off/den
// voxels (the paper's future work, Sec. 7: such grids need the B-spline weights
// computed on the fly instead of from look-up tables).  Cell and offset of
// voxel x: q = x den + off, f = floor(q / num), u = (q - f num) / num, computed
// in integers exactly, u rounded once to FP32.
//
// With a non-integer spacing a control cell holds a varying number of voxels,
// so the strip-of-tiles decomposition of the integer path does not apply.  One
// warp per output row (y, z) instead: the lanes first contract the stored grid
// over z and y into a line of nx columns in shared memory (16 FMAs per column
// and channel), then walk the row voxel by voxel -- consecutive lanes,
// consecutive voxels -- with the 4-tap x sum, writing coalesced streaming
// stores.  Each lane advances its cell and remainder by exact integer steps
// (32 den = a num + b), so there is no integer division per voxel.
#include "bsi_kernels.cuh"
#include "bsi_launch.h"

namespace bsi {

static __device__ unsigned g_err;

constexpr int kRatWarps = 8;

// The four cubic B-spline weights at offset u (FP32, Horner with FMAs).
__device__ __forceinline__ void bspline4(float u, float B[4]) {
    const float s = 1.f - u;
    const float u2 = u * u;
    constexpr float k6 = 1.f / 6.f;
    B[0] = s * s * s * k6;
    B[1] = fmaf(fmaf(3.f, u, -6.f), u2, 4.f) * k6;
    B[2] = fmaf(fmaf(fmaf(-3.f, u, 3.f), u, 3.f), u, 1.f) * k6;
    B[3] = u2 * u * k6;
}

// Cell and weights of coordinate x on one axis (one integer division: per row).
__device__ __forceinline__ int axis_cell(int x, int num, int den, int off, float B[4]) {
    const int q = x * den + off;
    const int f = q / num;
    bspline4(__fdiv_rn((float)(q - f * num), (float)num), B);
    return f;
}

__global__ void __launch_bounds__(kRatWarps * 32) bsi_rational_kernel(const __grid_constant__ RatDesc d) {
    extern __shared__ __align__(16) float rline[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    float* L = rline + (size_t)warp * 3 * d.nx;
    // voxel x = lane of every row: its cell and remainder; a step of 32 voxels
    // adds step_f cells and step_r to the remainder
    const int q0 = lane * d.den[0] + d.off[0];
    const int f_start = q0 / d.num[0], r_start = q0 - f_start * d.num[0];
    const int step_q = 32 * d.den[0];
    const int step_f = step_q / d.num[0], step_r = step_q - step_f * d.num[0];
    const float fnum = (float)d.num[0];
    const long long rows = (long long)d.Y * d.Z;
    for (long long row = (long long)blockIdx.x * wpc + warp; row < rows; row += (long long)gridDim.x * wpc) {
        const int y = (int)(row % d.Y), z = (int)(row / d.Y);
        float By[4], Bz[4];
        const int fy = axis_cell(y, d.num[1], d.den[1], d.off[1], By);
        const int fz = axis_cell(z, d.num[2], d.den[2], d.off[2], Bz);
        // z / y contraction of the grid into the line L[g][c], g = 0 .. nx - 1
        for (int g = lane; g < d.nx; g += 32) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
            for (int n = 0; n < 4; ++n)
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float w = Bz[n] * By[m];
                    const long long e = (((long long)(fz + n) * d.ny + (fy + m)) * d.nx + g) * 3;
                    BSI_GUARD(e >= 0 && e + 3 <= 3LL * d.nx * d.ny * d.nz, kErrPhiRead, &g_err) {
                        const float* p = d.phi + e;
                        a0 = fmaf(w, __ldg(p), a0);
                        a1 = fmaf(w, __ldg(p + 1), a1);
                        a2 = fmaf(w, __ldg(p + 2), a2);
                    }
                }
            L[3 * g] = a0;
            L[3 * g + 1] = a1;
            L[3 * g + 2] = a2;
        }
        __syncwarp();
        float* out = d.field + row * d.X * 3;
        int f = f_start, r = r_start;
        for (int x = lane; x < d.X; x += 32) {
            float B[4];
            bspline4(__fdiv_rn((float)r, fnum), B);
            const float* l = L + 3 * f;   // columns f .. f + 3
            BSI_GUARD(f >= 0 && f + 4 <= d.nx && r >= 0 && r < d.num[0], kErrStage, &g_err) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    __stcs(out + 3LL * x + c,
                           fmaf(B[3], l[9 + c], fmaf(B[2], l[6 + c], fmaf(B[1], l[3 + c], B[0] * l[c]))));
            }
            f += step_f;
            r += step_r;
            if (r >= d.num[0]) {
                r -= d.num[0];
                ++f;
            }
        }
        __syncwarp();   // the line is read by every lane before the next row overwrites it
    }
}

// Rows per warp of the windowed kernel, and the grid widths it takes (its
// shared memory per warp: 4 z-contracted grid rows + the line, 60 nx bytes).
constexpr int kRatRun = 16;
constexpr int kRatWindowMaxNx = 1024;
constexpr int kRatTableMaxX = 2048;   // x cells and weights tabulated per CTA up to this width

// A warp takes a run of kRatRun consecutive rows of one voxel plane z.  It keeps
// the z-contraction of the four grid rows the current row needs,
//   P[g'][col] = sum_n Bz[n] phi[fz+n][g'][col]   (g' = fy .. fy+3, a ring of 4),
// and adds one grid row whenever the row's cell fy advances (spacing >= 1: at
// most one per row), so each output row's line costs 4 taps from shared memory
// instead of 16 grid reads.  Same arithmetic per voxel as bsi_rational_kernel.
template <bool TABLE>
__global__ void __launch_bounds__(kRatWarps * 32) bsi_rational_window_kernel(const __grid_constant__ RatDesc d) {
    extern __shared__ __align__(16) float rwin[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    // TABLE: the x cell and the four x weights of every voxel x, the same for
    // every row, once per CTA (5 words per x) before the warps' rings
    float* xtab = rwin;
    float* P = rwin + (TABLE ? 5 * d.X : 0) + (size_t)warp * 15 * d.nx;   // 4 rows x nx x 3, then the line
    float* L = P + 12 * d.nx;
    if (TABLE) {
        for (int x = threadIdx.x; x < d.X; x += blockDim.x) {
            float B[4];
            const int f = axis_cell(x, d.num[0], d.den[0], d.off[0], B);
            xtab[5 * x] = __int_as_float(f);
            xtab[5 * x + 1] = B[0];
            xtab[5 * x + 2] = B[1];
            xtab[5 * x + 3] = B[2];
            xtab[5 * x + 4] = B[3];
        }
        __syncthreads();
    }
    const int q0 = lane * d.den[0] + d.off[0];
    const int f_start = q0 / d.num[0], r_start = q0 - f_start * d.num[0];
    const int step_q = 32 * d.den[0];
    const int step_f = step_q / d.num[0], step_r = step_q - step_f * d.num[0];
    const float fnum = (float)d.num[0];
    const int runs_y = (d.Y + kRatRun - 1) / kRatRun;
    const long long units = (long long)d.Z * runs_y;
    for (long long un = (long long)blockIdx.x * wpc + warp; un < units; un += (long long)gridDim.x * wpc) {
        const int z = (int)(un / runs_y), ya = (int)(un % runs_y) * kRatRun, yb = imin(ya + kRatRun, d.Y);
        float Bz[4];
        const int fz = axis_cell(z, d.num[2], d.den[2], d.off[2], Bz);
        int have = -1;   // grid rows have-3 .. have are in the ring (slot = row & 3)
        for (int y = ya; y < yb; ++y) {
            float By[4];
            const int fy = axis_cell(y, d.num[1], d.den[1], d.off[1], By);
            for (int gy = imax(have + 1, fy); gy <= fy + 3; ++gy) {   // the grid rows this row adds
                float* Pr = P + (gy & 3) * 3 * d.nx;
                for (int g = lane; g < d.nx; g += 32) {
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
                    for (int n = 0; n < 4; ++n) {
                        const long long e = (((long long)(fz + n) * d.ny + gy) * d.nx + g) * 3;
                        BSI_GUARD(e >= 0 && e + 3 <= 3LL * d.nx * d.ny * d.nz, kErrPhiRead, &g_err) {
                            const float* p = d.phi + e;
                            a0 = fmaf(Bz[n], __ldg(p), a0);
                            a1 = fmaf(Bz[n], __ldg(p + 1), a1);
                            a2 = fmaf(Bz[n], __ldg(p + 2), a2);
                        }
                    }
                    Pr[3 * g] = a0;
                    Pr[3 * g + 1] = a1;
                    Pr[3 * g + 2] = a2;
                }
            }
            have = fy + 3;
            __syncwarp();
            // the line: y contraction of the four ring rows
            const float* R0 = P + ((fy + 0) & 3) * 3 * d.nx;
            const float* R1 = P + ((fy + 1) & 3) * 3 * d.nx;
            const float* R2 = P + ((fy + 2) & 3) * 3 * d.nx;
            const float* R3 = P + ((fy + 3) & 3) * 3 * d.nx;
            for (int i = lane; i < 3 * d.nx; i += 32)
                L[i] = fmaf(By[3], R3[i], fmaf(By[2], R2[i], fmaf(By[1], R1[i], By[0] * R0[i])));
            __syncwarp();
            float* out = d.field + ((long long)z * d.Y + y) * d.X * 3;
            int f = f_start, r = r_start;
            for (int x = lane; x < d.X; x += 32) {
                float B[4];
                if (TABLE) {
                    f = __float_as_int(xtab[5 * x]);
                    B[0] = xtab[5 * x + 1];
                    B[1] = xtab[5 * x + 2];
                    B[2] = xtab[5 * x + 3];
                    B[3] = xtab[5 * x + 4];
                } else {
                    bspline4(__fdiv_rn((float)r, fnum), B);
                }
                const float* l = L + 3 * f;
                BSI_GUARD(f >= 0 && f + 4 <= d.nx, kErrStage, &g_err) {
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        __stcs(out + 3LL * x + c,
                               fmaf(B[3], l[9 + c], fmaf(B[2], l[6 + c], fmaf(B[1], l[3 + c], B[0] * l[c]))));
                }
                if (!TABLE) {
                    f += step_f;
                    r += step_r;
                    if (r >= d.num[0]) {
                        r -= d.num[0];
                        ++f;
                    }
                }
            }
            __syncwarp();   // the line and the ring rows are read before the next row writes
        }
    }
}

int rational_warps_per_cta(int nx) {
    const int per_warp = 12 * nx;
    int w = kSmemBudget / per_warp;
    return w < 1 ? 1 : (w > kRatWarps ? kRatWarps : w);
}

cudaError_t launch_forward_rational(const RatDesc& d, cudaStream_t s, LaunchInfo* info) {
    if (d.nx <= kRatWindowMaxNx) {   // the windowed kernel
        const bool table = d.X <= kRatTableMaxX;
        const int table_bytes = table ? 20 * d.X : 0;
        const int per_warp = 60 * d.nx;
        int wpc = (kSmemBudget - table_bytes) / per_warp;
        wpc = wpc < 1 ? 1 : (wpc > kRatWarps ? kRatWarps : wpc);
        const int threads = wpc * 32, smem = table_bytes + wpc * per_warp;
        const void* kern = table ? reinterpret_cast<const void*>(bsi_rational_window_kernel<true>)
                                 : reinterpret_cast<const void*>(bsi_rational_window_kernel<false>);
        KernelFacts f;
        cudaError_t e = kernel_facts(kern, threads, smem, &f);
        if (e != cudaSuccess) return e;
        const long long want = cdiv((long long)d.Z * cdiv(d.Y, kRatRun), wpc);
        const long long cap = (long long)f.sms * f.ctas_per_sm;
        const int grid = (int)(want < cap ? want : cap);
        if (info) *info = LaunchInfo{grid, threads, smem, f.ctas_per_sm};
        if (grid <= 0) return cudaSuccess;
        if (table) bsi_rational_window_kernel<true><<<grid, threads, smem, s>>>(d);
        else bsi_rational_window_kernel<false><<<grid, threads, smem, s>>>(d);
        return cudaGetLastError();
    }
    const int wpc = rational_warps_per_cta(d.nx);
    const int threads = wpc * 32, smem = wpc * 12 * d.nx;
    KernelFacts f;
    cudaError_t e = kernel_facts(reinterpret_cast<const void*>(bsi_rational_kernel), threads, smem, &f);
    if (e != cudaSuccess) return e;
    const long long want = cdiv((long long)d.Y * d.Z, wpc);
    const long long cap = (long long)f.sms * f.ctas_per_sm;
    const int grid = (int)(want < cap ? want : cap);
    if (info) *info = LaunchInfo{grid, threads, smem, f.ctas_per_sm};
    if (grid <= 0) return cudaSuccess;
    bsi_rational_kernel<<<grid, threads, smem, s>>>(d);
    return cudaGetLastError();
}

cudaError_t rational_err_read_clear(unsigned* out, cudaStream_t s) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_err, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_err);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(p, 0, sizeof(unsigned), s);
}

}  // namespace bsi
