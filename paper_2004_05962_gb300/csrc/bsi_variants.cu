// bsi_variants.cu -- the paper's own GPU formulations of Eq. 1, kept as an
// option for its accuracy comparison (Sec. 5.4, Tables of the average
// absolute error against an FP64 reference) and as a measured contrast to the
// separable strip kernel of bsi_forward.cu:
//
//  * TT   (thread per tile, Sec. 3.2): one thread per control cell keeps the
//    cell's 4 x 4 x 4 control points in registers and evaluates the triple sum
//    of Eq. 1 for every voxel of the cell (64 weighted terms per channel).
//  * TTLI (thread per tile with linear interpolations, Sec. 3.3, App. B): the
//    same thread evaluates the sum as 8 trilinear interpolations of the 2x2x2
//    sub-cubes and a ninth of their 8 results (9 x 7 lerps, each one FMA and
//    one subtraction: 126 operations per channel).  Along one axis
//      B0 p0 + B1 p1 + B2 p2 + B3 p3 = lerp(lerp(p0, p1, h0), lerp(p2, p3, h1), g1)
//    with g1 = B2 + B3, h0 = B1 / (B0 + B1), h1 = B3 / (B2 + B3) (B0 + B1 = 1 - g1),
//    the tensor product of which gives the 3-D form.
//
// Both write each voxel's three channels where its thread computes them, as
// the paper's kernels do (the uncoalesced output Sec. 5.2.1 measures); they
// are not the fast path.
#include "bsi_kernels.cuh"
#include "bsi_launch.h"

namespace bsi {

static __device__ unsigned g_err;

constexpr int kLerpMaxSpacing = 32;
BSI_HD constexpr int lerp_base(int d) { return 3 * (d * (d - 1) / 2); }   // 3 per offset
constexpr int kLerpCount = lerp_base(kLerpMaxSpacing + 1);

struct LerpTable {
    float w[kLerpCount];   // per spacing d, per offset r: g1, h0, h1
};

constexpr LerpTable make_lerp_table() {
    LerpTable t{};
    for (int d = 1; d <= kLerpMaxSpacing; ++d)
        for (int r = 0; r < d; ++r) {
            const double u = static_cast<double>(r) / static_cast<double>(d);
            const double om = 1.0 - u;
            const double b0 = om * om * om / 6.0;
            const double b1 = ((3.0 * u - 6.0) * u * u + 4.0) / 6.0;
            const double b2 = (((-3.0 * u + 3.0) * u + 3.0) * u + 1.0) / 6.0;
            const double b3 = u * u * u / 6.0;
            const int o = lerp_base(d) + 3 * r;
            t.w[o + 0] = static_cast<float>(b2 + b3);
            t.w[o + 1] = static_cast<float>(b1 / (b0 + b1));
            t.w[o + 2] = static_cast<float>(b3 / (b2 + b3));
        }
    return t;
}

static __constant__ LerpTable c_lerp = make_lerp_table();

__device__ __forceinline__ float lerp(float a, float b, float t) { return fmaf(t, b - a, a); }

// One tile (control cell) of one channel: the paper's per-thread loop.
template <bool LERP>
__device__ __forceinline__ void tile_channel(const InstDesc& d, int cx, int cy, int cz, int c, float* __restrict__ out,
                                             unsigned* err) {
    float p[4][4][4];   // [n][m][l]: z, y, x
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const long long e = phi_elem(d, cz + n, cy + m, cx + l) + c;
                BSI_GUARD(e >= 0 && e < 3LL * d.nx * d.ny * d.nz, kErrPhiRead, err) { p[n][m][l] = __ldg(d.phi + e); }
            }
    const int x0 = cx * d.dx, y0 = cy * d.dy, z0 = cz * d.dz;
    const int xn = imin(d.dx, d.X - x0), yn = imin(d.dy, d.Y - y0), zn = imin(d.dz, d.Z - z0);
    for (int rz = 0; rz < zn; ++rz)
        for (int ry = 0; ry < yn; ++ry)
            for (int rx = 0; rx < xn; ++rx) {
                float v;
                if (!LERP) {
                    const float* bu = &c_lut.w[weight_base(d.dx) + 4 * rx];
                    const float* bv = &c_lut.w[weight_base(d.dy) + 4 * ry];
                    const float* bw = &c_lut.w[weight_base(d.dz) + 4 * rz];
                    v = 0.f;
#pragma unroll
                    for (int n = 0; n < 4; ++n)
#pragma unroll
                        for (int m = 0; m < 4; ++m)
#pragma unroll
                            for (int l = 0; l < 4; ++l) v = fmaf(bu[l] * bv[m] * bw[n], p[n][m][l], v);
                } else {
                    const float* lu = &c_lerp.w[lerp_base(d.dx) + 3 * rx];
                    const float* lv = &c_lerp.w[lerp_base(d.dy) + 3 * ry];
                    const float* lw = &c_lerp.w[lerp_base(d.dz) + 3 * rz];
                    float s[2][2][2];   // sub-cube (k, j, i) trilinear interpolations
#pragma unroll
                    for (int k = 0; k < 2; ++k)
#pragma unroll
                        for (int j = 0; j < 2; ++j)
#pragma unroll
                            for (int i = 0; i < 2; ++i) {
                                const float hx = lu[1 + i], hy = lv[1 + j], hz = lw[1 + k];
                                const int l0 = 2 * i, m0 = 2 * j, n0 = 2 * k;
                                const float a0 = lerp(p[n0][m0][l0], p[n0][m0][l0 + 1], hx);
                                const float a1 = lerp(p[n0][m0 + 1][l0], p[n0][m0 + 1][l0 + 1], hx);
                                const float a2 = lerp(p[n0 + 1][m0][l0], p[n0 + 1][m0][l0 + 1], hx);
                                const float a3 = lerp(p[n0 + 1][m0 + 1][l0], p[n0 + 1][m0 + 1][l0 + 1], hx);
                                s[k][j][i] = lerp(lerp(a0, a1, hy), lerp(a2, a3, hy), hz);
                            }
                    const float gx = lu[0], gy = lv[0], gz = lw[0];
                    const float b0 = lerp(s[0][0][0], s[0][0][1], gx), b1 = lerp(s[0][1][0], s[0][1][1], gx);
                    const float b2 = lerp(s[1][0][0], s[1][0][1], gx), b3 = lerp(s[1][1][0], s[1][1][1], gx);
                    v = lerp(lerp(b0, b1, gy), lerp(b2, b3, gy), gz);
                }
                const long long o = field_elem(d, z0 + rz, y0 + ry, x0 + rx) + c;
                BSI_GUARD(o >= 0 && o < 3LL * d.X * d.Y * d.Z, kErrFieldWrite, err) { out[o] = v; }
            }
}

// One thread per tile, tiles x-fastest (neighbouring threads share control points in L1).
template <bool LERP>
__global__ void __launch_bounds__(256) bsi_tile_kernel(const __grid_constant__ Batch<1> b) {
    const InstDesc& d = b.inst[0];
    const long long ntiles = (long long)d.ncx * d.ncy * d.ncz;
    float* out = static_cast<float*>(d.field);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += (long long)gridDim.x * blockDim.x) {
        const int cx = (int)(t % d.ncx);
        const long long q = t / d.ncx;
        const int cy = (int)(q % d.ncy), cz = (int)(q / d.ncy);
        for (int c = 0; c < 3; ++c) tile_channel<LERP>(d, cx, cy, cz, c, out, &g_err);
    }
}

cudaError_t launch_forward_tile_variant(const Batch<1>& b, bool lerp, cudaStream_t s, LaunchInfo* info) {
    const void* kern = lerp ? reinterpret_cast<const void*>(bsi_tile_kernel<true>)
                            : reinterpret_cast<const void*>(bsi_tile_kernel<false>);
    KernelFacts f;
    cudaError_t e = kernel_facts(kern, 256, 0, &f);
    if (e != cudaSuccess) return e;
    const InstDesc& d = b.inst[0];
    const long long want = cdiv((long long)d.ncx * d.ncy * d.ncz, 256);
    const long long cap = (long long)f.sms * f.ctas_per_sm;
    const int grid = (int)(want < cap ? want : cap);
    if (info) *info = LaunchInfo{grid, 256, 0, f.ctas_per_sm};
    if (grid <= 0) return cudaSuccess;
    if (lerp) bsi_tile_kernel<true><<<grid, 256, 0, s>>>(b);
    else bsi_tile_kernel<false><<<grid, 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t variants_err_read_clear(unsigned* out, cudaStream_t s) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_err, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_err);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(p, 0, sizeof(unsigned), s);
}

}  // namespace bsi
