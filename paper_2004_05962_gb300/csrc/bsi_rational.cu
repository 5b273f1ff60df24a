// bsi_rational.cu -- Eq. 1 for control grids that are not aligned to the voxel
// grid: per axis a spacing of num/den voxels and a lattice shift of off/den
// voxels (the paper's future work, Sec. 8: such grids need the B-spline weights
// computed on the fly instead of from look-up tables).  Cell and offset of
// voxel x: q = x den + off, f = floor(q / num), u = (q - f num) / num, computed
// in integers exactly, u rounded once to FP32.
//
// Three forward kernels:
// - bsi_rational_strip_kernel (x-cells of 4 to 8 voxels whose 29-cell strips
//   are mostly full): the integer path's decomposition with cells of varying
//   width.  A warp takes the voxels of one
//   z-cell x one y-cell x a strip of 29 x-cells; lane = stored grid column,
//   whose 4 x 4 control points it contracts over z and y in registers; the
//   x stage gets the three neighbouring columns by shuffles, and each lane
//   writes the (floor or ceil of num/den) voxels of its cell into a staging row
//   that leaves by bulk copy.
// - bsi_rational_window_kernel (other x-spacings, nx <= 1024): a warp takes a run
//   of rows of a plane; the lanes contract the grid over z into a ring of four
//   grid rows and over y into a line of nx columns in shared memory, then walk
//   the row voxel by voxel (consecutive lanes, consecutive voxels).
// - bsi_rational_kernel (other x-spacings, nx > 1024): the same walk, one warp per
//   row, the line built from the grid directly.  Each lane advances its cell
//   and remainder by exact integer steps (32 den = a num + b), so there is no
//   integer division per voxel.
// All three sum in the same order (z, then y, then x; lowest tap first), so
// they give bit-identical fields.  The adjoint (two kernels, deterministic)
// follows the strip kernel's decomposition; see its section below.
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

// ---------------------------------------------------------------- strip kernel

// The strip kernel takes channels 0 and 1 through packed FP32x2 arithmetic
// (combine4; bitwise the scalar results): 2% faster at spacings 4.7 and 6.5 on
// a 512 x 512 x 300 volume.  The adjoint stays scalar: packed, it ran 1.4-2.6%
// slower there.
constexpr bool kRatFwdPacked = true;
constexpr bool kRatAdjPacked = false;

constexpr int kRatStripMaxCell = 8;                            // voxels per x-cell (ceil(num/den)) it takes
constexpr int kRatStripMinCell = 4;                            // x-spacing num/den it takes, at least
constexpr int kRatStripVox = kGroupCells * kRatStripMaxCell;   // voxels of one staged row segment
constexpr int kRatStripBuf = 12 * kRatStripVox + 16;           // + the segment's 16-byte phase
constexpr int kRatStripWarps = 8;
constexpr int kRatTableMaxX = 2048;   // x cells and weights tabulated per CTA up to this width
constexpr int kRatCellMax = 64;   // rows (planes) of a y-cell (z-cell): spacing <= 64
constexpr int kRatWeightBytes = 2 * kRatCellMax * 16;   // per warp: the unit's y and z weights

// First voxel of cell k on one axis: the least x with x den + off >= k num.
__device__ __forceinline__ int cell_first(int k, int num, int den, int off) {
    const long long t = (long long)k * num - off;
    return t <= 0 ? 0 : (int)((t + den - 1) / den);
}

// The four weights of voxel x on one axis, given its cell f.
__device__ __forceinline__ void axis_weights(int x, int f, int num, int den, int off, float B[4]) {
    const int r = x * den + off - f * num;
    bspline4(__fdiv_rn((float)r, (float)num), B);
}

// Units: (z-cell kz, part zp of its planes, y-cell jy, x-strip xs), xs fastest,
// so neighbouring warps share grid rows in L1.  ncx / ncy / ncz: cells per
// axis; nsx: strips per row; zsplit: parts per z-cell (more, smaller units when
// a volume has few cells for the resident warps).
// TABLE: the four x weights of every voxel tabulated once per CTA (16 bytes
// per x, after the staging rings); else computed per voxel.  The y and z
// weights of a unit's rows and planes are computed once per unit, one row
// (plane) per lane, into the warp's weight buffer (after the table).
template <bool TABLE, int CMAX>
__global__ void __launch_bounds__(kRatStripWarps * 32, 2)
    bsi_rational_strip_kernel(const __grid_constant__ RatDesc d, int ncx, int ncy, int ncz, int nsx, int zsplit) {
    extern __shared__ __align__(16) unsigned char rstrip[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    unsigned char* stage = rstrip + (size_t)warp * kStoreStages * kRatStripBuf;
    float4* xw = reinterpret_cast<float4*>(rstrip + (size_t)wpc * kStoreStages * kRatStripBuf);
    float4* yw = xw + (TABLE ? d.X : 0) + (size_t)warp * 2 * kRatCellMax;   // the unit's rows, then its planes
    float4* zw = yw + kRatCellMax;
    if (TABLE) {
        for (int x = threadIdx.x; x < d.X; x += blockDim.x) {
            float B[4];
            const int f = (x * d.den[0] + d.off[0]) / d.num[0];
            axis_weights(x, f, d.num[0], d.den[0], d.off[0], B);
            xw[x] = make_float4(B[0], B[1], B[2], B[3]);
        }
        __syncthreads();
    }
    int ring = 0;
    const long long units = (long long)ncz * zsplit * ncy * nsx;
    for (long long un = (long long)blockIdx.x * wpc + warp; un < units; un += (long long)gridDim.x * wpc) {
        const int xs = (int)(un % nsx);
        const long long t = un / nsx;
        const int jy = (int)(t % ncy);
        const long long t2 = t / ncy;
        const int zp = (int)(t2 % zsplit), kz = (int)(t2 / zsplit);
        const int zc0 = cell_first(kz, d.num[2], d.den[2], d.off[2]);
        const int zcn = imin(d.Z, cell_first(kz + 1, d.num[2], d.den[2], d.off[2])) - zc0;
        const int z0 = zc0 + zcn * zp / zsplit, z1 = zc0 + zcn * (zp + 1) / zsplit;   // this part's planes
        const int y0 = cell_first(jy, d.num[1], d.den[1], d.off[1]);
        const int y1 = imin(d.Y, cell_first(jy + 1, d.num[1], d.den[1], d.off[1]));
        __syncwarp();   // the previous unit's weights are read
        for (int i = lane; i < y1 - y0; i += 32) {
            float B[4];
            axis_weights(y0 + i, jy, d.num[1], d.den[1], d.off[1], B);
            yw[i] = make_float4(B[0], B[1], B[2], B[3]);
        }
        for (int i = lane; i < z1 - z0; i += 32) {
            float B[4];
            axis_weights(z0 + i, kz, d.num[2], d.den[2], d.off[2], B);
            zw[i] = make_float4(B[0], B[1], B[2], B[3]);
        }
        __syncwarp();
        // this lane's grid column and (lanes < 29) its cell's voxels [xa, xb)
        const int c0 = xs * kGroupCells, col = c0 + lane;
        const int xa = imin(d.X, cell_first(col, d.num[0], d.den[0], d.off[0]));
        const int xb = (lane < kGroupCells && col < ncx) ? imin(d.X, cell_first(col + 1, d.num[0], d.den[0], d.off[0]))
                                                         : xa;
        // the strip's voxels [sx0, sx1) (warp-uniform)
        const int sx0 = cell_first(c0, d.num[0], d.den[0], d.off[0]);
        const int sx1 = imin(d.X, cell_first(imin(c0 + kGroupCells, ncx), d.num[0], d.den[0], d.off[0]));

        float ph[4][4][3];
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                float a = 0.f, b = 0.f, c = 0.f;
                if (col < d.nx) {
                    const long long e = (((long long)(kz + n) * d.ny + (jy + m)) * d.nx + col) * 3;
                    BSI_GUARD(e >= 0 && e + 3 <= 3LL * d.nx * d.ny * d.nz, kErrPhiRead, &g_err) {
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

        for (int z = z0; z < z1; ++z) {
            const float4 wz = zw[z - z0];
            const float Bz[4] = {wz.x, wz.y, wz.z, wz.w};
            float pz[4][3];
#pragma unroll
            for (int m = 0; m < 4; ++m)
                combine4<3, kRatFwdPacked>(pz[m], Bz[0], Bz[1], Bz[2], Bz[3], ph[0][m], ph[1][m], ph[2][m], ph[3][m]);
            for (int y = y0; y < y1; ++y) {
                const float4 wy = yw[y - y0];
                const float By[4] = {wy.x, wy.y, wy.z, wy.w};
                float p0[3], p1[3], p2[3], p3[3];
                combine4<3, kRatFwdPacked>(p0, By[0], By[1], By[2], By[3], pz[0], pz[1], pz[2], pz[3]);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    p1[c] = __shfl_down_sync(kFull, p0[c], 1);
                    p2[c] = __shfl_down_sync(kFull, p0[c], 2);
                    p3[c] = __shfl_down_sync(kFull, p0[c], 3);
                }
                unsigned char* g = reinterpret_cast<unsigned char*>(d.field + (((long long)z * d.Y + y) * d.X + sx0) * 3);
                const int shift = (int)(reinterpret_cast<uintptr_t>(g) & 15);
                unsigned char* sb = stage + ring * kRatStripBuf + shift;
                ring = ring + 1 == kStoreStages ? 0 : ring + 1;
                // (the ring buffer is free: store_row of the previous row waited for it)
                // CMAX = ceil(num / den) >= xb - xa: a fixed, unrolled trip count
#pragma unroll
                for (int i = 0; i < CMAX; ++i) {
                    const int x = xa + i;
                    if (x >= xb) break;
                    float B[4];
                    if (TABLE) {
                        const float4 w = xw[x];
                        B[0] = w.x;
                        B[1] = w.y;
                        B[2] = w.z;
                        B[3] = w.w;
                    } else {
                        axis_weights(x, col, d.num[0], d.den[0], d.off[0], B);
                    }
                    BSI_GUARD(shift + 12 * (x - sx0) + 12 <= kRatStripBuf && x >= sx0, kErrStage, &g_err) {
                        const uint32_t sv = smem_u32(sb) + 12u * (uint32_t)(x - sx0);
                        float v[3];
                        combine4<3, kRatFwdPacked>(v, B[0], B[1], B[2], B[3], p0, p1, p2, p3);
#pragma unroll
                        for (int c = 0; c < 3; ++c) sts_f32(sv + 4 * c, v[c]);
                    }
                }
                fence_proxy_async_smem();   // this lane's staging writes before the bulk copy reads them
                __syncwarp();
                BSI_GUARD(sx1 > sx0 && shift + 12 * (sx1 - sx0) <= kRatStripBuf, kErrFieldWrite, &g_err) {
                    store_row<4>(sb, g, shift, 12 * (sx1 - sx0), lane);
                }
                __syncwarp();   // lane 0's ring wait precedes every lane's next staging write
            }
        }
    }
    // the staging ring must outlive every bulk copy that reads it
    if (lane == 0) bulk_wait_all<0>();
    __syncwarp();
}

// --------------------------------------------------------------- adjoint
//
// The transpose of Eq. 1 on such a grid (the gradient with respect to the
// control points).  bsi_rational_adjoint_kernel walks units of zc consecutive
// z-cells x one y-cell x a strip of sc x-cells: the unit's gradient rows arrive
// by bulk copy in a ring of kRatAdjStages buffers per warp; lane l < sc gathers
// the voxels of its cell with their four x weights, the column of lane l
// collects the taps of the cells 0..3 lanes below it by shuffles, y is summed
// in registers and z in a rolling window of four grid planes, one of which is
// complete (and written) after each z-cell.  Each unit writes the partial sums
// of its zc + 3 planes x 4 rows x 32 columns; bsi_rational_adjoint_reduce_kernel
// then sums, per control point, the partials of every unit that covers it in
// a fixed order: deterministic, no atomics.

constexpr int kRatAdjStages = 4;
constexpr int kRatAdjWarps = 8;
// Ring buffer bytes for row segments of up to nvox voxels (+ the 16-byte phase
// and the copy's rounding), and a warp's mbarriers + ring.
BSI_HD int rat_adj_buf(int nvox) { return (12 * nvox + 32 + 15) & ~15; }
BSI_HD int rat_adj_warp_bytes(int buf) { return kRatAdjStages * (16 + buf); }
constexpr int kRatAdjMaxZc = 4;          // z-cells per unit, at most
constexpr int kRatAdjMinUnits = 6000;    // fewer z-cells per unit while there are fewer units (device-independent)
constexpr int kRatPartPlane = 4 * 32 * 3;   // partial floats of one grid plane: rows x columns x channels

// One grid plane of a unit's partial sums: [row m][column lane][channel].
__device__ __forceinline__ void rat_flush_plane(float* P, const float (&h)[4][3], int lane) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float* e = P + (m * 32 + lane) * 3;
        e[0] = h[m][0];
        e[1] = h[m][1];
        e[2] = h[m][2];
    }
}

template <bool TABLE, int CMAX>
__global__ void __launch_bounds__(kRatAdjWarps * 32, 2)
    bsi_rational_adjoint_kernel(const __grid_constant__ RatDesc d, const float* __restrict__ grad,
                                float* __restrict__ part, int ncx, int ncy, int ncz, int nsx, int sc, int zc,
                                int buf) {
    extern __shared__ __align__(16) unsigned char radj[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    unsigned char* wsm = radj + (size_t)warp * rat_adj_warp_bytes(buf);
    uint64_t* bars = reinterpret_cast<uint64_t*>(wsm);          // bars[s] in 16-byte slots' first 8 bytes
    unsigned char* bufs = wsm + 16 * kRatAdjStages;
    float4* xw = reinterpret_cast<float4*>(radj + (size_t)wpc * rat_adj_warp_bytes(buf));
    float4* yw = xw + (TABLE ? d.X : 0) + (size_t)warp * 2 * kRatCellMax;   // the unit's rows, then its planes
    float4* zw = yw + kRatCellMax;
    if (lane == 0) {
        for (int st = 0; st < kRatAdjStages; ++st) mbar_init(bars + 2 * st, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (TABLE)
        for (int x = threadIdx.x; x < d.X; x += blockDim.x) {
            float B[4];
            const int f = (x * d.den[0] + d.off[0]) / d.num[0];
            axis_weights(x, f, d.num[0], d.den[0], d.off[0], B);
            xw[x] = make_float4(B[0], B[1], B[2], B[3]);
        }
    __syncthreads();
    const uintptr_t gbase = reinterpret_cast<uintptr_t>(grad);
    const uintptr_t A0 = ceil16(gbase);
    const uintptr_t A1 = floor16(gbase + (uintptr_t)(12LL * d.X * d.Y * d.Z));
    unsigned q = 0;   // row copies this warp has consumed (ring stage and phase)
    bool ok = true;
    const long long nch = cdiv(ncz, zc);
    const long long units = nch * ncy * nsx;
    for (long long un = (long long)blockIdx.x * wpc + warp; ok && un < units; un += (long long)gridDim.x * wpc) {
        const int xs = (int)(un % nsx);
        const long long t = un / nsx;
        const int jy = (int)(t % ncy);
        const int kz0 = (int)(t / ncy) * zc, kz1 = imin(kz0 + zc, ncz);
        const int z0 = cell_first(kz0, d.num[2], d.den[2], d.off[2]);
        const int z1 = imin(d.Z, cell_first(kz1, d.num[2], d.den[2], d.off[2]));
        const int y0 = cell_first(jy, d.num[1], d.den[1], d.off[1]);
        const int y1 = imin(d.Y, cell_first(jy + 1, d.num[1], d.den[1], d.off[1]));
        const int c0 = xs * sc, col = c0 + lane;
        const bool owns = lane < sc && col < ncx;
        const int xa = owns ? cell_first(col, d.num[0], d.den[0], d.off[0]) : 0;
        const int xb = owns ? imin(d.X, cell_first(col + 1, d.num[0], d.den[0], d.off[0])) : 0;
        const int sx0 = cell_first(c0, d.num[0], d.den[0], d.off[0]);
        const int sx1 = imin(d.X, cell_first(imin(c0 + sc, ncx), d.num[0], d.den[0], d.off[0]));
        const int nbytes = 12 * (sx1 - sx0);
        const int nyu = y1 - y0, rows = (z1 - z0) * nyu;
        __syncwarp();   // the previous unit's weights are read
        for (int i = lane; i < nyu; i += 32) {
            float B[4];
            axis_weights(y0 + i, jy, d.num[1], d.den[1], d.off[1], B);
            yw[i] = make_float4(B[0], B[1], B[2], B[3]);
        }
        // the planes' weights (z1 - z0 <= zc ceil(num / den) <= kRatCellMax: the plan's bound)
        for (int i = lane; i < z1 - z0; i += 32) {
            float B[4];
            const int z = z0 + i;
            axis_weights(z, (z * d.den[2] + d.off[2]) / d.num[2], d.num[2], d.den[2], d.off[2], B);
            zw[i] = make_float4(B[0], B[1], B[2], B[3]);
        }
        __syncwarp();

        // row k of the unit: plane z0 + k / nyu, row y0 + k % nyu, voxels [sx0, sx1)
        const unsigned q0 = q;
        auto row_addr = [&](int k) -> uintptr_t {
            const long long z = z0 + k / nyu, y = y0 + k % nyu;
            return gbase + (uintptr_t)(12LL * ((z * d.Y + y) * d.X + sx0));
        };
        auto issue = [&](int k) {   // lane 0: row k into ring stage (q0 + k) % kRatAdjStages
            const unsigned st = (q0 + (unsigned)k) % kRatAdjStages;
            const RowLoad L = row_load(reinterpret_cast<const unsigned char*>(row_addr(k)), nbytes, A0, A1);
            if (L.s1 > L.s0) {
                mbar_arrive_expect_tx(bars + 2 * st, (uint32_t)(L.s1 - L.s0));
                bulk_load(bufs + st * buf + (L.s0 - L.lo), reinterpret_cast<const void*>(L.s0),
                          (uint32_t)(L.s1 - L.s0), bars + 2 * st);
            } else {
                mbar_arrive(bars + 2 * st);
            }
        };
        if (lane == 0)
            for (int k = 0; k < rows && k < kRatAdjStages; ++k) issue(k);

        float hz[4][4][3];
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int c = 0; c < 3; ++c) hz[n][m][c] = 0.f;
        float* P = part + un * (long long)(zc + 3) * kRatPartPlane;   // the unit's planes kz0 .. kz0 + zc + 2
        int k = 0;
        for (int kz = kz0; ok && kz < kz1; ++kz) {
            const int zb = imax(z0, cell_first(kz, d.num[2], d.den[2], d.off[2]));
            const int ze = imin(z1, cell_first(kz + 1, d.num[2], d.den[2], d.off[2]));
            for (int z = zb; ok && z < ze; ++z) {
                float hy[4][3];
#pragma unroll
                for (int m = 0; m < 4; ++m)
#pragma unroll
                    for (int c = 0; c < 3; ++c) hy[m][c] = 0.f;
                for (int y = y0; y < y1; ++y, ++k) {
                    const unsigned qq = q0 + (unsigned)k, st = qq % kRatAdjStages;
                    if (!mbar_wait_bounded(bars + 2 * st, (qq / kRatAdjStages) & 1u)) {
                        // a bulk copy never completed: record it, give the copies still in
                        // flight a bounded chance to land, and stop this warp
                        if (lane == 0) atomicOr(&g_err, kErrTimeout);
                        for (int p = k + 1; p < rows && p < k + kRatAdjStages; ++p) {
                            const unsigned qp = q0 + (unsigned)p;
                            (void)mbar_wait_bounded(bars + 2 * (qp % kRatAdjStages), (qp / kRatAdjStages) & 1u);
                        }
                        ok = false;
                        break;
                    }
                    const uintptr_t g = row_addr(k);
                    unsigned char* sb = bufs + st * buf + (g & 15);
                    if (g < A0 || g + (uintptr_t)nbytes > A1) {
                        // first or last row of the array: its elements outside the bulk copy
                        const RowLoad L = row_load(reinterpret_cast<const unsigned char*>(g), nbytes, A0, A1);
                        for (int i = lane; i < nbytes / 4; i += 32) {
                            const uintptr_t a = g + 4u * (uintptr_t)i;
                            if (a < L.s0 || a >= L.s1) reinterpret_cast<float*>(sb)[i] = *reinterpret_cast<const float*>(a);
                        }
                    }
                    __syncwarp();
                    float q4[4][3];
#pragma unroll
                    for (int l = 0; l < 4; ++l)
#pragma unroll
                        for (int c = 0; c < 3; ++c) q4[l][c] = 0.f;
                    // x-transpose of the lane's cell: q_l += B_l(x) G(x), voxels in order
                    auto gather = [&](int x) {
                        float B[4];
                        if (TABLE) {
                            const float4 w = xw[x];
                            B[0] = w.x;
                            B[1] = w.y;
                            B[2] = w.z;
                            B[3] = w.w;
                        } else {
                            axis_weights(x, col, d.num[0], d.den[0], d.off[0], B);
                        }
                        BSI_GUARD(x >= sx0 && (int)(g & 15) + 12 * (x - sx0) + 12 <= buf, kErrStage, &g_err) {
                            const uint32_t sv = smem_u32(sb) + 12u * (uint32_t)(x - sx0);
                            const float g0 = lds_f32(sv), g1 = lds_f32(sv + 4), g2 = lds_f32(sv + 8);
#pragma unroll
                            for (int l = 0; l < 4; ++l) fma3_sel<kRatAdjPacked>(q4[l], B[l], g0, g1, g2);
                        }
                    };
                    if (CMAX > 0) {   // CMAX >= ceil(num / den) >= xb - xa: unrolled
#pragma unroll
                        for (int i = 0; i < (CMAX > 0 ? CMAX : 1); ++i) {
                            if (xa + i >= xb) break;
                            gather(xa + i);
                        }
                    } else {
                        for (int x = xa; x < xb; ++x) gather(x);
                    }
                    // this ring buffer may be refilled once every lane has read it
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0 && k + kRatAdjStages < rows) issue(k + kRatAdjStages);
                    // column sums: column c0 + lane collects tap l of the cell l lanes below
                    const float4 wy = yw[y - y0];
                    const float By[4] = {wy.x, wy.y, wy.z, wy.w};
                    float h[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float t1 = __shfl_up_sync(kFull, q4[1][c], 1);
                        const float t2 = __shfl_up_sync(kFull, q4[2][c], 2);
                        const float t3 = __shfl_up_sync(kFull, q4[3][c], 3);
                        h[c] = q4[0][c] + (lane >= 1 ? t1 : 0.f) + (lane >= 2 ? t2 : 0.f) + (lane >= 3 ? t3 : 0.f);
                    }
#pragma unroll
                    for (int m = 0; m < 4; ++m) fma3_sel<kRatAdjPacked>(hy[m], By[m], h[0], h[1], h[2]);
                }
                if (!ok) break;
                const float4 wz = zw[z - z0];
                const float Bz[4] = {wz.x, wz.y, wz.z, wz.w};
#pragma unroll
                for (int n = 0; n < 4; ++n)
#pragma unroll
                    for (int m = 0; m < 4; ++m) fma3_sel<kRatAdjPacked>(hz[n][m], Bz[n], hy[m][0], hy[m][1], hy[m][2]);
            }
            if (!ok) break;
            // grid plane kz is complete for this unit: write it, roll the window by one plane
            rat_flush_plane(P + (kz - kz0) * kRatPartPlane, hz[0], lane);
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
        q = q0 + (unsigned)rows;
        if (!ok) break;
        // planes kz1 .. kz1 + 2 get contributions from this unit's last cells only
#pragma unroll
        for (int n = 0; n < 3; ++n) rat_flush_plane(P + (kz1 - kz0 + n) * kRatPartPlane, hz[n], lane);
    }
    __syncwarp();
    if (lane == 0)
        for (int st = 0; st < kRatAdjStages; ++st) mbar_inval(bars + 2 * st);
}

// One thread per stored control point (gx, gy, gz): the units that cover it are
// the z-chunks whose planes [kz0, kz0 + cells + 3) hold gz, y-cells jy = gy - m
// (m = 0..3), and the strips xs whose 32 columns [xs sc, xs sc + 32) hold gx.
__global__ void __launch_bounds__(256, 4)
    bsi_rational_adjoint_reduce_kernel(const __grid_constant__ RatDesc d, const float* __restrict__ part,
                                       float* __restrict__ dphi, int ncy, int ncz, int nsx, int sc, int zc) {
    const long long npts = (long long)d.nx * d.ny * d.nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npts; p += stride) {
        const int gx = (int)(p % d.nx);
        const long long t = p / d.nx;
        const int gy = (int)(t % d.ny), gz = (int)(t / d.ny);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        const int nch = (ncz + zc - 1) / zc;
        for (int ch = imin(nch - 1, gz / zc); ch >= 0; --ch) {
            const int pz = gz - ch * zc;                  // plane slot within the chunk
            if (pz >= imin(zc, ncz - ch * zc) + 3) break;  // beyond the chunk's planes (and every earlier chunk's)
            for (int jy = imax(0, gy - 3); jy <= imin(gy, ncy - 1); ++jy)
                for (int xs = imin(nsx - 1, gx / sc); xs >= 0 && gx - xs * sc < 32; --xs) {
                    const long long un = ((long long)ch * ncy + jy) * nsx + xs;
                    const float* e = part + un * (long long)(zc + 3) * kRatPartPlane +
                                     ((pz * 4 + (gy - jy)) * 32 + (gx - xs * sc)) * 3;
                    s0 += e[0];
                    s1 += e[1];
                    s2 += e[2];
                }
        }
        dphi[3 * p] = s0;
        dphi[3 * p + 1] = s1;
        dphi[3 * p + 2] = s2;
    }
}

// Cells per axis, strips and z-parts of the adjoint's units (host, shared with
// the workspace query).
RatAdjPlan rational_adjoint_plan(const RatDesc& d) {
    RatAdjPlan pl;
    pl.ncx = (int)(((long long)(d.X - 1) * d.den[0] + d.off[0]) / d.num[0]) + 1;
    pl.ncy = (int)(((long long)(d.Y - 1) * d.den[1] + d.off[1]) / d.num[1]) + 1;
    pl.ncz = (int)(((long long)(d.Z - 1) * d.den[2] + d.off[2]) / d.num[2]) + 1;
    const int cmax = (d.num[0] + d.den[0] - 1) / d.den[0];
    pl.sc = imin(kGroupCells, kRatStripVox / cmax);
    pl.nsx = (int)cdiv(pl.ncx, pl.sc);
    // a unit's planes (at most zc ceil(num_z / den_z)) fit the kernel's weight buffer
    const int zmax = (d.num[2] + d.den[2] - 1) / d.den[2];
    pl.zc = kRatAdjMaxZc;
    while (pl.zc > 1 && (cdiv(pl.ncz, pl.zc) * pl.ncy * pl.nsx < kRatAdjMinUnits || pl.zc * zmax > kRatCellMax))
        pl.zc /= 2;
    pl.part_floats = cdiv(pl.ncz, pl.zc) * pl.ncy * pl.nsx * (pl.zc + 3) * kRatPartPlane;
    return pl;
}

cudaError_t launch_adjoint_rational(const RatDesc& d, const float* grad, float* dphi, float* part,
                                    cudaStream_t s) {
    const RatAdjPlan pl = rational_adjoint_plan(d);
    const int cmax = (d.num[0] + d.den[0] - 1) / d.den[0];
    const bool table = d.X <= kRatTableMaxX;
    const int table_bytes = table ? 16 * d.X : 0;
    const int buf = rat_adj_buf(pl.sc * cmax);   // a strip holds at most sc cells of cmax voxels
    const int per_warp = rat_adj_warp_bytes(buf) + 2 * kRatCellMax * 16;
    int wpc = (kSmemBudget - table_bytes) / per_warp;
    wpc = wpc < 1 ? 1 : (wpc > kRatAdjWarps ? kRatAdjWarps : wpc);
    const int threads = wpc * 32, smem = wpc * per_warp + table_bytes;
    const void* kern = nullptr;
#define BSI_RAT_ADJ_KERN(CM)                                                                      \
    kern = table ? reinterpret_cast<const void*>(bsi_rational_adjoint_kernel<true, CM>)           \
                 : reinterpret_cast<const void*>(bsi_rational_adjoint_kernel<false, CM>)
    if (cmax <= 4) BSI_RAT_ADJ_KERN(4);
    else if (cmax <= 8) BSI_RAT_ADJ_KERN(8);
    else BSI_RAT_ADJ_KERN(0);
#undef BSI_RAT_ADJ_KERN
    KernelFacts f;
    cudaError_t e = kernel_facts(kern, threads, smem, &f);
    if (e != cudaSuccess) return e;
    const long long units = pl.part_floats / ((pl.zc + 3) * kRatPartPlane);
    const long long want = cdiv(units, wpc);
    const long long cap = (long long)f.sms * f.ctas_per_sm;
    const int grid = (int)(want < cap ? want : cap);
    if (grid > 0) {
        int ncx = pl.ncx, ncy = pl.ncy, ncz = pl.ncz, nsx = pl.nsx, sc = pl.sc, zc = pl.zc, bufb = buf;
        const float* gptr = grad;
        void* args[] = {const_cast<RatDesc*>(&d), (void*)&gptr, (void*)&part, (void*)&ncx, (void*)&ncy,
                        (void*)&ncz, (void*)&nsx, (void*)&sc, (void*)&zc, (void*)&bufb};
        e = cudaLaunchKernel(kern, dim3(grid), dim3(threads), args, (size_t)smem, s);
        if (e != cudaSuccess) return e;
    }
    const long long npts = (long long)d.nx * d.ny * d.nz;
    const long long rgrid = cdiv(npts, 256);
    const int rg = (int)(rgrid < 4LL * f.sms * 8 ? rgrid : 4LL * f.sms * 8);
    if (rg > 0)
        bsi_rational_adjoint_reduce_kernel<<<rg, 256, 0, s>>>(d, part, dphi, pl.ncy, pl.ncz, pl.nsx, pl.sc, pl.zc);
    return cudaGetLastError();
}

// Rows per warp of the windowed kernel, and the grid widths it takes (its
// shared memory per warp: 4 z-contracted grid rows + the line, 60 nx bytes).
constexpr int kRatRun = 16;
constexpr int kRatWindowMaxNx = 1024;

// A warp takes a run of `run` (<= kRatRun) consecutive rows of one voxel plane z.  It keeps
// the z-contraction of the four grid rows the current row needs,
//   P[g'][col] = sum_n Bz[n] phi[fz+n][g'][col]   (g' = fy .. fy+3, a ring of 4),
// and adds one grid row whenever the row's cell fy advances (spacing >= 1: at
// most one per row), so each output row's line costs 4 taps from shared memory
// instead of 16 grid reads.  Same arithmetic per voxel as bsi_rational_kernel.
template <bool TABLE>
__global__ void __launch_bounds__(kRatWarps * 32) bsi_rational_window_kernel(const __grid_constant__ RatDesc d, int run) {
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
    const int runs_y = (d.Y + run - 1) / run;
    const long long units = (long long)d.Z * runs_y;
    for (long long un = (long long)blockIdx.x * wpc + warp; un < units; un += (long long)gridDim.x * wpc) {
        const int z = (int)(un / runs_y), ya = (int)(un % runs_y) * run, yb = imin(ya + run, d.Y);
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
    // The strip kernel for x-cells of 4 to 8 voxels whose strips are mostly full
    // (a strip costs the same with few cells as with 29).  Measured on 256- to
    // 512-voxel rows: 1.2-1.5x faster than the windowed kernel at spacing
    // 4.3-5; slower at 3.3 (the per-row work of a strip outweighs its voxels)
    // and at 6.5 on 256 voxels (40 cells in two strips).
    const int ncx = (int)(((long long)(d.X - 1) * d.den[0] + d.off[0]) / d.num[0]) + 1;
    const int nsx = (int)cdiv(ncx, kGroupCells);
    if (d.num[0] >= kRatStripMinCell * d.den[0] && (d.num[0] + d.den[0] - 1) / d.den[0] <= kRatStripMaxCell &&
        4 * ncx >= 3 * kGroupCells * nsx) {
        const int ncy = (int)(((long long)(d.Y - 1) * d.den[1] + d.off[1]) / d.num[1]) + 1;
        const int ncz = (int)(((long long)(d.Z - 1) * d.den[2] + d.off[2]) / d.num[2]) + 1;
        const bool table = d.X <= kRatTableMaxX;
        const int ring_bytes = kStoreStages * kRatStripBuf;
        const int table_bytes = table ? 16 * d.X : 0;
        int wpc = (kSmemBudget - table_bytes) / (ring_bytes + kRatWeightBytes);
        wpc = wpc < 1 ? 1 : (wpc > kRatStripWarps ? kRatStripWarps : wpc);
        const int threads = wpc * 32, smem = wpc * (ring_bytes + kRatWeightBytes) + table_bytes;
        const int cmax = (d.num[0] + d.den[0] - 1) / d.den[0];   // 4 .. 8
        const void* kern = nullptr;
        switch (cmax) {
#define BSI_RAT_STRIP_KERN(CM)                                                                      \
    case CM:                                                                                        \
        kern = table ? reinterpret_cast<const void*>(bsi_rational_strip_kernel<true, CM>)           \
                     : reinterpret_cast<const void*>(bsi_rational_strip_kernel<false, CM>);         \
        break;
            BSI_RAT_STRIP_KERN(4)
            BSI_RAT_STRIP_KERN(5)
            BSI_RAT_STRIP_KERN(6)
            BSI_RAT_STRIP_KERN(7)
            BSI_RAT_STRIP_KERN(8)
#undef BSI_RAT_STRIP_KERN
            default: return cudaErrorInvalidValue;
        }
        KernelFacts f;
        cudaError_t e = kernel_facts(kern, threads, smem, &f);
        if (e != cudaSuccess) return e;
        // split z-cells while the units are fewer than the resident warps (a short
        // volume has few cells); smaller units cost more per voxel, so no further
        const long long slots = (long long)f.sms * f.ctas_per_sm * wpc;
        int zsplit = 1;
        while (2 * zsplit <= d.num[2] / d.den[2] && (long long)ncz * zsplit * ncy * nsx < slots) zsplit *= 2;
        const long long want = cdiv((long long)ncz * zsplit * ncy * nsx, wpc);
        const long long cap = (long long)f.sms * f.ctas_per_sm;
        const int grid = (int)(want < cap ? want : cap);
        if (info) *info = LaunchInfo{grid, threads, smem, f.ctas_per_sm};
        if (grid <= 0) return cudaSuccess;
        void* args[] = {const_cast<RatDesc*>(&d), (void*)&ncx, (void*)&ncy, (void*)&ncz, (void*)&nsx, (void*)&zsplit};
        return cudaLaunchKernel(kern, dim3(grid), dim3(threads), args, (size_t)smem, s);
        return cudaGetLastError();
    }
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
        // runs of kRatRun rows, shorter while that leaves fewer runs than a quarter
        // of the resident warps (a short, wide volume has few rows)
        const long long slots = (long long)f.sms * f.ctas_per_sm * wpc;
        int run = kRatRun;
        while (run > 1 && 4 * (long long)d.Z * cdiv(d.Y, run) < slots) run >>= 1;
        const long long want = cdiv((long long)d.Z * cdiv(d.Y, run), wpc);
        const long long cap = (long long)f.sms * f.ctas_per_sm;
        const int grid = (int)(want < cap ? want : cap);
        if (info) *info = LaunchInfo{grid, threads, smem, f.ctas_per_sm};
        if (grid <= 0) return cudaSuccess;
        if (table) bsi_rational_window_kernel<true><<<grid, threads, smem, s>>>(d, run);
        else bsi_rational_window_kernel<false><<<grid, threads, smem, s>>>(d, run);
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
