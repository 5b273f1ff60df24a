// bsi_adjoint.cu -- adjoint (transpose of Eq. 1) kernels and their launchers.
//
// Phase 1 (bsi_adjoint_partials_kernel, bsi_adjoint_partials_tma_kernel): each
// warp unit walks a chunk of tile-planes of one tile-row (two on the
// tensor-copy path where chosen) and one x-group and writes the complete-in-x,
// partial-in-y/z sums of its (chunk+3) x (tile-rows+3) x 29 control points.
// Phase 2 (bsi_adjoint_reduce_kernel): each control point sums the <= 2 x 4
// partials that cover it, in a fixed order, and writes grad_phi.
#include "bsi_kernels.cuh"
#include "bsi_launch.h"

namespace bsi {

static __device__ unsigned g_err;

// 4-warp CTAs, 3 per SM: the unit's rolling z window (48 accumulators per lane)
// fits in <= 170 registers without spilling; measured ~4% faster than 8-warp
// CTAs capped at 128 registers.
constexpr int kAdjMaxWarps = kAdjWarpsMax;

template <int MAXB, bool GENERIC>
__global__ void __launch_bounds__(kAdjMaxWarps * kLanes, 3)
    bsi_adjoint_partials_kernel(const __grid_constant__ Batch<MAXB> b, float* __restrict__ part,
                                long long ws_floats) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & (kLanes - 1);
    const int warp = threadIdx.x >> 5;
    unsigned char* wsm = smem + (size_t)warp * adj_warp_smem(b.buf_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(wsm);           // mbarrier of stage s: bars[s]
    unsigned char* bufs = wsm + 16 * kLoadStages;                 // kLoadStages ring buffers
    if (lane == 0) {
        for (int s = 0; s < kLoadStages; ++s) mbar_init(bars + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    asm volatile("griddepcontrol.wait;" ::: "memory");   // the previous kernel's writes are visible
    const int wpc = blockDim.x >> 5;
    int ii = 0;
    unsigned q = 0;
    for (long long r = 0;; ++r) {
        const long long uu = slot_unit(r, blockIdx.x, warp, gridDim.x, wpc, b.total_units);
        if (uu < 0) break;
        while (ii + 1 < b.n && uu >= b.inst[ii + 1].unit_begin) ++ii;
        const InstDesc& d = b.inst[ii];
        const long long ul = uu - d.unit_begin;
        bool ok;
        if (GENERIC) {
            ok = adjoint_unit<0>(d, ul, bars, bufs, b.buf_bytes, lane, q, part, ws_floats, &g_err);
        } else {
            switch (d.dx) {
                case 1: ok = adjoint_unit<1>(d, ul, bars, bufs, b.buf_bytes, lane, q, part, ws_floats, &g_err); break;
                case 2: ok = adjoint_unit<2>(d, ul, bars, bufs, b.buf_bytes, lane, q, part, ws_floats, &g_err); break;
                case 3: ok = adjoint_unit<3>(d, ul, bars, bufs, b.buf_bytes, lane, q, part, ws_floats, &g_err); break;
                case 4: ok = adjoint_unit<4>(d, ul, bars, bufs, b.buf_bytes, lane, q, part, ws_floats, &g_err); break;
                case 5: ok = adjoint_unit<5>(d, ul, bars, bufs, b.buf_bytes, lane, q, part, ws_floats, &g_err); break;
                case 6: ok = adjoint_unit<6>(d, ul, bars, bufs, b.buf_bytes, lane, q, part, ws_floats, &g_err); break;
                case 7: ok = adjoint_unit<7>(d, ul, bars, bufs, b.buf_bytes, lane, q, part, ws_floats, &g_err); break;
                default: ok = adjoint_unit<8>(d, ul, bars, bufs, b.buf_bytes, lane, q, part, ws_floats, &g_err); break;
            }
        }
        if (!ok) break;  // a lost bulk copy: the error word says so; stop this warp
    }
    __syncwarp();
    if (lane == 0)
        for (int s = 0; s < kLoadStages; ++s) mbar_inval(bars + s);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   // as in the tensor-copy kernel
}

// Tensor-copy path (adjoint_unit_tma): x-spacing <= 8, dy <= 8, X % 4 == 0.
// One CTA per SM with as many warps as the stage rings fit in shared memory;
// warp w's ring of b.stages stages of b.buf_bytes sits after its 128 bytes of
// mbarriers.
template <int MAXB, int JR>
__global__ void __launch_bounds__((JR == 1 ? kTmaMaxWarps : kTmaMaxWarps2) * kLanes, 1)
    bsi_adjoint_partials_tma_kernel(const __grid_constant__ Batch<MAXB> b, const __grid_constant__ TmaMaps<MAXB> maps,
                                    float* __restrict__ part, long long ws_floats) {
    extern __shared__ __align__(128) unsigned char tsmem[];
    const int lane = threadIdx.x & (kLanes - 1);
    const int warp = threadIdx.x >> 5;
    // tensor copies land on 128-byte boundaries: round the base up (the launch
    // allocates 128 spare bytes for this)
    unsigned char* base = tsmem + ((128u - (smem_u32(tsmem) & 127u)) & 127u);
    unsigned char* wsm = base + (size_t)warp * tma_warp_smem(b.buf_bytes, b.stages);
    uint64_t* bars = reinterpret_cast<uint64_t*>(wsm);
    unsigned char* ring = wsm + 128;
    BSI_GUARD((smem_u32(ring) & 127) == 0 && (b.buf_bytes & 127) == 0 && b.stages >= 1 && b.stages <= kTmaMaxStages,
              kErrStage, &g_err) {}
    if (lane == 0) {
        for (int s = 0; s < b.stages; ++s) mbar_init(bars + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    asm volatile("griddepcontrol.wait;" ::: "memory");   // the previous kernel's writes are visible
    const int wpc = blockDim.x >> 5;
    int ii = 0;
    unsigned q = 0;
    for (long long r = 0;; ++r) {
        const long long uu = slot_unit(r, blockIdx.x, warp, gridDim.x, wpc, b.total_units);
        if (uu < 0) break;
        while (ii + 1 < b.n && uu >= b.inst[ii + 1].unit_begin) ++ii;
        const InstDesc& d = b.inst[ii];
        const void* tm = &maps.m[ii];
        const long long ul = uu - d.unit_begin;
        bool ok;
        switch (d.dx) {
            case 1: ok = adjoint_unit_tma<1, JR>(d, tm, ul, bars, ring, b.buf_bytes, b.stages, lane, q, part, ws_floats, &g_err); break;
            case 2: ok = adjoint_unit_tma<2, JR>(d, tm, ul, bars, ring, b.buf_bytes, b.stages, lane, q, part, ws_floats, &g_err); break;
            case 3: ok = adjoint_unit_tma<3, JR>(d, tm, ul, bars, ring, b.buf_bytes, b.stages, lane, q, part, ws_floats, &g_err); break;
            case 4: ok = adjoint_unit_tma<4, JR>(d, tm, ul, bars, ring, b.buf_bytes, b.stages, lane, q, part, ws_floats, &g_err); break;
            case 5: ok = adjoint_unit_tma<5, JR>(d, tm, ul, bars, ring, b.buf_bytes, b.stages, lane, q, part, ws_floats, &g_err); break;
            case 6: ok = adjoint_unit_tma<6, JR>(d, tm, ul, bars, ring, b.buf_bytes, b.stages, lane, q, part, ws_floats, &g_err); break;
            case 7: ok = adjoint_unit_tma<7, JR>(d, tm, ul, bars, ring, b.buf_bytes, b.stages, lane, q, part, ws_floats, &g_err); break;
            default: ok = adjoint_unit_tma<8, JR>(d, tm, ul, bars, ring, b.buf_bytes, b.stages, lane, q, part, ws_floats, &g_err); break;
        }
        if (!ok) break;  // a lost box: the error word says so; stop this warp
    }
    __syncwarp();
    if (lane == 0)
        for (int s = 0; s < b.stages; ++s) mbar_inval(bars + s);
    // this CTA's partial sums are written: the reduce grid may be scheduled
    // (it still waits for this whole grid before reading them)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// One thread per stored control point of every instance.  The units that
// cover point (gx, gy, gz): x-group gx / 29 (columns are complete within a
// unit), the units whose tile-rows [jy, jy + jrows) reach grid row gy (tile-rows
// gy - 3 .. gy), and the tile-plane chunks whose plane window [chunk start,
// chunk start + planes + 3) contains gz.
template <int MAXB, int JR>
__global__ void __launch_bounds__(256)
    bsi_adjoint_reduce_kernel(const __grid_constant__ Batch<MAXB> b, const float* __restrict__ part,
                              long long ws_floats) {
    // launched as a programmatic dependent of the partials kernel: wait here until
    // that grid has finished and its partial sums are visible (a no-op otherwise)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < b.total_points; p += stride) {
        int lo = 0, hi = b.n - 1;  // last instance with point_begin <= p
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.inst[mid].point_begin <= p) lo = mid;
            else hi = mid - 1;
        }
        const InstDesc& d = b.inst[lo];
        const long long pl = p - d.point_begin;
        int gx, gy, gz;
        if (pl < 0xFFFFFFFFLL) {   // 32-bit division (64-bit division is a long sequence)
            const unsigned u = (unsigned)pl, t = u / (unsigned)d.nx;
            gx = (int)(u - t * (unsigned)d.nx);
            gy = (int)(t % (unsigned)d.ny);
            gz = (int)(t / (unsigned)d.ny);
        } else {
            const long long t = pl / d.nx;
            gx = (int)(pl - t * d.nx);
            gy = (int)(t % d.ny);
            gz = (int)(t / d.ny);
        }
        const int xg = gx / kGroupCells, j = gx - xg * kGroupCells;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        if (d.nzc > 0) {
            // The covering partials: at most two tile-plane chunks (zc_hi - 1, zc_hi)
            // times four unit rows, uy0 - q (q = 0..3), each holding grid row gy as its
            // row m0 + q jrows when that is below jrows + 3.  Their offsets differ by
            // constants of the instance: e(t, q) = e(0, 0) + t sz - q sy (part_elem
            // written out), so one 64-bit offset per point and adds give all eight.
            // All 8 x 3 loads are issued before any sum, and the sum runs in the
            // fixed order (chunk, row); channels 0 and 1 are added as packed pairs
            // (bitwise the scalar sums).
            const int zc_hi = imin(d.nzc - 1, gz / d.zchunk);
            constexpr int jr = JR, nr = JR + kHalo;   // every instance of a launch has JR tile-rows per unit
            const int uy0 = JR == 2 ? gy >> 1 : gy, m0 = gy - uy0 * JR;
            const long long uf = adj_unit_floats(d);
            const long long sy = (long long)d.nxg * uf - (long long)jr * kGroupCells * 3;   // one unit row less
            const long long sz = (long long)d.ncyu * d.nxg * uf - (long long)d.zchunk * nr * kGroupCells * 3;  // next chunk
            const int zc0 = zc_hi - 1, pz0 = gz - zc0 * d.zchunk;
            const long long e00 = d.part_off + (((long long)zc0 * d.ncyu + uy0) * d.nxg + xg) * uf +
                                  (((long long)pz0 * nr + m0) * kGroupCells + j) * 3;
            float v[2][4][3];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int zc = zc0 + t;
                const bool zok = zc >= 0 && pz0 - t * d.zchunk < imin(d.zchunk, d.ncz - zc * d.zchunk) + kHalo;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int uy = uy0 - q;
                    v[t][q][0] = v[t][q][1] = v[t][q][2] = 0.f;
                    if (zok && uy >= 0 && uy < d.ncyu && m0 + q * jr < nr) {
                        const long long e = e00 + t * sz - q * sy;
                        BSI_GUARD(e >= 0 && e + 3 <= ws_floats, kErrPartRead, &g_err) {
                            v[t][q][0] = __ldcs(part + e);
                            v[t][q][1] = __ldcs(part + e + 1);
                            v[t][q][2] = __ldcs(part + e + 2);
                        }
                    }
                }
            }
            float2 a = make_float2(s0, s1);
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    a = __fadd2_rn(a, make_float2(v[t][m][0], v[t][m][1]));
                    s2 += v[t][m][2];
                }
            s0 = a.x;
            s1 = a.y;
        }
        float* o = d.dphi + pl * 3;
        BSI_GUARD(pl >= 0 && pl < (long long)d.nx * d.ny * d.nz, kErrDphiWrite, &g_err) {
            o[0] = s0;
            o[1] = s1;
            o[2] = s2;
        }
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   // this CTA's points are written
}

template <int MAXB, bool GENERIC>
static cudaError_t launch_part_t(const Batch<MAXB>& b, float* part, long long ws_floats, cudaStream_t s,
                                 LaunchInfo* info) {
    auto kern = bsi_adjoint_partials_kernel<MAXB, GENERIC>;
    const int wpc = warps_per_cta(adj_warp_smem(b.buf_bytes),
                                  b.warps_req > 0 && b.warps_req < kAdjMaxWarps ? b.warps_req : kAdjMaxWarps);
    const int threads = wpc * kLanes;
    const int smem = wpc * adj_warp_smem(b.buf_bytes);
    KernelFacts f;
    cudaError_t e = kernel_facts(reinterpret_cast<const void*>(kern), threads, smem, &f);
    if (e != cudaSuccess) return e;
    const long long want = cdiv(b.total_units, wpc);
    const long long cap = (long long)f.sms * f.ctas_per_sm;
    const int grid = (int)(want < cap ? want : cap);
    if (info) *info = LaunchInfo{grid, threads, smem, f.ctas_per_sm};
    if (grid <= 0) return cudaSuccess;
    return launch_pdl(kern, grid, threads, smem, s, b, part, ws_floats);
}

template <int MAXB>
cudaError_t launch_adjoint_partials(const Batch<MAXB>& b, bool generic, float* part, long long ws_floats,
                                    cudaStream_t s, LaunchInfo* info) {
    return generic ? launch_part_t<MAXB, true>(b, part, ws_floats, s, info)
                   : launch_part_t<MAXB, false>(b, part, ws_floats, s, info);
}

// Warps per CTA of the tensor-copy kernel: as many as the rings fit in one
// SM's shared memory (<= kTmaMaxWarps, or kTmaMaxWarps2 for units of two
// tile-rows), at most `req` when that is set.
int tma_warps_per_cta(int stage_bytes, int stages, int req, int jrows) {
    const int wmax = jrows > 1 ? kTmaMaxWarps2 : kTmaMaxWarps;
    int w = (kTmaSmemBudget - 128) / tma_warp_smem(stage_bytes, stages);
    if (w > wmax) w = wmax;
    if (req > 0 && req < w) w = req;
    return w < 1 ? 1 : w;
}

template <int MAXB>
cudaError_t launch_adjoint_partials_tma(const Batch<MAXB>& b, const TmaMaps<MAXB>& maps, float* part,
                                        long long ws_floats, cudaStream_t s, LaunchInfo* info) {
    // every instance of a tensor-copy launch has the same tile-rows per unit
    const int jr = b.inst[0].jrows > 1 ? 2 : 1;
    auto kern = jr == 2 ? bsi_adjoint_partials_tma_kernel<MAXB, 2> : bsi_adjoint_partials_tma_kernel<MAXB, 1>;
    const int wpc = tma_warps_per_cta(b.buf_bytes, b.stages, b.warps_req, jr);
    const int threads = wpc * kLanes;
    const int smem = wpc * tma_warp_smem(b.buf_bytes, b.stages) + 128;
    KernelFacts f;
    cudaError_t e = kernel_facts(reinterpret_cast<const void*>(kern), threads, smem, &f);
    if (e != cudaSuccess) return e;
    const long long want = cdiv(b.total_units, wpc);
    const long long cap = (long long)f.sms * f.ctas_per_sm;
    const int grid = (int)(want < cap ? want : cap);
    if (info) *info = LaunchInfo{grid, threads, smem, f.ctas_per_sm};
    if (grid <= 0) return cudaSuccess;
    return launch_pdl(kern, grid, threads, smem, s, b, maps, part, ws_floats);
}

template <int MAXB>
cudaError_t launch_adjoint_reduce(const Batch<MAXB>& b, const float* part, long long ws_floats, cudaStream_t s,
                                  LaunchInfo* info) {
    auto kern = b.inst[0].jrows > 1 ? bsi_adjoint_reduce_kernel<MAXB, 2> : bsi_adjoint_reduce_kernel<MAXB, 1>;
    KernelFacts f;
    cudaError_t e = kernel_facts(reinterpret_cast<const void*>(kern), 256, 0, &f);
    if (e != cudaSuccess) return e;
    // one point per thread: more loads in flight than a grid-stride loop over one
    // resident wave (512^3 at spacing 3: 0.403 -> 0.388 ms for the adjoint); the
    // loop in the kernel covers what exceeds 64 waves
    const long long want = cdiv(b.total_points, 256);
    const long long cap = (long long)f.sms * f.ctas_per_sm * 64;
    const int grid = (int)(want < cap ? want : cap);
    if (info) *info = LaunchInfo{grid, 256, 0, f.ctas_per_sm};
    if (grid <= 0) return cudaSuccess;
    return launch_pdl(kern, grid, 256, 0, s, b, part, ws_floats);   // may start while the partials drain
}

template cudaError_t launch_adjoint_partials<1>(const Batch<1>&, bool, float*, long long, cudaStream_t, LaunchInfo*);
template cudaError_t launch_adjoint_partials<kMaxBatch>(const Batch<kMaxBatch>&, bool, float*, long long,
                                                         cudaStream_t, LaunchInfo*);
template cudaError_t launch_adjoint_partials_tma<1>(const Batch<1>&, const TmaMaps<1>&, float*, long long,
                                                    cudaStream_t, LaunchInfo*);
template cudaError_t launch_adjoint_partials_tma<kMaxBatch>(const Batch<kMaxBatch>&, const TmaMaps<kMaxBatch>&,
                                                            float*, long long, cudaStream_t, LaunchInfo*);
template cudaError_t launch_adjoint_reduce<1>(const Batch<1>&, const float*, long long, cudaStream_t, LaunchInfo*);
template cudaError_t launch_adjoint_reduce<kMaxBatch>(const Batch<kMaxBatch>&, const float*, long long,
                                                       cudaStream_t, LaunchInfo*);

// Failure-detection self-test: one warp arms an mbarrier for 16 bytes that no
// copy will deliver and waits with the kernels' own bounded wait; when it gives
// up it records kErrTimeout, exactly as a lost bulk copy would, and returns.
// Nothing is ever in flight on the barrier, so invalidating it is legal.
__global__ void __launch_bounds__(32) bsi_selftest_lost_copy_kernel() {
    __shared__ __align__(8) uint64_t bar;
    const int lane = threadIdx.x;
    if (lane == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_arrive_expect_tx(&bar, 16);   // the arrival is there; the 16 bytes never come
    }
    __syncwarp();
    if (!mbar_wait_bounded(&bar, 0) && lane == 0) atomicOr(&g_err, kErrTimeout);
    __syncwarp();
    if (lane == 0) mbar_inval(&bar);
}

cudaError_t launch_selftest_lost_copy(cudaStream_t s) {
    bsi_selftest_lost_copy_kernel<<<1, 32, 0, s>>>();
    return cudaGetLastError();
}

cudaError_t adjoint_err_read_clear(unsigned* out, cudaStream_t s) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_err, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_err);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(p, 0, sizeof(unsigned), s);
}

}  // namespace bsi
