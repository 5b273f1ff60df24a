// bsi_forward.cu -- forward BSI kernels (Eq. 1, Sec. 2.1) and their launcher.
#include "bsi_kernels.cuh"
#include "bsi_launch.h"

namespace bsi {

static __device__ unsigned g_err;

// Persistent grid: in round r every warp of the launch takes one unit of the
// concatenated unit lists of all instances (slot_unit, CTA-major: the warps of
// a CTA take neighbouring units).  The per-unit work is near-uniform,
// so the static assignment balances without an atomic ticket and is
// deterministic.
// Batched launches pack every spacing's arithmetic (see fwd_packed): their
// narrow volumes fill 63% of the lanes, so the per-row instructions bound them.
constexpr bool kBatchFwdPacked = true;

template <int MAXB, bool BF16, bool GENERIC, int C = 3>
__global__ void __launch_bounds__(kMaxWarpsPerCta * kLanes, 2)
    bsi_forward_kernel(const __grid_constant__ Batch<MAXB> b) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & (kLanes - 1);
    const int warp = threadIdx.x >> 5;
    unsigned char* stage = smem + (size_t)warp * fwd_warp_smem(b.buf_bytes);
    const int wpc = blockDim.x >> 5;
    constexpr bool PA = MAXB > 1 && kBatchFwdPacked;
    int ii = 0;
    int ring = 0;  // next staging buffer of the warp's store ring
    asm volatile("griddepcontrol.wait;" ::: "memory");   // the previous kernel's writes are visible
    for (long long r = 0;; ++r) {
        const long long uu = slot_unit(r, blockIdx.x, warp, gridDim.x, wpc, b.total_units, false);
        if (uu < 0) break;
        while (ii + 1 < b.n && uu >= b.inst[ii + 1].unit_begin) ++ii;
        const InstDesc& d = b.inst[ii];
        // FP32 output at x-spacings <= 3 (bound by per-row instructions) reads the
        // descriptor through a constant index in single-volume launches (512^3 at 3:
        // 0.400 -> 0.390 ms); at larger spacings, and for BF16 output, the same
        // measured 0.3-1.3% slower
        const InstDesc& dc = b.inst[BF16 ? ii : inst_index<MAXB>(ii)];
        const long long ul = uu - d.unit_begin;
        if (GENERIC) {
            forward_unit<0, BF16, C, PA>(d, ul, stage, b.buf_bytes, lane, ring, &g_err);
        } else {
            switch (d.dx) {
                case 1: forward_unit<1, BF16, C, PA>(dc, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 2: forward_unit<2, BF16, C, PA>(dc, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 3: forward_unit<3, BF16, C, PA>(dc, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 4: forward_unit<4, BF16, C, PA>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 5: forward_unit<5, BF16, C, PA>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 6: forward_unit<6, BF16, C, PA>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                case 7: forward_unit<7, BF16, C, PA>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
                default: forward_unit<8, BF16, C, PA>(d, ul, stage, b.buf_bytes, lane, ring, &g_err); break;
            }
        }
    }
    // the staging ring must outlive every bulk copy that reads it
    if (lane == 0) bulk_wait_all<0>();
    __syncwarp();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   // this CTA's rows are written
}

template <int MAXB, bool BF16, bool GENERIC, int C = 3>
static cudaError_t launch_fwd_t(const Batch<MAXB>& b, cudaStream_t s, LaunchInfo* info) {
    auto kern = bsi_forward_kernel<MAXB, BF16, GENERIC, C>;
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
    return launch_pdl(kern, grid, threads, smem, s, b);
}

template <int MAXB>
cudaError_t launch_forward(const Batch<MAXB>& b, bool bf16, bool generic, cudaStream_t s,
                           LaunchInfo* info) {
    if (bf16) return generic ? launch_fwd_t<MAXB, true, true>(b, s, info) : launch_fwd_t<MAXB, true, false>(b, s, info);
    return generic ? launch_fwd_t<MAXB, false, true>(b, s, info) : launch_fwd_t<MAXB, false, false>(b, s, info);
}

// Forward on the tensor-store path (one volume, C = 3 or 1 channels; see
// fwd_tma_rows): the same persistent unit walk as bsi_forward_kernel, rows
// leaving in blocks of rb.
template <bool BF16, int C>
__global__ void __launch_bounds__(kMaxWarpsPerCta * kLanes, 2)
    bsi_forward_tma_kernel(const __grid_constant__ Batch<1> b, const __grid_constant__ CUtensorMap map, int rb,
                           int blk_bytes) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned base (the launch adds 128 bytes for it)
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int lane = threadIdx.x & (kLanes - 1);
    const int warp = threadIdx.x >> 5;
    unsigned char* stage = smem + (size_t)warp * fwd_tma_warp_smem(blk_bytes);
    const int wpc = blockDim.x >> 5;
    int ring = 0;
    const InstDesc& d = b.inst[0];
    asm volatile("griddepcontrol.wait;" ::: "memory");   // the previous kernel's writes are visible
    for (long long r = 0;; ++r) {
        const long long ul = slot_unit(r, blockIdx.x, warp, gridDim.x, wpc, b.total_units, false);
        if (ul < 0) break;
        switch (d.dx) {
            case 1: forward_unit_tma<1, BF16, C>(d, &map, ul, stage, blk_bytes, rb, lane, ring, &g_err); break;
            case 2: forward_unit_tma<2, BF16, C>(d, &map, ul, stage, blk_bytes, rb, lane, ring, &g_err); break;
            case 3: forward_unit_tma<3, BF16, C>(d, &map, ul, stage, blk_bytes, rb, lane, ring, &g_err); break;
            case 4: forward_unit_tma<4, BF16, C>(d, &map, ul, stage, blk_bytes, rb, lane, ring, &g_err); break;
            case 5: forward_unit_tma<5, BF16, C>(d, &map, ul, stage, blk_bytes, rb, lane, ring, &g_err); break;
            case 6: forward_unit_tma<6, BF16, C>(d, &map, ul, stage, blk_bytes, rb, lane, ring, &g_err); break;
            case 7: forward_unit_tma<7, BF16, C>(d, &map, ul, stage, blk_bytes, rb, lane, ring, &g_err); break;
            default: forward_unit_tma<8, BF16, C>(d, &map, ul, stage, blk_bytes, rb, lane, ring, &g_err); break;
        }
    }
    // the blocks must outlive every tensor store that reads them
    if (lane == 0) bulk_wait_all<0>();
    __syncwarp();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <bool BF16, int C>
static cudaError_t launch_fwd_tma_t(const Batch<1>& b, const CUtensorMap& map, int rb, cudaStream_t s,
                                    LaunchInfo* info) {
    const InstDesc& d = b.inst[0];
    const int blk_bytes = pad128(rb * fwd_tma_row_bytes(d.gcells, d.dx, BF16, C));
    const int wsm = fwd_tma_warp_smem(blk_bytes);
    const int wpc = warps_per_cta(wsm, b.warps_req);
    const int threads = wpc * kLanes;
    const int smem = wpc * wsm + 128;
    const void* kern = reinterpret_cast<const void*>(bsi_forward_tma_kernel<BF16, C>);
    KernelFacts f;
    cudaError_t e = kernel_facts(kern, threads, smem, &f);
    if (e != cudaSuccess) return e;
    const long long want = cdiv(b.total_units, wpc);
    const long long cap = (long long)f.sms * f.ctas_per_sm;
    const int grid = (int)(want < cap ? want : cap);
    if (info) *info = LaunchInfo{grid, threads, smem, f.ctas_per_sm};
    if (grid <= 0) return cudaSuccess;
    return launch_pdl(bsi_forward_tma_kernel<BF16, C>, grid, threads, smem, s, b, map, rb, blk_bytes);
}

cudaError_t launch_forward_tma(const Batch<1>& b, bool bf16, int channels, const CUtensorMap& map, int rb,
                               cudaStream_t s, LaunchInfo* info) {
    if (channels == 1)
        return bf16 ? launch_fwd_tma_t<true, 1>(b, map, rb, s, info) : launch_fwd_tma_t<false, 1>(b, map, rb, s, info);
    return bf16 ? launch_fwd_tma_t<true, 3>(b, map, rb, s, info) : launch_fwd_tma_t<false, 3>(b, map, rb, s, info);
}

// Scalar (one-channel) interpolation of a single volume.
cudaError_t launch_forward_scalar(const Batch<1>& b, bool bf16, bool generic, cudaStream_t s, LaunchInfo* info) {
    if (bf16)
        return generic ? launch_fwd_t<1, true, true, 1>(b, s, info) : launch_fwd_t<1, true, false, 1>(b, s, info);
    return generic ? launch_fwd_t<1, false, true, 1>(b, s, info) : launch_fwd_t<1, false, false, 1>(b, s, info);
}

template cudaError_t launch_forward<1>(const Batch<1>&, bool, bool, cudaStream_t, LaunchInfo*);
template cudaError_t launch_forward<kMaxBatch>(const Batch<kMaxBatch>&, bool, bool, cudaStream_t, LaunchInfo*);

cudaError_t forward_err_read_clear(unsigned* out, cudaStream_t s) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_err, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_err);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(p, 0, sizeof(unsigned), s);
}

}  // namespace bsi
