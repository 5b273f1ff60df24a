// bsi_probe.cu -- bsi_probe_fill: the write-only HBM peak, measured with the
// same store path as the forward kernel (TMA bulk copies from shared memory).
// It is the denominator of the forward's store roofline; the paper has no
// counterpart.
#include <cuda_runtime.h>

#include "bsi.h"
#include "bsi_async.cuh"
#include "bsi_launch.h"

namespace bsi {

constexpr int kFillChunk = 16 * 1024;    // bytes per bulk store
constexpr int kFillThreads = 256;

// Each warp's lane 0 streams whole chunks of dst from one shared buffer holding
// the pattern (written once, never changed, so a store need not wait for the
// previous one to finish reading it); at most 8 bulk groups per thread in
// flight.  CTA 0 also writes the tail (< kFillChunk bytes, a multiple of 16).
__global__ void __launch_bounds__(kFillThreads) bsi_probe_fill_kernel(unsigned char* dst, long long nchunks,
                                                                       int tail, uint32_t value) {
    extern __shared__ __align__(128) unsigned char fbuf[];
    for (int i = threadIdx.x; i < kFillChunk / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(fbuf)[i] = value;
    fence_proxy_async_smem();
    __syncthreads();
    if ((threadIdx.x & 31) != 0) return;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long step = (long long)gridDim.x * nw;
    for (long long c = (long long)blockIdx.x * nw + warp; c < nchunks; c += step) {
        bulk_store(dst + c * kFillChunk, fbuf, kFillChunk);
        bulk_commit();
        bulk_wait_read<8>();
    }
    if (blockIdx.x == 0 && warp == 0 && tail > 0) {
        bulk_store(dst + nchunks * kFillChunk, fbuf, (uint32_t)tail);
        bulk_commit();
    }
    bulk_wait_all<0>();
}

}  // namespace bsi

using namespace bsi;

extern "C" bsi_status bsi_probe_fill(void* dst, size_t bytes, uint32_t value, bsi_stream_t stream) {
    if (bytes == 0) return BSI_OK;
    if (!dst) return BSI_ERR_NULL;
    if (((uintptr_t)dst & 15) != 0 || (bytes & 15) != 0) return BSI_ERR_ALIGN;
    const void* kern = reinterpret_cast<const void*>(bsi_probe_fill_kernel);
    KernelFacts f;
    cudaError_t e = kernel_facts(kern, kFillThreads, kFillChunk, &f);
    if (e == cudaSuccess) {
        const long long nchunks = (long long)(bytes / kFillChunk);
        const int tail = (int)(bytes % kFillChunk);
        const long long want = nchunks / (kFillThreads / 32) + 1;
        const long long cap = (long long)f.sms * f.ctas_per_sm;
        const int grid = (int)(want < cap ? want : cap);
        bsi_probe_fill_kernel<<<grid, kFillThreads, kFillChunk, reinterpret_cast<cudaStream_t>(stream)>>>(
            static_cast<unsigned char*>(dst), nchunks, tail, value);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return BSI_ERR_CUDA;
    }
    return BSI_OK;
}
