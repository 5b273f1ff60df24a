// bsi_launch.h -- host-side launchers shared by the C ABI (bsi_abi.cu) and the
// kernel translation units (bsi_forward.cu, bsi_adjoint.cu).
#pragma once

#include <cuda.h>   // CUtensorMap (the type only: maps are encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

#include "bsi_geometry.h"

namespace bsi {

// Launches kern on s as a programmatic dependent of the previous kernel on s: it
// may be scheduled while that kernel's CTAs drain (they signal
// griddepcontrol.launch_dependents when done) and waits in griddepcontrol.wait
// for that grid's completion before touching memory.  After a kernel that never
// signals, this is an ordinary launch.
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kern)(P...), int grid, int threads, int smem, cudaStream_t s, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

// What a launcher chose; returned for diagnostics and the self-check.
struct LaunchInfo {
    int grid = 0;
    int block = 0;
    int smem = 0;
    int ctas_per_sm = 0;
};

template <int MAXB>
cudaError_t launch_forward(const Batch<MAXB>& b, bool bf16, bool generic, cudaStream_t s,
                           LaunchInfo* info);

// The paper's thread-per-tile kernels (TT, TTLI with lerp = true) for one volume.
cudaError_t launch_forward_tile_variant(const Batch<1>& b, bool lerp, cudaStream_t s, LaunchInfo* info);
cudaError_t variants_err_read_clear(unsigned* out, cudaStream_t s);

// Non-integer, non-aligned spacing (bsi_rational.cu).
int rational_warps_per_cta(int nx);
cudaError_t launch_forward_rational(const RatDesc& d, cudaStream_t s, LaunchInfo* info);
// Adjoint of the non-integer-spacing path: its unit counts and partial-sum
// floats (the workspace), and its two launches (partials, reduce).
struct RatAdjPlan {
    int ncx, ncy, ncz, nsx, sc, zc;   // cells per axis, strips, cells per strip, z-cells per unit
    long long part_floats;
};
RatAdjPlan rational_adjoint_plan(const RatDesc& d);
cudaError_t launch_adjoint_rational(const RatDesc& d, const float* grad, float* dphi, float* part, cudaStream_t s);
cudaError_t rational_err_read_clear(unsigned* out, cudaStream_t s);

// Forward of one volume on the tensor-store path (fwd_tma_rows gives rb > 0;
// map: the output as a 3-D tensor of 8-byte elements, box (strip, rb, 1));
// channels: 3 (displacement field) or 1 (scalar interpolation).
cudaError_t launch_forward_tma(const Batch<1>& b, bool bf16, int channels, const CUtensorMap& map, int rb,
                               cudaStream_t s, LaunchInfo* info);

// Scalar (one-channel) interpolation: Eq. 1 with grid [nz][ny][nx], output [Z][Y][X].
cudaError_t launch_forward_scalar(const Batch<1>& b, bool bf16, bool generic, cudaStream_t s, LaunchInfo* info);

template <int MAXB>
cudaError_t launch_adjoint_partials(const Batch<MAXB>& b, bool generic, float* part,
                                    long long ws_floats, cudaStream_t s, LaunchInfo* info);

// Tensor maps of the voxel gradients of a batch on the adjoint's tensor-copy
// path (one per instance, a kernel parameter).
template <int MAXB>
struct TmaMaps {
    CUtensorMap m[MAXB];
};

int tma_warps_per_cta(int stage_bytes, int stages, int req, int jrows = 1);

template <int MAXB>
cudaError_t launch_adjoint_partials_tma(const Batch<MAXB>& b, const TmaMaps<MAXB>& maps, float* part,
                                        long long ws_floats, cudaStream_t s, LaunchInfo* info);

template <int MAXB>
cudaError_t launch_adjoint_reduce(const Batch<MAXB>& b, const float* part, long long ws_floats,
                                  cudaStream_t s, LaunchInfo* info);

// BSI fused with the resampling of a floating image (one volume): value mode
// writes warped [Z][Y][X], gradient mode G [Z][Y][X][3] (d.field), reading
// dL/dwarped (d.gwarp).
cudaError_t launch_resample(const Batch<1>& b, bool grad, bool generic, cudaStream_t s, LaunchInfo* info);
cudaError_t resample_err_read_clear(unsigned* out, cudaStream_t s);

// Failure-detection self-test (a wait that runs out; see bsi_selftest_lost_copy).
cudaError_t launch_selftest_lost_copy(cudaStream_t s);

// Reads and clears the kernel error word of each translation unit (enqueued
// on s; the caller synchronises before looking at *out).
cudaError_t forward_err_read_clear(unsigned* out, cudaStream_t s);
cudaError_t adjoint_err_read_clear(unsigned* out, cudaStream_t s);

// Per-device, per-kernel launch facts, computed once (outside any capture the
// first call per device does this host-side work; no stream work is issued).
struct KernelFacts {
    int sms = 0;
    int ctas_per_sm = 0;
};

// Looks up (and on first use per device computes) the SM count and the
// resident CTAs per SM of `kernel` at `threads` x `smem`.  Raises the dynamic
// shared-memory limit of the kernel when smem exceeds 48 KB.
cudaError_t kernel_facts(const void* kernel, int threads, int smem, KernelFacts* out);

}  // namespace bsi
