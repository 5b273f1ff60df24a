// bsi_async.cuh -- inline-PTX wrappers for the Blackwell bulk-copy (TMA) engine
// and shared-memory mbarriers, as used by the BSI kernels.
//
//  * bulk stores  shared -> global: cp.async.bulk ... .bulk_group, completion
//    tracked per issuing thread with commit_group / wait_group[.read]
//    (hardware waits: they always finish, no spin loop);
//  * bulk loads   global -> shared: cp.async.bulk ... .mbarrier::complete_tx,
//    completion observed on an mbarrier phase with try_wait.parity in a loop
//    bounded by kSpinLimit, so a lost completion ends in an error flag, never
//    in a hang.
// Every bulk copy moves a multiple of 16 bytes between 16-byte-aligned
// addresses; callers guarantee it.
#pragma once

#include <stdint.h>

namespace bsi {

constexpr uint32_t kSuspendHintNs = 100000;   // longest sleep of one try_wait round
constexpr int kSpinLimit = 20000;              // try_wait rounds before a wait is declared lost

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory loads and stores by 32-bit shared-window address.  The staging
// buffers are addressed through these rather than through generic pointers, so
// every access is a single LDS/STS with an immediate offset and no 64-bit
// address arithmetic.  They are unpredicated: the kernels lay out their
// staging rows so that every lane's accesses stay inside its warp's buffer
// (reads of voxels outside the volume hit zeroed bytes, writes past the row
// end are never copied out).
__device__ __forceinline__ float lds_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void sts_f32(uint32_t addr, float v) {
    asm volatile("st.shared.f32 [%0], %1;" :: "r"(addr), "f"(v) : "memory");
}

// Vector forms: addr must be 8-byte (v2) or 16-byte (v4) aligned.
__device__ __forceinline__ void lds_v2_f32(uint32_t addr, float& a, float& b) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "r"(addr));
}

__device__ __forceinline__ void lds_v4_f32(uint32_t addr, float& a, float& b, float& c, float& d) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(a), "=f"(b), "=f"(c), "=f"(d) : "r"(addr));
}

__device__ __forceinline__ void sts_v2_f32(uint32_t addr, float a, float b) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" :: "r"(addr), "f"(a), "f"(b) : "memory");
}

__device__ __forceinline__ void sts_v4_f32(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" :: "r"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

__device__ __forceinline__ void sts_b16(uint32_t addr, unsigned short v) {
    asm volatile("st.shared.b16 [%0], %1;" :: "r"(addr), "h"(v) : "memory");
}

// 32-bit words (two packed BF16 values); addr 4-, 8- or 16-byte aligned.
__device__ __forceinline__ void sts_b32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" :: "r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void sts_v2_b32(uint32_t addr, uint32_t a, uint32_t b) {
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" :: "r"(addr), "r"(a), "r"(b) : "memory");
}

__device__ __forceinline__ void sts_v4_b32(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" :: "r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------- bulk stores

// The streamed output is written once and not read back by the same kernel:
// its lines are marked first for eviction from L2, so that they leave for HBM
// while the kernel runs instead of lingering dirty into the next kernel (the
// adjoint right after the forward ran 7% faster in a step).
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;"
                 :: "l"(gdst), "r"(smem_u32(ssrc)), "r"(bytes), "l"(pol) : "memory");
}

// Tiled tensor store (TMA) of one box of a 3-D tensor map from shared memory
// at ssrc (128-byte aligned) into global memory, in the current bulk group;
// parts of the box outside the tensor are not written.  tmap is the generic
// address of a CUtensorMap held in kernel parameter space; the innermost
// coordinate c0 times the element size must be a multiple of 16 bytes and no
// coordinate may be negative.  Lines marked first for eviction, as bulk_store.
__device__ __forceinline__ void tensor_store_3d(const void* tmap, int c0, int c1, int c2, const void* ssrc) {
    asm volatile(
        "{\n\t.reg .b64 pol;\n\t"
        "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
        "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group.L2::cache_hint"
        " [%0, {%1, %2, %3}], [%4], pol;\n}"
        :: "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(ssrc)) : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Waits until at most N of this thread's committed bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" :: "n"(N) : "memory");
}

// Waits until at most N of this thread's committed bulk groups are incomplete.
template <int N>
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group %0;" :: "n"(N) : "memory");
}

// ---------------------------------------------------------------- bulk loads

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(smem_u32(bar)) : "memory");
}

// One arrival that also announces `bytes` of transaction count for this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(sdst)), "l"(gsrc), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Tiled tensor copy (TMA) of one box of a 3-D tensor map into shared memory
// at sdst (128-byte aligned), completing on bar with the box's full byte count
// (parts of the box outside the tensor arrive as zeros).  tmap is the generic
// address of a CUtensorMap held in kernel parameter space; the innermost
// coordinate c0 times the element size must be a multiple of 16 bytes.  The
// gradient is read once: its lines are marked first for eviction from L2, which
// keeps the adjoint's partial sums there for the reduce that follows.
__device__ __forceinline__ void tensor_load_3d(void* sdst, const void* tmap, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .b64 pol;\n\t"
        "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], pol;\n}"
        :: "r"(smem_u32(sdst)), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)) : "memory");
}

// One bounded wait round: the thread may sleep up to kSuspendHintNs for the
// phase of `parity` to complete (it wakes when it does); true if it completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendHintNs) : "memory");
    return ok != 0;
}

// Waits for the phase of `parity` to complete, at most kSpinLimit rounds of
// at most kSuspendHintNs each (about 2 s in all).  Returns false
// (warp-uniformly) if any lane gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    bool ok = false;
    for (int i = 0; i < kSpinLimit && !ok; ++i) ok = mbar_try_wait(bar, parity);
    return __all_sync(0xffffffffu, ok);
}

}  // namespace bsi
