// Fifth-generation tensor core (tcgen05) primitives used by the learned
// gate's convolutions: shared-memory matrix descriptors, the instruction
// descriptor of a BF16 x BF16 -> FP32 MMA, MMA issue and commit, bulk and
// tiled-tensor (TMA) global -> shared copies, mbarrier init, transaction
// counts and bounded wait, and tensor-memory (TMEM) allocation and loads.
// sm_100-family PTX (compiled for sm_103a).
#pragma once

#include <stdint.h>

namespace sn {
namespace umma {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor for a K-major operand without swizzle.
// The operand is made of core matrices of 8 rows x 16 bytes (8 BF16), rows
// 16 bytes apart; `lbo` is the byte distance between core matrices adjacent
// in K, `sbo` between core matrices adjacent in M (or N).  Fields: start
// address >> 4 (bits 0-13), lbo >> 4 (16-29), sbo >> 4 (32-45), descriptor
// version 1 (bits 46-47), base offset 0, swizzle mode 0 (none).
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::f16 with FP32 accumulation (bits 4-5 = 1),
// BF16 A and B (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22 and M >> 4 in bits 24-28.
template <int M, int N>
constexpr uint32_t idesc_bf16() {
    static_assert(M == 128 && N % 16 == 0 && N >= 16 && N <= 256, "cta_group::1 shape with M = 128");
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A B^T for one K = 16 step; issued by a single thread.
template <uint32_t IDESC>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"((uint32_t)accumulate));
}

// Arrives once on the mbarrier when all MMAs issued so far by this thread
// have completed.
__device__ __forceinline__ void commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival on the mbarrier that also expects `bytes` of asynchronous
// copies to land before its phase completes.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// Bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16),
// completing on the mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(mbar))
                 : "memory");
}

// 2-D tiled tensor copy global -> shared (TMA) of the box at (x, y) of the
// tensor map (elements outside the tensor read as zero), completing on the
// mbarrier's transaction count.  x times the element size must be a
// multiple of 16 bytes; dst 128-byte aligned.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_addr(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_addr(mbar))
        : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with the given parity to complete.  Between polls the
// thread may sleep in hardware until the phase completes or about 20 us
// pass, so a long wait costs almost no issue slots.  Gives up (returns
// false) once `timeout_ns` nanoseconds of the global timer have passed since
// the call, or after 2^24 polls should that timer not advance.
__device__ __forceinline__ bool mbar_wait_ns(uint64_t* mbar, uint32_t parity, uint64_t timeout_ns) {
    const uint32_t a = smem_addr(mbar);
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 24); it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity), "r"(20000u)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > timeout_ns) return false;
    }
    return false;
}

// Bounds of the waits above.  A tile's copy or a tile's MMAs complete in
// microseconds; a wait that runs out of kWaitNs reports a device error, and
// the wait that then drains what is still in flight gets kDrainNs more
// before the CTA frees its TMEM and shared memory.
constexpr uint64_t kWaitNs = 500000000ull;    // 0.5 s
constexpr uint64_t kDrainNs = 2000000000ull;  // 2 s

// Warp-wide: allocates `ncols` TMEM columns (a power of two >= 32) and writes
// their address to *slot; then gives up the CTA's right to allocate more.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Warp-wide: frees columns allocated by tmem_alloc.
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Warp-wide: lane i reads 16 consecutive 32-bit columns of TMEM lane
// (lane base of taddr) + i.  The values are valid after wait_ld().
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Ordering of tcgen05 operations across a thread barrier.
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Makes this thread's generic-proxy shared-memory writes visible to the
// tensor core's (async-proxy) operand reads.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace umma
}  // namespace sn
