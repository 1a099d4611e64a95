// Inline-PTX helpers for sm_103a: mbarriers with wall-clock-bounded waits,
// bulk (TMA) copies, tensor-memory allocation and loads, tcgen05.mma.
//
// Operand layout used with these helpers ("K-major, no swizzle"): a tile of
// R rows is stored as K-slabs; one slab holds 16 bytes' worth of K in each of
// two 8 x 16-byte core matrices (16 bf16 or 32 fp8 values per row). Inside a
// slab, row r, byte b (0..31) lives at
//     (r / 8) * 256 + (b / 16) * 128 + (r % 8) * 16 + (b % 16)
// so the descriptor's leading-dimension offset (next core matrix along K) is
// 128 bytes and its stride-dimension offset (next 8-row group) is 256 bytes.
// Slab s of a tile with R rows starts at s * R * 32 bytes.
#pragma once

#include <cstdint>

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Adds `bytes` to the transaction count the current phase waits for
// (no arrival).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Tests the phase with the given parity; the thread may be suspended for up
// to `hint_ns` nanoseconds while the phase is incomplete (it does not spin).
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity,
                                              uint32_t hint_ns = 20000u) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
// One elected lane of the (converged) warp arrives.
__device__ __forceinline__ void mbar_arrive_elect(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "elect.sync _|p, 0xffffffff;\n\t"
        "@p mbarrier.arrive.shared::cta.b64 _, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}
// Waits for the phase with the given parity to complete; gives up (returns
// false) once the global timer passes `deadline` (nanoseconds).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t deadline) {
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() > deadline) return false;
    return true;
}

// ---------------------------------------------------------------- bulk copy (TMA, non-tensor)
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Generic-proxy shared-memory writes become visible to the async proxy
// (tensor-core operand reads) after this fence.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------- tensor memory
// Whole warp: allocate ncols (power of two >= 32) columns; address -> *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns: thread t of the warp gets lane
// (taddr lane + t), columns col..col+15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// One 16-column load (32 lanes x 32 bits), its wait, and the values as 8
// packed pairs (column 2i in the low half).
__device__ __forceinline__ void tmem_ld16_wait_pk(uint32_t ta, uint64_t (&ra)[8]) {
    asm volatile(
        "{\n\t.reg .b32 a<16>;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {a0,a1,a2,a3,a4,a5,a6,a7,a8,a9,a10,a11,a12,a13,a14,a15}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n\t"
        "mov.b64 %0, {a0, a1};\n\t""mov.b64 %1, {a2, a3};\n\t""mov.b64 %2, {a4, a5};\n\t""mov.b64 %3, {a6, a7};\n\t""mov.b64 %4, {a8, a9};\n\t""mov.b64 %5, {a10, a11};\n\t""mov.b64 %6, {a12, a13};\n\t""mov.b64 %7, {a14, a15};\n\t""}"
        : "=l"(ra[0]), "=l"(ra[1]), "=l"(ra[2]), "=l"(ra[3]), "=l"(ra[4]), "=l"(ra[5]), "=l"(ra[6]), "=l"(ra[7])
        : "r"(ta)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- descriptors and MMA
// Shared-memory matrix descriptor, no swizzle, K-major, LBO 128 B, SBO 256 B.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    const uint32_t a = smem_u32(p);
    uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;  // leading-dimension byte offset
    d |= (uint64_t)(256u >> 4) << 32;  // stride-dimension byte offset
    d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
    return d;                          // base offset 0, relative LBO, no swizzle
}

// Instruction descriptor: D f32, A and B of the given format, both K-major.
// kind::f16 formats: 0 = f16, 1 = bf16. kind::f8f6f4 formats: 0 = e4m3.
__host__ __device__ constexpr uint32_t idesc(int M, int N, int a_fmt, int b_fmt) {
    return (1u << 4) | ((uint32_t)a_fmt << 7) | ((uint32_t)b_fmt << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T; one thread issues.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_fp8(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}
// Arrive on `bar` once all previously issued MMAs of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Byte offset of (row r, byte b) inside one K-slab (see the layout above).
__host__ __device__ __forceinline__ uint32_t slab_off(uint32_t r, uint32_t b) {
    return (r >> 3) * 256u + (b >> 4) * 128u + (r & 7u) * 16u + (b & 15u);
}

// Descriptors from the low word of a base descriptor: a slab at byte
// offset `off` from the base has the low word lo + off / 16 (the address
// field holds bits 4..17 of a shared-memory address below 2^18, so the sum
// never carries out of it); the high words are constants.
constexpr uint32_t DESC_HI = (256u >> 4) | (1u << 14);  // SBO 256 B, version 1
__device__ __forceinline__ uint32_t desc_lo(const void* p) {  // LBO 128 B
    return (smem_u32(p) >> 4) | ((128u >> 4) << 16);
}
__device__ __forceinline__ uint64_t desc_of(uint32_t lo, uint32_t hi) {
    return ((uint64_t)hi << 32) | lo;
}
// The other no-swizzle arrangement of a 128-row, 16-wide bf16 K-slab: the
// rows' first 16-byte K-chunks (elements 0..7) fill the first 2 KB and their
// second chunks (elements 8..15) the next 2 KB, each as 16 groups of 8 rows
// 128 B apart: LBO 2048 B (K-chunk to K-chunk), SBO 128 B (8-row group to
// 8-row group), so that each half is one contiguous block. Its descriptor:
// low word desc_lo(p) + DESC_HALVES_LBO, high word DESC_HALVES_HI.
constexpr uint32_t DESC_HALVES_LBO = ((2048u >> 4) - (128u >> 4)) << 16;
constexpr uint32_t DESC_HALVES_HI = (128u >> 4) | (1u << 14);
// Byte offset of (row r, K-chunk c) in that arrangement.
__host__ __device__ __forceinline__ uint32_t halves_off(uint32_t r, uint32_t c) {
    return c * 2048u + (r >> 3) * 128u + (r & 7u) * 16u;
}

}  // namespace tc
