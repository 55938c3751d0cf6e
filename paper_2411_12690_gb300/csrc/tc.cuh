// Fifth-generation tensor-core (tcgen05) building blocks for sm_103a, as
// inline PTX: tensor-memory allocation, shared-memory matrix descriptors,
// instruction descriptors, MMA issue/commit, mbarrier waits with an iteration
// limit, and tensor-memory loads.
//
// Operand layouts, both K-major. (1) No swizzle, for the apply and the
// recovery of small bases: the smallest unit is a "core matrix" of 8 rows x 16
// bytes stored as 128 contiguous bytes (row r at byte 16 r). Core matrices
// adjacent along K are LBO = 128 bytes apart; groups of 8 rows are SBO =
// (K bytes / 16) * 128 bytes apart. One MMA consumes 32 bytes of K (two core
// matrices), so consecutive K steps advance the descriptor start address by
// 256 bytes. (2) 128-byte swizzle, for the streamed recovery of large bases
// (described at sw128_offset below).
#pragma once

#include <cstdint>

namespace ms {
namespace tc {

constexpr uint32_t kLBO = 128;

__host__ __device__ constexpr uint32_t sbo_bytes(int k_elems, int esz) { return (uint32_t)(k_elems * esz / 16) * 128u; }

// Byte offset of element (row, k) in a K-major no-swizzle operand image.
__host__ __device__ inline uint32_t operand_offset(int row, int k, int k_elems, int esz) {
    const int ke = 16 / esz;
    return (uint32_t)(row >> 3) * sbo_bytes(k_elems, esz) + (uint32_t)(k / ke) * kLBO + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k % ke) * (uint32_t)esz;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4 in bits 0-13, LBO >> 4 in
// 16-29, SBO >> 4 in 32-45, descriptor version 1 in 46-47, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// 128-byte swizzled K-major layout (the other operand layout used here): rows
// of 128 bytes of K, eight rows form a 1024-byte atom (atoms 1024-byte aligned
// and SBO = 1024 bytes apart along M/N), and the 16-byte chunk c of row r is
// stored at chunk position c ^ (r % 8), so the eight rows of a core matrix
// fall in different bank groups. One MMA consumes 32 bytes of a row; the K
// steps within a row advance the descriptor start address by 32 bytes (the
// hardware applies the XOR to the address bits).
constexpr uint32_t kSw128Atom = 1024;

__host__ __device__ inline uint32_t sw128_offset(int row, int kbyte) {
    return (uint32_t)(row >> 3) * kSw128Atom + (uint32_t)(row & 7) * 128u +
           ((uint32_t)(((kbyte >> 4) ^ (row & 7)) & 7) << 4) + (uint32_t)(kbyte & 15);
}

// Descriptor of a 128-byte swizzled K-major operand: SBO = 1024 bytes, layout
// type 2 (128-byte swizzle) in bits 61-63, version 1, base offset 0.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)((kSw128Atom >> 4) & 0x3FFF) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B formats
// (bits 7-9, 10-12: 1 = bf16 for kind::f16, 2 = tf32 for kind::tf32), both
// K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(bool tf32, int M, int N) {
    return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

// Allocation with a compile-time column count (an immediate in the
// instruction, so the kernel's tensor-memory need is known when it is built).
template <uint32_t NCOLS>
__device__ __forceinline__ void tmem_alloc_c(uint32_t* dst_smem) {
    static_assert(NCOLS >= 32 && NCOLS <= 512 && (NCOLS & (NCOLS - 1)) == 0, "power of two in [32, 512]");
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
                 "n"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

template <uint32_t NCOLS>
__device__ __forceinline__ void tmem_free_c(uint32_t taddr) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(NCOLS));
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make generic-proxy shared-memory writes visible to the tensor cores
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate) {
    if (TF32)
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
    else
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

// Arrive on the mbarrier once every MMA issued so far by this thread is done.
__device__ __forceinline__ void commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for the given phase parity of an mbarrier, giving up after max_tries
// polls (each try_wait may itself suspend briefly) or about two seconds,
// whichever comes first. Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int max_tries) {
    uint32_t done = 0;
    unsigned long long t0 = 0;
    for (int it = 0; it < max_tries && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(mbar)), "r"(parity)
            : "memory");
        if ((it & 1023) == 1023 && !done) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
            if (t0 == 0) t0 = t;
            else if (t - t0 > 2000000000ull) break;
        }
    }
    return done != 0;
}

// Plain arrive (one of the barrier's expected arrivals).
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
}

// Arrive on the mbarrier and raise its expected transaction count by bytes.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// One bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16); its bytes complete the transaction count of mbar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(mbar))
                 : "memory");
}

// Each thread of a warp reads 16 consecutive 32-bit columns of its own TMEM
// lane (lane = 32 * (warp % 4) + lane id), starting at column taddr & 0xffff.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// The same read without the wait: a group of loads is issued back to back and
// completed by one tmem_wait16 per group (the first waits for all of them; the
// register operands tie the values' later uses to the wait).
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

__device__ __forceinline__ float to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

}  // namespace tc
}  // namespace ms
