// Device helpers shared by the tensor-core (tcgen05, split TF32) trailing
// updates: operand layout, shared-memory and instruction descriptors, the MMA,
// its commit to an mbarrier with a bounded wait, and accumulator loads from
// tensor memory.
//
// Operands are FP32 values split as x = hi + lo (both exactly representable in
// TF32); hi*hi + hi*lo + lo*hi reproduces the FP32 product to about FP32
// accuracy.  They are stored K-major in "core matrices" of 8 rows x 16 bytes (4
// TF32 values along K), no swizzle.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tcx {

constexpr int KMAX = 32;                  // K elements per staged chunk
constexpr int CORE_BYTES = 128;           // 8 rows x 16 bytes
constexpr long long WAIT_LIMIT = 1LL << 24;

// byte offset of element (row, k) in the K-major core-matrix layout of a
// rows x KMAX operand: core matrix (row/8, k/4) at ((row/8)*(KMAX/4) + k/4)*128
__device__ __forceinline__ int cm_off(int row, int k) {
    return ((row >> 3) * (KMAX / 4) + (k >> 2)) * CORE_BYTES + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading-dimension byte offset (between
// core matrices adjacent in K), stride byte offset (between core matrices
// adjacent in M/N), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;   // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4)                 // D format F32
           | (2u << 7)               // A format TF32
           | (2u << 10)              // B format TF32
           | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Split-TF32 MMAs of one staged chunk (kw <= KMAX valid K entries) into the
// 128 x 128 accumulator at tmem; the first MMA overwrites it when first != 0.
__device__ __forceinline__ void mma_chunk(uint32_t tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                          int kw, bool first) {
    const uint32_t idesc = instr_desc(128, 128);
    const uint32_t lbo = CORE_BYTES;                     // next core matrix along K
    const uint32_t sbo = (KMAX / 4) * CORE_BYTES;        // next 8-row group along M / N
    for (int kk = 0; kk < (kw + 7) / 8; ++kk) {
        const uint32_t koff = kk * 2 * CORE_BYTES;       // 8 TF32 = two core matrices along K
        const uint64_t ah = smem_desc(a_hi + koff, lbo, sbo);
        const uint64_t al = smem_desc(a_lo + koff, lbo, sbo);
        const uint64_t bh = smem_desc(b_hi + koff, lbo, sbo);
        const uint64_t bl = smem_desc(b_lo + koff, lbo, sbo);
        mma_tf32(tmem, ah, bh, idesc, (first && kk == 0) ? 0 : 1);
        mma_tf32(tmem, ah, bl, idesc, 1);
        mma_tf32(tmem, al, bh, idesc, 1);
    }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar));
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    long long itn = 0;
    while (!done && itn < WAIT_LIMIT) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity));
        ++itn;
    }
    return done != 0;
}

// Bounded wait for the mbarrier phase with the given parity; false on expiry.  An
// expired wait is followed by a second bounded one, so that the MMAs in flight
// (which read the operand buffers and write the accumulator) have finished before
// the caller reuses either or releases the tensor memory.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    if (mbar_try(mbar, parity)) return true;
    mbar_try(mbar, parity);
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tcx

// ---------------------------------------------------------------------------
// BF16 operands (kind::f16 with A = B = BF16, FP32 accumulation): one MMA per
// product, 8 BF16 values along K per core-matrix row, K = 16 per MMA.
namespace tcx {

// byte offset of element (row, k) in the K-major core-matrix layout of a
// rows x KMAX BF16 operand: core matrix (row/8, k/8) at ((row/8)*(KMAX/8) + k/8)*128
__device__ __forceinline__ int cm_off16(int row, int k) {
    return ((row >> 3) * (KMAX / 8) + (k >> 3)) * CORE_BYTES + (row & 7) * 16 + (k & 7) * 2;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
    return (1u << 4)                 // D format F32
           | (1u << 7)               // A format BF16
           | (1u << 10)              // B format BF16
           | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// MMAs of one staged BF16 chunk (kw <= KMAX valid K entries).
__device__ __forceinline__ void mma_chunk_bf16(uint32_t tmem, uint32_t a, uint32_t b, int kw, bool first) {
    const uint32_t idesc = instr_desc_bf16(128, 128);
    const uint32_t lbo = CORE_BYTES;                     // next core matrix along K
    const uint32_t sbo = (KMAX / 8) * CORE_BYTES;        // next 8-row group along M / N
    for (int kk = 0; kk < (kw + 15) / 16; ++kk) {
        const uint32_t koff = kk * 2 * CORE_BYTES;       // 16 BF16 = two core matrices along K
        mma_bf16(tmem, smem_desc(a + koff, lbo, sbo), smem_desc(b + koff, lbo, sbo), idesc,
                 (first && kk == 0) ? 0 : 1);
    }
}

}  // namespace tcx
