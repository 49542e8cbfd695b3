// Trailing update of the Schur engine on the 5th-generation tensor cores.
//
// C[r0:r0+128, c0:c0+128] -= L21[r0:r0+128, 0:K] * U12[0:K, c0:c0+128]   (K = panel width)
//
// One CTA (4 warps) per 128 x 128 tile; K (the panel width, up to 128) is
// consumed 32 at a time: the threads stage the FP32 operands in
// shared memory split into TF32 high and low parts (x = hi + lo, both exactly
// representable in TF32), laid out as K-major "core matrices" (8 rows x 16
// bytes, no swizzle); one elected thread issues tcgen05.mma kind::tf32 with
// M = 128, N = 128, K = 8 for hi*hi + hi*lo + lo*hi (split TF32: the FP32
// product to about FP32 accuracy) accumulating in tensor memory; completion is
// signalled through an mbarrier (bounded wait); each warp then reads its 32
// accumulator lanes with tcgen05.ld and subtracts them from C.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "bddc_internal.h"

namespace {

constexpr int TM = 128, TN = 128;         // tile; the MMA is M = 128, N = 128
constexpr int KMAX = 32;                  // panel width handled per launch
constexpr int TC_THREADS = 128;
constexpr int CORE_BYTES = 128;           // 8 rows x 16 bytes
constexpr long long WAIT_LIMIT = 1LL << 24;

// byte offset of element (row, k) in a K-major core-matrix layout of a
// rows x KMAX FP32 operand: core matrix (row/8, k/4) at ((row/8)*(KMAX/4) + k/4)*128
__device__ __forceinline__ int cm_off(int row, int k) {
    return ((row >> 3) * (KMAX / 4) + (k >> 2)) * CORE_BYTES + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

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

// Stage a 128 x K FP32 block (row r, column k at src[r*ld + k], rows >= nrows and
// k >= K are zero) as TF32 hi / lo core-matrix operands.
__device__ __forceinline__ void stage(const float* __restrict__ src, long long ld, int nrows, int K,
                                      unsigned char* hi, unsigned char* lo, bool transposed) {
    // transposed: element (row, k) lives at src[k*ld + row] (U12 is K x N, N contiguous)
    for (int q = threadIdx.x; q < TM * KMAX; q += TC_THREADS) {
        int row, k;
        if (transposed) {
            k = q / TM;
            row = q - k * TM;
        } else {
            row = q / KMAX;
            k = q - row * KMAX;
        }
        float v = 0.f;
        if (row < nrows && k < K) v = transposed ? src[(long long)k * ld + row] : src[(long long)row * ld + k];
        float h = tf32_round(v);
        float l = tf32_round(v - h);
        *reinterpret_cast<float*>(hi + cm_off(row, k)) = h;
        *reinterpret_cast<float*>(lo + cm_off(row, k)) = l;
    }
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

// One 128 x 128 tile: C[0:nr, 0:nc] (row stride ldc) -= A[0:nr, 0:K] * B[0:K, 0:nc]
// A row-major (lda), B row-major K x N (ldb).  K is consumed in chunks of KMAX:
// stage the chunk, issue its MMAs, wait for them (the next chunk overwrites the
// operand buffers).  Returns through *err on a wait timeout.
__device__ void tc_tile(const float* __restrict__ A, long long lda, const float* __restrict__ B, long long ldb,
                        float* __restrict__ C, long long ldc, int nr, int nc, int K, unsigned char* smem,
                        uint64_t* mbar, uint32_t* tmem_slot, int* err) {
    unsigned char* a_hi = smem;
    unsigned char* a_lo = a_hi + TM * KMAX * 4;
    unsigned char* b_hi = a_lo + TM * KMAX * 4;
    unsigned char* b_lo = b_hi + TN * KMAX * 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    int chunk = 0;
    for (int k0 = 0; k0 < K && ok; k0 += KMAX, ++chunk) {
        const int kw = min(KMAX, K - k0);
        stage(A + k0, lda, nr, kw, a_hi, a_lo, false);
        stage(B + (long long)k0 * ldb, ldb, nc, kw, b_hi, b_lo, true);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (threadIdx.x == 0) {
            const uint32_t idesc = instr_desc(TM, TN);
            const uint32_t lbo = CORE_BYTES;                     // next core matrix along K
            const uint32_t sbo = (KMAX / 4) * CORE_BYTES;        // next 8-row group along M / N
            for (int kk = 0; kk < (kw + 7) / 8; ++kk) {
                const uint32_t koff = kk * 2 * CORE_BYTES;       // 8 TF32 = two core matrices along K
                const uint64_t ah = smem_desc(smem_u32(a_hi) + koff, lbo, sbo);
                const uint64_t al = smem_desc(smem_u32(a_lo) + koff, lbo, sbo);
                const uint64_t bh = smem_desc(smem_u32(b_hi) + koff, lbo, sbo);
                const uint64_t bl = smem_desc(smem_u32(b_lo) + koff, lbo, sbo);
                mma_tf32(tmem, ah, bh, idesc, (chunk > 0 || kk > 0) ? 1 : 0);
                mma_tf32(tmem, ah, bl, idesc, 1);
                mma_tf32(tmem, al, bh, idesc, 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(mbar)));
        }
        // bounded wait for this chunk's MMAs (mbarrier phase = chunk parity)
        uint32_t done = 0;
        long long itn = 0;
        const uint32_t parity = (uint32_t)(chunk & 1);
        while (!done && itn < WAIT_LIMIT) {
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}\n"
                : "=r"(done)
                : "r"(smem_u32(mbar)), "r"(parity));
            ++itn;
        }
        if (!done) {
            atomicOr(err, ERR_TIMEOUT_TC);
            ok = false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // every thread has seen the phase complete before the buffers are restaged
        __syncthreads();
        ok = __syncthreads_and(ok ? 1 : 0) != 0;
    }
    if (ok && K > 0) {
        // warp w owns accumulator lanes (rows) 32w .. 32w+31; each 32 x 32 block goes
        // through shared memory (the operand buffers are free now) so that the lanes
        // update 32 consecutive columns of one row at a time (coalesced)
        float* Tt = reinterpret_cast<float*>(smem) + warp * 32 * 33;
        for (int c0 = 0; c0 < TN; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) Tt[lane * 33 + j] = v[j];
            __syncwarp();
            const int col = c0 + lane;
            for (int r = 0; r < 32; ++r) {
                const int row = warp * 32 + r;
                if (row < nr && col < nc) C[(long long)row * ldc + col] -= Tt[r * 33 + lane];
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TN));
}

__global__ void __launch_bounds__(TC_THREADS) k_tc_selftest(const float* A, const float* B, float* C, int nr, int nc,
                                                            int K, int* err) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    tc_tile(A, KMAX, B, TN, C, TN, nr, nc, K, tsm, &mbar, &tslot, err);
}

__global__ void __launch_bounds__(TC_THREADS) k_tc_update(const EngItem<float>* __restrict__ items, int p, int nb,
                                                          int nt, int* err) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const EngItem<float> it = items[blockIdx.x];
    if (p >= it.k) return;
    const int w = min(nb, it.k - p);
    const int n = it.n;
    const long long ld = it.ld;
    const int m0 = p + w;
    const int y = blockIdx.y;
    const int ti = y / nt, tj = y - ti * nt;
    const int r0 = m0 + ti * TM, c0 = m0 + tj * TN;
    if (r0 >= n || c0 >= n) return;
    float* A = it.a;
    tc_tile(A + (long long)r0 * ld + p, ld, A + (long long)p * ld + c0, ld, A + (long long)r0 * ld + c0, ld,
            min(TM, n - r0), min(TN, n - c0), w, tsm, &mbar, &tslot, err);
}

constexpr size_t TC_SMEM = (size_t)4 * TM * KMAX * 4;    // a_hi, a_lo, b_hi, b_lo

}  // namespace

// Self-test entry used by the tests: C (128 x 128, row stride 128) -= A (128 x 32) * B (32 x 128).
int tc_selftest_run(const float* A, const float* B, float* C, int nr, int nc, int K, int* err, cudaStream_t st) {
    if (K > KMAX || nr > TM || nc > TN) return BDDC_EINVAL;
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    k_tc_selftest<<<1, TC_THREADS, TC_SMEM, st>>>(A, B, C, nr, nc, K, err);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

int tc_update_run(const EngItem<float>* items_dev, int count, int maxn, int p, int nb, int* err, cudaStream_t st) {
    const int mrem = std::max(maxn - p, 1);
    const int nt = (mrem + TM - 1) / TM;
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_tc_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    k_tc_update<<<dim3(count, nt * nt), TC_THREADS, TC_SMEM, st>>>(items_dev, p, nb, nt, err);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
