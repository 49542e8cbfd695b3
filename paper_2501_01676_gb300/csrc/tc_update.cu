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
#include "tc_common.cuh"

namespace {

using namespace tcx;
constexpr int TM = 128, TN = 128;         // tile; the MMA is M = 128, N = 128
constexpr int TC_THREADS = 128;

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
        // bounded wait for this chunk's MMAs (mbarrier phase = chunk parity; an
        // expired wait is followed by a second bounded one)
        if (!mbar_wait(smem_u32(mbar), (uint32_t)(chunk & 1))) {
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
