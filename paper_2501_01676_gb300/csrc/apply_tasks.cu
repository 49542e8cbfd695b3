// The BDDC preconditioner M^-1 r = R~^T D~ S~^-1 D~^T R~ r (Sect. 3) as one
// persistent launch.
//
// The host lists the work items of the apply in three queues:
//   restriction: y = zc[nG:nG+nPi] += Psi_i^T D_i^T r_i     (gather -> GEMV -> scatter-add)
//   coarse, in topological order:
//      the coarse solve S_Pi x = y: the forward sweep of the nested-dissection
//      factors, front by front from the leaves (each front after its children),
//      then the backward sweep from the roots (each front after its parent);
//      or the product with the explicit inverse when the coarse problem is small;
//      then the prolongation zc[0:nG] += D_i Phi_i x_i     (transposed operators)
//   local: zc[0:nG] += P_i r_i, the bulk of the apply's bytes, which depends on
//      nothing else and streams while the coarse solve's dependency chain runs.
// Every CTA drains the restriction queue first; then a quarter of the CTAs take
// the coarse queue and the rest the local queue, and a CTA whose queue is empty
// moves to the other one.  Coarse items wait
// (bounded) on completion counters of the items they depend on and bump their
// own counters when their scatter-adds are done; items are dispensed in queue
// order and wait only on earlier items of the coarse queue, which running CTAs
// hold, so the launch needs no co-residency.  Inputs written during the launch
// are read through L2 (ld.global.cg); matrices through the read-only path, the
// rows of a waiting item prefetched into L2 before it waits.
#include <cuda_runtime.h>

#include "bddc_internal.h"

namespace {

constexpr int AP_THREADS = 256;
constexpr int AP_MAXCOLS = 2048;                 // column-slice width of the work items
constexpr long long AP_WAIT_LIMIT = 1LL << 24;   // x ~0.1 us sleeps: a few seconds

__device__ __forceinline__ int ld_acquire_i(const int* f) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    return v;
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class MT>
struct VecT;
template <>
struct VecT<double> {
    typedef double2 type;
    static constexpr int W = 2;
    __device__ static double dot(const double2& a, const double* x) { return a.x * x[0] + a.y * x[1]; }
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
};
template <>
struct VecT<float> {
    typedef float4 type;
    static constexpr int W = 4;
    __device__ static float dot(const float4& a, const float* x) {
        return a.x * x[0] + a.y * x[1] + a.z * x[2] + a.w * x[3];
    }
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};

// out[oidx[r]] += sum_c M[r][c] in[iidx[c]] over the item's rows; the input
// slice is staged in shared memory (in the matrix precision).  `coherent`:
// the input was written during this launch (read through L2).
template <class MT>
__device__ void row_gemv(const MT* __restrict__ pool, const GemvItem& it, const int* __restrict__ idx,
                         const double* in, double* out, MT* xs, bool coherent) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int* iidx = idx + it.iidx_off;
    const int* oidx = idx + it.oidx_off;
    const MT* M = pool + it.moff + it.col0;
    const int ncols = it.ncols;
    for (int q = t; q < ncols; q += AP_THREADS) {
        const int g = iidx[it.col0 + q];
        xs[q] = (MT)(coherent ? __ldcg(in + g) : __ldg(in + g));
    }
    __syncthreads();
    typedef typename VecT<MT>::type VT;
    constexpr int VW = VecT<MT>::W;
    constexpr int CH = 4;
    const int rend = it.row0 + it.nrows;
    const bool aligned = ((it.moff + it.col0) % VW) == 0 && (it.ld % VW) == 0;
    const int nvec = aligned ? ncols / VW : 0;
    for (int r = it.row0 + 2 * wid; r < rend; r += 2 * (AP_THREADS / 32)) {
        const bool two = r + 1 < rend;
        const MT* row0 = M + (long long)r * it.ld;
        const MT* row1 = M + (long long)(two ? r + 1 : r) * it.ld;
        MT acc0 = 0, acc1 = 0;
        if (aligned) {
            const VT* rv0 = reinterpret_cast<const VT*>(row0);
            const VT* rv1 = reinterpret_cast<const VT*>(row1);
            for (int base = 0; base < nvec; base += 32 * CH) {
                VT a0[CH], a1[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const int v = base + lane + 32 * u;
                    a0[u] = v < nvec ? __ldg(rv0 + v) : VecT<MT>::zero();
                    a1[u] = (v < nvec && two) ? __ldg(rv1 + v) : VecT<MT>::zero();
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const int v = base + lane + 32 * u;
                    if (v < nvec) {
                        acc0 += VecT<MT>::dot(a0[u], xs + v * VW);
                        acc1 += VecT<MT>::dot(a1[u], xs + v * VW);
                    }
                }
            }
        }
        for (int q = nvec * VW + lane; q < ncols; q += 32) {
            acc0 += __ldg(row0 + q) * xs[q];
            if (two) acc1 += __ldg(row1 + q) * xs[q];
        }
        acc0 = wsum(acc0);
        acc1 = wsum(acc1);
        if (lane == 0) {
            atomicAdd(&out[oidx[r]], (double)acc0);
            if (two) atomicAdd(&out[oidx[r + 1]], (double)acc1);
        }
    }
}

// Tall narrow operator stored transposed (ncols x rows, row stride ld): one
// thread per output row.
template <class MT>
__device__ void col_gemv(const MT* __restrict__ pool, const GemvItem& it, const int* __restrict__ idx,
                         const double* in, double* out, MT* xs) {
    const int t = threadIdx.x;
    const int* iidx = idx + it.iidx_off;
    const int* oidx = idx + it.oidx_off;
    const MT* Mt = pool + it.moff;
    for (int q = t; q < it.ncols; q += AP_THREADS) xs[q] = (MT)__ldcg(in + iidx[it.col0 + q]);
    __syncthreads();
    for (int r = it.row0 + t; r < it.row0 + it.nrows; r += AP_THREADS) {
        const MT* col = Mt + (long long)it.col0 * it.ld + r;
        MT acc = 0;
        int q = 0;
        // eight independent loads in flight per thread
        for (; q + 8 <= it.ncols; q += 8) {
            MT a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = __ldg(col + (long long)(q + u) * it.ld);
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += a[u] * xs[q + u];
        }
        for (; q < it.ncols; ++q) acc += __ldg(col + (long long)q * it.ld) * xs[q];
        atomicAdd(&out[oidx[r]], (double)acc);
    }
}

// Prefetch the matrix lines of an item into L2 (row-major rows, or the
// transposed layout of the prolongation).
template <class MT>
__device__ __forceinline__ void prefetch_item(const MT* pool, const GemvItem& it, bool transposed) {
    const int per_line = 128 / (int)sizeof(MT);
    const int outer = transposed ? it.ncols : it.nrows;
    const int inner = transposed ? it.nrows : it.ncols;
    const int lines = (inner + per_line - 1) / per_line + 1;
    for (int q = threadIdx.x; q < outer * lines; q += AP_THREADS) {
        const int o = q / lines, l = q - o * lines;
        const MT* base = transposed ? pool + it.moff + (long long)(it.col0 + o) * it.ld + it.row0
                                    : pool + it.moff + (long long)(it.row0 + o) * it.ld + it.col0;
        const MT* a = base + l * per_line;
        if (l * per_line < inner + per_line) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
}

// Bounded wait of one thread until ctr[w] >= target.  Gives up when another
// waiter has given up (abort flag) or after `limit` polls (~0.1 us each):
// then it flags ERR_TIMEOUT_APPLY, raises the abort flag and returns false.
__device__ bool ap_wait_ge(const int* ctr, int w, int target, int* abort_flag, int* err, long long limit) {
    long long it = 0;
    while (ld_acquire_i(ctr + w) < target) {
        if (*(volatile int*)abort_flag) return false;
        if (++it > limit) {
            atomicOr(err, ERR_TIMEOUT_APPLY);
            atomicExch(abort_flag, 1);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// The wait above on a counter that nothing increments (host self-test of the
// bounded waits): ends by itself after `limit` polls with the error flagged.
__global__ void k_wait_selftest(int* ctr, int* err, long long limit) {
    if (threadIdx.x == 0) ap_wait_ge(ctr, 0, 1, ctr + 1, err, limit);
}

template <class T>
__global__ void __launch_bounds__(AP_THREADS) k_apply_tasks(const ApTask* __restrict__ tasks, int nres, int ntasks,
                                                           int nlocal, int ncoarse_ctas, int* ctr,
                                                           const T* __restrict__ MA, const double* __restrict__ CO,
                                                           const T* __restrict__ MC, const int* __restrict__ idxA,
                                                           const int* __restrict__ idxB, const double* r,
                                                           double* zc, int nG, int nPi, int* err,
                                                           const int* skip) {
    if (skip && *skip) return;
    __shared__ __align__(16) double xs_raw[AP_MAXCOLS];
    __shared__ int s_task, s_abort, s_q;
    if (threadIdx.x == 0) {
        s_abort = 0;
        s_q = 0;
    }
    double* y2 = zc + nG;                 // [y | x]: coarse right-hand side, coarse solution
    // queue order of this CTA: restriction first, then coarse / local or local / coarse
    const bool coarse_first = blockIdx.x < ncoarse_ctas;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int k = -1;
            while (s_q < 3) {
                const int q = s_q == 0 ? 0 : ((s_q == 1) == coarse_first ? 1 : 2);
                const int v = atomicAdd(ctr + (q == 0 ? AP_CTR_NEXT_RES : q == 1 ? AP_CTR_NEXT : AP_CTR_NEXT_LOCAL), 1);
                const int nq = q == 0 ? nres : q == 1 ? ntasks : nlocal;
                if (v < nq) {
                    k = q == 0 ? v : q == 1 ? nres + v : nres + ntasks + v;
                    break;
                }
                ++s_q;
            }
            s_task = k;
        }
        __syncthreads();
        const int k = s_task;
        if (k < 0) return;
        const ApTask tk = tasks[k];
        if (tk.w0 >= 0 || tk.w1 >= 0) {
            if (tk.kind == AP_PROLONG) prefetch_item<T>(MC, tk.it, true);
            else if (tk.kind != AP_LOCAL) prefetch_item<double>(CO, tk.it, false);
        }
        if (threadIdx.x == 0) {
            for (int q = 0; q < 2; ++q) {
                const int w = q == 0 ? tk.w0 : tk.w1;
                const int target = q == 0 ? tk.t0 : tk.t1;
                if (w < 0 || s_abort) continue;
                if (!ap_wait_ge(ctr, w, target, ctr + AP_CTR_ABORT, err, AP_WAIT_LIMIT)) s_abort = 1;
            }
            __threadfence();
        }
        __syncthreads();
        switch (tk.kind) {
            case AP_LOCAL: row_gemv<T>(MA, tk.it, idxA, r, zc, reinterpret_cast<T*>(xs_raw), false); break;
            case AP_SWEEP: row_gemv<double>(CO, tk.it, idxB, y2, y2, xs_raw, true); break;
            case AP_DENSE: row_gemv<double>(CO, tk.it, idxA, y2, y2, xs_raw, true); break;
            default: col_gemv<T>(MC, tk.it, idxA, y2 + nPi, zc, reinterpret_cast<T*>(xs_raw)); break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (tk.s0 >= 0) atomicAdd(ctr + tk.s0, 1);
            if (tk.s1 >= 0) atomicAdd(ctr + tk.s1, 1);
        }
    }
}

}  // namespace

template <class T>
int apply_tasks_blocks() {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_apply_tasks<T>, AP_THREADS, 0) != cudaSuccess ||
        per < 1)
        per = 1;
    return sms * per;
}

template <class T>
int apply_tasks_run(const ApTask* tasks, int nres, int ntasks, int nlocal, int nblocks, int* ctr, int nctr,
                    const T* MA, const double* CO, const T* MC, const int* idxA, const int* idxB, const double* r,
                    double* zc, int nG, int nPi, int* err, const int* skip, double bytes, cudaStream_t st) {
    if (nres + ntasks + nlocal <= 0) return BDDC_OK;
    BDDC_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(int) * nctr, st));
    ktimer_begin(KT_APPLY_TASKS, st);
    const int grid = std::max(1, std::min(nres + ntasks + nlocal, nblocks));
    const int ncoarse = ntasks > 0 ? std::max(1, grid / 4) : 0;
    k_apply_tasks<T><<<grid, AP_THREADS, 0, st>>>(tasks, nres, ntasks, nlocal, ncoarse, ctr, MA, CO, MC, idxA, idxB,
                                                  r, zc, nG, nPi, err, skip);
    bddc_note_launches(1);
    ktimer_end(KT_APPLY_TASKS, st, 0.0, bytes);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

template int apply_tasks_blocks<float>();
template int apply_tasks_blocks<double>();
template int apply_tasks_run<float>(const ApTask*, int, int, int, int, int*, int, const float*, const double*,
                                    const float*, const int*, const int*, const double*, double*, int, int, int*,
                                    const int*, double, cudaStream_t);
template int apply_tasks_run<double>(const ApTask*, int, int, int, int, int*, int, const double*, const double*,
                                     const double*, const int*, const int*, const double*, double*, int, int, int*,
                                     const int*, double, cudaStream_t);

int wait_selftest_run(long long limit, int* timed_out) {
    int* d = nullptr;
    BDDC_CUDA_TRY(cudaMalloc(&d, 3 * sizeof(int)));
    cudaError_t e = cudaMemset(d, 0, 3 * sizeof(int));
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>(d, d + 2, limit);
        bddc_note_launches(1);
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d + 2, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        bddc_set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
        return BDDC_ECUDA;
    }
    *timed_out = (h & ERR_TIMEOUT_APPLY) ? 1 : 0;
    return BDDC_OK;
}
