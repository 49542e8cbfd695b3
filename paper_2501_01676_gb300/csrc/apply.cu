// Per-iteration operators of the Schur system (Sect. 3) on the GPU.
//
// One kernel serves every dense per-subdomain product of the hot loop:
//   out[oidx[r]] += sum_c M[r][c] * in[iidx[c]]     (gather -> GEMV -> scatter-add)
// * S x          : M = S^(i),                 iidx = oidx = R_i (interface map)
// * M^-1 r, part 1: M = [P_i ; (D_i Psi_i)^T], iidx = R_i, oidx = [R_i ; R_Pi_i]
// * coarse solve : M = S_Pi^{-1} (FP64),      iidx = oidx = identity on the coarse space
// * M^-1 r, part 3: M = D_i Phi_i,            iidx = R_Pi_i, oidx = R_i
// The matrices are packed per subdomain with 16-byte aligned rows and are
// streamed once per product with 128-bit loads; the gathered input of a
// subdomain sits in shared memory; a warp reduces each row with shuffles and
// scatters with FP64 atomics.  Work items are (matrix, 32-row slice), all
// subdomains of uneven size in one launch.
#include <cuda_runtime.h>

#include "bddc_internal.h"

namespace {

constexpr int GEMV_THREADS = 256;
constexpr int GEMV_MAXCOLS = 2048;     // must match the column-slice width of the work items

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
struct Vec;
template <>
struct Vec<double> {
    typedef double2 type;
    static constexpr int W = 2;
};
template <>
struct Vec<float> {
    typedef float4 type;
    static constexpr int W = 4;
};

template <class T>
__device__ __forceinline__ T dot_vec(const typename Vec<T>::type& a, const T* x);
template <>
__device__ __forceinline__ double dot_vec<double>(const double2& a, const double* x) {
    return a.x * x[0] + a.y * x[1];
}
template <>
__device__ __forceinline__ float dot_vec<float>(const float4& a, const float* x) {
    return a.x * x[0] + a.y * x[1] + a.z * x[2] + a.w * x[3];
}

template <class T>
__device__ __forceinline__ typename Vec<T>::type vzero();
template <>
__device__ __forceinline__ double2 vzero<double>() { return make_double2(0.0, 0.0); }
template <>
__device__ __forceinline__ float4 vzero<float>() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// Each warp streams two rows at a time and issues up to CH 128-bit loads per
// lane for both rows before it multiplies, so every lane keeps 2*CH loads in
// flight; the gathered input sits in shared memory.
template <class T>
__global__ void __launch_bounds__(GEMV_THREADS) k_gemv(const T* __restrict__ pool,
                                                       const GemvItem* __restrict__ items,
                                                       const int* __restrict__ idx,
                                                       const double* __restrict__ in,
                                                       double* __restrict__ out, int nrhs,
                                                       int in_ld, int out_ld,
                                                       const int* __restrict__ skip) {
    if (skip && *skip) return;
    const GemvItem it = items[blockIdx.x];
    if (it.ncols > GEMV_MAXCOLS) return;          // never built so (items are sliced); no staging overrun
    __shared__ __align__(16) T xs[GEMV_MAXCOLS];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int* iidx = idx + it.iidx_off;
    const int* oidx = idx + it.oidx_off;
    const T* M = pool + it.moff + it.col0;
    constexpr int VW = Vec<T>::W;
    constexpr int CH = 4;
    typedef typename Vec<T>::type VT;
    const int ncols = it.ncols;
    const int nvec = ncols / VW;
    const int rend = it.row0 + it.nrows;
    for (int c = 0; c < nrhs; ++c) {
        const double* inc = in + (long long)c * in_ld;
        double* outc = out + (long long)c * out_ld;
        for (int q = t; q < ncols; q += GEMV_THREADS) xs[q] = (T)inc[iidx[it.col0 + q]];
        __syncthreads();
        if (((it.moff + it.col0) % VW) != 0 || (it.ld % VW) != 0) {
            // rows not 16-byte aligned: scalar loads, several in flight per lane
            for (int r = it.row0 + 2 * wid; r < rend; r += 2 * (GEMV_THREADS / 32)) {
                const bool two = r + 1 < rend;
                const T* row0 = M + (long long)r * it.ld;
                const T* row1 = M + (long long)(two ? r + 1 : r) * it.ld;
                T acc0 = 0, acc1 = 0;
#pragma unroll 4
                for (int q = lane; q < ncols; q += 32) {
                    const T x = xs[q];
                    acc0 += __ldg(row0 + q) * x;
                    if (two) acc1 += __ldg(row1 + q) * x;
                }
                acc0 = warp_sum(acc0);
                acc1 = warp_sum(acc1);
                if (lane == 0) {
                    atomicAdd(&outc[oidx[r]], (double)acc0);
                    if (two) atomicAdd(&outc[oidx[r + 1]], (double)acc1);
                }
            }
            __syncthreads();
            continue;
        }
        for (int r = it.row0 + 2 * wid; r < rend; r += 2 * (GEMV_THREADS / 32)) {
            const bool two = r + 1 < rend;
            const VT* rv0 = reinterpret_cast<const VT*>(M + (long long)r * it.ld);
            const VT* rv1 = reinterpret_cast<const VT*>(M + (long long)(two ? r + 1 : r) * it.ld);
            T acc0 = 0, acc1 = 0;
            for (int base = 0; base < nvec; base += 32 * CH) {
                VT a0[CH], a1[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const int v = base + lane + 32 * u;
                    a0[u] = v < nvec ? __ldg(rv0 + v) : vzero<T>();
                    a1[u] = (v < nvec && two) ? __ldg(rv1 + v) : vzero<T>();
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const int v = base + lane + 32 * u;
                    if (v < nvec) {
                        acc0 += dot_vec<T>(a0[u], xs + v * VW);
                        acc1 += dot_vec<T>(a1[u], xs + v * VW);
                    }
                }
            }
            const T* row0 = M + (long long)r * it.ld;
            const T* row1 = M + (long long)(two ? r + 1 : r) * it.ld;
            for (int q = nvec * VW + lane; q < ncols; q += 32) {
                acc0 += row0[q] * xs[q];
                if (two) acc1 += row1[q] * xs[q];
            }
            acc0 = warp_sum(acc0);
            acc1 = warp_sum(acc1);
            if (lane == 0) {
                atomicAdd(&outc[oidx[r]], (double)acc0);
                if (two) atomicAdd(&outc[oidx[r + 1]], (double)acc1);
            }
        }
        __syncthreads();
    }
}

// Tall narrow operators stored transposed (cols x rows, row stride ld):
// one thread per output row, the input of the item in shared memory.
template <class T>
__global__ void __launch_bounds__(GEMV_THREADS) k_gemv_t(const T* __restrict__ pool,
                                                         const GemvItem* __restrict__ items,
                                                         const int* __restrict__ idx,
                                                         const double* __restrict__ in,
                                                         double* __restrict__ out, int nrhs,
                                                         int in_ld, int out_ld,
                                                         const int* __restrict__ skip) {
    if (skip && *skip) return;
    const GemvItem it = items[blockIdx.x];
    if (it.ncols > GEMV_MAXCOLS) return;
    __shared__ T xs[GEMV_MAXCOLS];
    const int t = threadIdx.x;
    const int* iidx = idx + it.iidx_off;
    const int* oidx = idx + it.oidx_off;
    const T* Mt = pool + it.moff;
    for (int c = 0; c < nrhs; ++c) {
        const double* inc = in + (long long)c * in_ld;
        double* outc = out + (long long)c * out_ld;
        for (int q = t; q < it.ncols; q += GEMV_THREADS) xs[q] = (T)inc[iidx[it.col0 + q]];
        __syncthreads();
        for (int r = it.row0 + t; r < it.row0 + it.nrows; r += GEMV_THREADS) {
            const T* col = Mt + (long long)it.col0 * it.ld + r;
            T acc = 0;
            int q = 0;
            // eight independent loads in flight per thread
            for (; q + 8 <= it.ncols; q += 8) {
                T a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = __ldg(col + (long long)(q + u) * it.ld);
#pragma unroll
                for (int u = 0; u < 8; ++u) acc += a[u] * xs[q + u];
            }
            for (; q < it.ncols; ++q) acc += __ldg(col + (long long)q * it.ld) * xs[q];
            atomicAdd(&outc[oidx[r]], (double)acc);
        }
        __syncthreads();
    }
}

}  // namespace

template <class T>
int gemv_run(const T* pool, const GemvItem* items_dev, int nitems, const int* idx, const double* in,
             double* out, int maxcols, int nrhs, int in_ld, int out_ld, cudaStream_t st,
             const int* skip, double bytes) {
    if (nitems <= 0) return BDDC_OK;
    (void)maxcols;                     // items are split into column slices of <= GEMV_MAXCOLS
    ktimer_begin(KT_GEMV, st);
    k_gemv<T><<<nitems, GEMV_THREADS, 0, st>>>(pool, items_dev, idx, in, out, nrhs, in_ld, out_ld,
                                               skip);
    bddc_note_launches(1);
    ktimer_end(KT_GEMV, st, 0.0, bytes * nrhs);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

template <class T>
int gemv_t_run(const T* pool, const GemvItem* items_dev, int nitems, const int* idx, const double* in,
               double* out, int nrhs, int in_ld, int out_ld, cudaStream_t st, const int* skip, double bytes) {
    if (nitems <= 0) return BDDC_OK;
    ktimer_begin(KT_GEMV, st);
    k_gemv_t<T><<<nitems, GEMV_THREADS, 0, st>>>(pool, items_dev, idx, in, out, nrhs, in_ld, out_ld, skip);
    bddc_note_launches(1);
    ktimer_end(KT_GEMV, st, 0.0, bytes * nrhs);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
template int gemv_t_run<double>(const double*, const GemvItem*, int, const int*, const double*, double*, int, int,
                                int, cudaStream_t, const int*, double);
template int gemv_t_run<float>(const float*, const GemvItem*, int, const int*, const double*, double*, int, int, int,
                               cudaStream_t, const int*, double);

template int gemv_run<double>(const double*, const GemvItem*, int, const int*, const double*,
                              double*, int, int, int, int, cudaStream_t, const int*, double);
template int gemv_run<float>(const float*, const GemvItem*, int, const int*, const double*, double*,
                             int, int, int, int, cudaStream_t, const int*, double);

// ---------------------------------------------------------------------------
// Condensation and interior recovery with the factors of the partial LU of
// A^(i) = [[L_II, 0], [L_BI, I]] [[U_II, U_IB], [0, S^(i)]]   (Sect. 3):
//   y_i = L_II^{-1} f_I,  g -= R_i^T L_BI y_i          (g^(i) = f_B - A_BI A_II^{-1} f_I)
//   u_I = U_II^{-1} (y_i - U_IB u_B)                   (u_I = A_II^{-1}(f_I - A_IB u_B))
// One CTA per subdomain; blocked left-looking substitution: all warps reduce the
// solved part into a 32-row block (several rows per warp, so that many factor
// loads are in flight), one warp solves the 32 x 32 diagonal block with
// shuffles.
// ---------------------------------------------------------------------------
namespace {

constexpr int TRI_THREADS = 256;

struct TriItem {
    long long aoff;    // matrix offset in the factor pool
    int n, nI, ld;
    int dof_off;       // offset of the local dof list (n entries: I then B)
    int gidx_off;      // offset of the interface -> Gamma list (nB entries)
    long long yoff;    // offset of the stored y_i (nI entries)
};

// The 32 x 32 diagonal block of a substitution step is staged in shared memory
// (one coalesced load) before the warp walks its dependent chain.
template <class T>
__device__ __forceinline__ void load_diag(const T* A, int ld, int b0, int bw, T (*D)[33]) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int r = wid; r < bw; r += TRI_THREADS / 32)
        if (lane < bw) D[r][lane] = A[(long long)(b0 + r) * ld + b0 + lane];
}

// s[j] = sum_{c0 <= c < c1} A[r0 + j][c] x[c] for the R rows r0 + j < rlim, by one
// warp (lanes across columns, the R rows' loads in flight together); the sums
// are returned in every lane.
template <class T, int R>
__device__ __forceinline__ void warp_rows_dot(const T* __restrict__ A, long long ld, int r0, int rlim, int c0,
                                              int c1, const T* x, T (&s)[R]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < R; ++j) s[j] = (T)0;
#pragma unroll 4
    for (int c = c0 + lane; c < c1; c += 32) {
        const T xv = x[c];
#pragma unroll
        for (int j = 0; j < R; ++j)
            if (r0 + j < rlim) s[j] += A[(long long)(r0 + j) * ld + c] * xv;
    }
#pragma unroll
    for (int j = 0; j < R; ++j) s[j] = warp_sum(s[j]);
}

// y <- L^{-1} y, L unit lower (the strictly lower part of A's leading nI x nI
// block).  Left-looking: the 32 rows of a block first subtract the solved
// columns (four rows per warp, all eight warps), then warp 0 finishes the block.
template <class T>
__device__ void fwd_unit_lower(const T* A, int ld, int nI, T* y) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    __shared__ T D[32][33];
    for (int b0 = 0; b0 < nI; b0 += 32) {
        const int bw = min(32, nI - b0);
        load_diag(A, ld, b0, bw, D);
        if (b0 > 0) {
            T s[4];
            warp_rows_dot<T, 4>(A, ld, b0 + 4 * wid, b0 + bw, 0, b0, y, s);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (lane == 0 && 4 * wid + j < bw) y[b0 + 4 * wid + j] -= s[j];
        }
        __syncthreads();
        if (wid == 0) {
            T v = lane < bw ? y[b0 + lane] : (T)0;
            for (int k = 0; k < bw; ++k) {
                T vk = __shfl_sync(0xffffffffu, v, k);
                if (lane > k && lane < bw) v -= D[lane][k] * vk;
            }
            if (lane < bw) y[b0 + lane] = v;
        }
        __syncthreads();
    }
}

// y <- U^{-1} y, U the upper part of A's leading nI x nI block; left-looking
// from the last block.
template <class T>
__device__ void bwd_upper(const T* A, int ld, int nI, T* y) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    __shared__ T D[32][33];
    for (int b1 = nI; b1 > 0; b1 -= 32) {
        const int b0 = max(0, b1 - 32);
        const int bw = b1 - b0;
        load_diag(A, ld, b0, bw, D);
        if (b1 < nI) {
            T s[4];
            warp_rows_dot<T, 4>(A, ld, b0 + 4 * wid, b1, b1, nI, y, s);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (lane == 0 && 4 * wid + j < bw) y[b0 + 4 * wid + j] -= s[j];
        }
        __syncthreads();
        if (wid == 0) {
            T v = lane < bw ? y[b0 + lane] : (T)0;
            for (int k = bw - 1; k >= 0; --k) {
                if (lane == k) v /= D[k][k];
                T vk = __shfl_sync(0xffffffffu, v, k);
                if (lane < k) v -= D[lane][k] * vk;
            }
            if (lane < bw) y[b0 + lane] = v;
        }
        __syncthreads();
    }
}

// Forward half of the condensation: y = L_II^{-1} f_I, stored negated (the
// batched GEMV then adds L_BI (-y) to g, and recovery continues from it).
template <class T>
__global__ void __launch_bounds__(TRI_THREADS) k_condense(const T* __restrict__ pool,
                                                          const TriItem* __restrict__ items,
                                                          const int* __restrict__ lists,
                                                          const double* __restrict__ F,
                                                          double* __restrict__ ystore, int nrhs,
                                                          long long ldF, long long ldY) {
    const TriItem it = items[blockIdx.x];
    extern __shared__ __align__(16) unsigned char tri_raw[];
    T* y = reinterpret_cast<T*>(tri_raw);          // nI entries (the launch sizes it for the largest)
    const int t = threadIdx.x;
    const T* A = pool + it.aoff;
    const int* dofs = lists + it.dof_off;
    for (int c = 0; c < nrhs; ++c) {
        for (int q = t; q < it.nI; q += TRI_THREADS) y[q] = (T)F[c * ldF + dofs[q]];
        __syncthreads();
        fwd_unit_lower<T>(A, it.ld, it.nI, y);
        for (int q = t; q < it.nI; q += TRI_THREADS) ystore[c * ldY + it.yoff + q] = -(double)y[q];
        __syncthreads();
    }
}

// Backward half of the recovery: ystore holds -(y - U_IB u_B) (the batched GEMV
// has added U_IB u_B to -y); u_I = U_II^{-1} (y - U_IB u_B), u_B copied.  uG may
// be u itself (the child boxes of local nested dissection recover from the
// solution already written on their boundaries), so neither is restrict.
template <class T>
__global__ void __launch_bounds__(TRI_THREADS) k_recover(const T* __restrict__ pool,
                                                         const TriItem* __restrict__ items,
                                                         const int* __restrict__ lists,
                                                         const double* uG,
                                                         const double* __restrict__ ystore,
                                                         double* u, int nrhs,
                                                         long long ldG, long long ldU,
                                                         long long ldY) {
    const TriItem it = items[blockIdx.x];
    extern __shared__ __align__(16) unsigned char tri_raw[];
    T* y = reinterpret_cast<T*>(tri_raw);          // nI entries (the launch sizes it for the largest)
    const int t = threadIdx.x;
    const T* A = pool + it.aoff;
    const int* dofs = lists + it.dof_off;
    const int* gidx = lists + it.gidx_off;
    const int nB = it.n - it.nI;
    for (int c = 0; c < nrhs; ++c) {
        for (int q = t; q < it.nI; q += TRI_THREADS) y[q] = (T)(-ystore[c * ldY + it.yoff + q]);
        __syncthreads();
        bwd_upper<T>(A, it.ld, it.nI, y);
        for (int q = t; q < it.nI; q += TRI_THREADS) u[c * ldU + dofs[q]] = (double)y[q];
        for (int q = t; q < nB; q += TRI_THREADS) u[c * ldU + dofs[it.nI + q]] = uG[c * ldG + gidx[q]];
        __syncthreads();
    }
}

}  // namespace

struct TriBatch {
    TriItem* items;
    int count;
};

// Dynamic shared memory of the substitution kernels: the largest interior vector.
template <class T, class K>
static int tri_smem(K kern, int maxnI, size_t* bytes) {
    if (maxnI < 1 || maxnI > BDDC_MAX_INTERIOR) return BDDC_EINVAL;
    *bytes = (size_t)maxnI * sizeof(T);
    if (*bytes > 48 * 1024)
        BDDC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*bytes));
    return BDDC_OK;
}

template <class T>
int condense_run(const T* pool, const void* items, int count, int maxnI, const int* lists, const double* F,
                 double* g, double* ystore, int nrhs, long long ldF, long long ldG, long long ldY,
                 const GemvItem* ci, int nci, double ci_bytes, cudaStream_t st) {
    size_t sm = 0;
    BDDC_TRY(tri_smem<T>(k_condense<T>, maxnI, &sm));
    ktimer_begin(KT_TRI, st);
    k_condense<T><<<count, TRI_THREADS, sm, st>>>(pool, (const TriItem*)items, lists, F, ystore, nrhs, ldF, ldY);
    ktimer_end(KT_TRI, st, 0.0, 0.0);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    // g += L_BI (-y)
    return gemv_run<T>(pool, ci, nci, lists, ystore, g, 0, nrhs, (int)ldY, (int)ldG, st, nullptr, ci_bytes);
}

template <class T>
int recover_run(const T* pool, const void* items, int count, int maxnI, const int* lists, const double* uG,
                double* ystore, double* u, int nrhs, long long ldG, long long ldU,
                long long ldY, const GemvItem* ri, int nri, double ri_bytes, cudaStream_t st) {
    // -y += U_IB u_B
    BDDC_TRY(gemv_run<T>(pool, ri, nri, lists, uG, ystore, 0, nrhs, (int)ldG, (int)ldY, st, nullptr, ri_bytes));
    size_t sm = 0;
    BDDC_TRY(tri_smem<T>(k_recover<T>, maxnI, &sm));
    ktimer_begin(KT_TRI, st);
    k_recover<T><<<count, TRI_THREADS, sm, st>>>(pool, (const TriItem*)items, lists, uG, ystore, u,
                                                nrhs, ldG, ldU, ldY);
    ktimer_end(KT_TRI, st, 0.0, 0.0);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

size_t tri_item_size() { return sizeof(TriItem); }
void tri_item_fill(void* dst, long long aoff, int n, int nI, int ld, int dof_off, int gidx_off,
                   long long yoff) {
    TriItem* t = (TriItem*)dst;
    t->aoff = aoff;
    t->n = n;
    t->nI = nI;
    t->ld = ld;
    t->dof_off = dof_off;
    t->gidx_off = gidx_off;
    t->yoff = yoff;
}

template int condense_run<double>(const double*, const void*, int, int, const int*, const double*, double*, double*,
                                  int, long long, long long, long long, const GemvItem*, int, double, cudaStream_t);
template int condense_run<float>(const float*, const void*, int, int, const int*, const double*, double*, double*,
                                 int, long long, long long, long long, const GemvItem*, int, double, cudaStream_t);
template int recover_run<double>(const double*, const void*, int, int, const int*, const double*, double*, double*,
                                 int, long long, long long, long long, const GemvItem*, int, double, cudaStream_t);
template int recover_run<float>(const float*, const void*, int, int, const int*, const double*, double*, double*,
                                int, long long, long long, long long, const GemvItem*, int, double, cudaStream_t);

// ---------------------------------------------------------------------------
// small vector kernels
// ---------------------------------------------------------------------------
__global__ void k_gather(const double* __restrict__ src, const int* __restrict__ idx,
                         double* __restrict__ dst, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

int gather_run(const double* src, const int* idx, double* dst, int n, cudaStream_t st) {
    if (n <= 0) return BDDC_OK;
    k_gather<<<(n + 255) / 256, 256, 0, st>>>(src, idx, dst, n);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
