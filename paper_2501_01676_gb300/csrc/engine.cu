// Batched partial LU without pivoting ("Schur engine").
//
// For every item (a dense n x n row-major matrix M) eliminate the leading k
// unknowns in place:
//
//   M = [ M11 M12 ]  ->  [ L11\U11   U12             ]
//       [ M21 M22 ]      [ L21       M22 - L21 U12    ]
//
// so the trailing (n-k) x (n-k) block becomes the Schur complement
// M22 - M21 M11^{-1} M12.  This one operation forms the subdomain Schur
// complements S^(i) = A_BB - A_BI A_II^{-1} A_IB (Sect. 3), the face and
// edge Schur complements of B^(i) used by the GEPs (Sect. 3), the
// constrained local solvers and coarse bases (block elimination of S~), and
// the explicit inverse of the coarse matrix.  Pivoting is not needed: every
// eliminated block has a positive definite symmetric part (the forms b_i are
// SPD and the primal constraints remove the constants), for which LU without
// pivoting exists.  Zero / non-finite pivots are flagged, not trapped.
//
// Right-looking blocked algorithm, panel width NB.  Per panel two launches
// batched over all items: (1) factor the NB x NB diagonal block (redundantly
// in every CTA, in shared memory) and solve for the L21 row chunks and the
// U12 column chunks; (2) the trailing update M22 -= L21 U12 in 64 x 64
// tiles, register-blocked 4 x 4 per thread.
#include <cuda_runtime.h>

#include <algorithm>

#include "bddc_internal.h"

namespace {

constexpr int PANEL_THREADS = 128;
constexpr int CHUNK = 128;            // rows (or columns) per panel CTA
constexpr int TILE = 64;
constexpr int UPD_THREADS = 256;

template <class T>
__device__ __forceinline__ bool bad_pivot(T v) {
    return !(fabs((double)v) > 1e-300) || !isfinite((double)v);
}

template <class T, int NB>
__global__ void __launch_bounds__(PANEL_THREADS) k_panel(const EngItem<T>* __restrict__ items, int p,
                                                         T* __restrict__ dscr, int* __restrict__ err) {
    static_assert(NB == 32, "one lane per panel column");
    const EngItem<T> it = items[blockIdx.x];
    if (p >= it.k) return;
    const int w = min(NB, it.k - p);
    const int n = it.n, ld = it.ld;
    const int m0 = p + w;                      // first trailing index
    const int mrem = n - m0;
    const int nch = (mrem + CHUNK - 1) / CHUNK;
    const int y = blockIdx.y;
    if (y > 2 * nch) return;
    __shared__ T D[NB][NB + 1];
    __shared__ T W[NB][CHUNK + 1];             // row chunk (transposed) or column chunk
    T* A = it.a;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    constexpr int NW = PANEL_THREADS / 32;
    for (int r = wid; r < w; r += NW)
        if (lane < w) D[r][lane] = A[(long long)(p + r) * ld + p + lane];
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        T piv = D[j][j];
        if (bad_pivot(piv)) {
            if (t == 0 && y == 0) atomicOr(err, ERR_PIVOT);
            piv = (T)1;
        }
        if (t > j && t < w) D[t][j] /= piv;
        __syncthreads();
        for (int i = j + 1 + wid; i < w; i += NW)
            if (lane > j && lane < w) D[i][lane] -= D[i][j] * D[j][lane];
        __syncthreads();
    }
    if (y == 0) {
        T* ds = dscr + (long long)blockIdx.x * NB * NB;
        for (int r = wid; r < w; r += NW)
            if (lane < w) ds[r * w + lane] = D[r][lane];
        return;
    }
    if (y <= nch) {
        // rows r0 .. r0+CHUNK of L21 = M21 U11^{-1}
        const int r0 = m0 + (y - 1) * CHUNK;
        const int nr = min(CHUNK, n - r0);
        for (int r = wid; r < nr; r += NW)
            if (lane < w) W[lane][r] = A[(long long)(r0 + r) * ld + p + lane];
        __syncthreads();
        if (t < nr) {
            for (int j = 0; j < w; ++j) {
                T x = W[j][t];
                for (int l = 0; l < j; ++l) x -= W[l][t] * D[l][j];
                T piv = D[j][j];
                if (bad_pivot(piv)) piv = (T)1;
                W[j][t] = x / piv;
            }
        }
        __syncthreads();
        for (int r = wid; r < nr; r += NW)
            if (lane < w) A[(long long)(r0 + r) * ld + p + lane] = W[lane][r];
    } else {
        // columns c0 .. c0+CHUNK of U12 = L11^{-1} M12
        const int c0 = m0 + (y - 1 - nch) * CHUNK;
        const int nc = min(CHUNK, n - c0);
        for (int r = 0; r < w; ++r)
            for (int c = t; c < nc; c += PANEL_THREADS) W[r][c] = A[(long long)(p + r) * ld + c0 + c];
        __syncthreads();
        if (t < nc) {
            for (int i = 1; i < w; ++i) {
                T x = W[i][t];
                for (int l = 0; l < i; ++l) x -= D[i][l] * W[l][t];
                W[i][t] = x;
            }
        }
        __syncthreads();
        for (int r = 0; r < w; ++r)
            for (int c = t; c < nc; c += PANEL_THREADS) A[(long long)(p + r) * ld + c0 + c] = W[r][c];
    }
}

template <class T>
__device__ __forceinline__ void lds4(const T* p, T out[4]);
template <>
__device__ __forceinline__ void lds4<float>(const float* p, float out[4]) {
    float4 v = *reinterpret_cast<const float4*>(p);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <>
__device__ __forceinline__ void lds4<double>(const double* p, double out[4]) {
    double2 v0 = *reinterpret_cast<const double2*>(p);
    double2 v1 = *reinterpret_cast<const double2*>(p + 2);
    out[0] = v0.x; out[1] = v0.y; out[2] = v1.x; out[3] = v1.y;
}

template <class T, int NB>
__global__ void __launch_bounds__(UPD_THREADS) k_update(const EngItem<T>* __restrict__ items, int p,
                                                        const T* __restrict__ dscr) {
    const EngItem<T> it = items[blockIdx.x];
    if (p >= it.k) return;
    const int w = min(NB, it.k - p);
    const int n = it.n, ld = it.ld;
    const int m0 = p + w;
    const int mrem = n - m0;
    const int nt = (mrem + TILE - 1) / TILE;
    const int y = blockIdx.y;
    T* A = it.a;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (y == 0) {
        const T* ds = dscr + (long long)blockIdx.x * NB * NB;
        for (int r = wid; r < w; r += UPD_THREADS / 32)
            if (lane < w) A[(long long)(p + r) * ld + p + lane] = ds[r * w + lane];
        return;
    }
    if (y > nt * nt) return;
    const int ti = (y - 1) / nt, tj = (y - 1) - ti * nt;
    const int r0 = m0 + ti * TILE, c0 = m0 + tj * TILE;
    constexpr int LDT = TILE + 4;      // 16-byte aligned rows for vector loads
    __shared__ __align__(16) T Ls[NB][LDT];    // L21 tile, transposed: Ls[k][r]
    __shared__ __align__(16) T Us[NB][LDT];    // U12 tile: Us[k][c]
    for (int r = wid; r < TILE; r += UPD_THREADS / 32) {
        int gr = r0 + r;
        if (lane < w) Ls[lane][r] = gr < n ? A[(long long)gr * ld + p + lane] : (T)0;
    }
    for (int k = t >> 6; k < w; k += UPD_THREADS / TILE) {
        int c = t & (TILE - 1);
        int gc = c0 + c;
        Us[k][c] = gc < n ? A[(long long)(p + k) * ld + gc] : (T)0;
    }
    __syncthreads();
    const int tr = (t >> 4) * 4, tc = (t & 15) * 4;   // 16 x 16 threads, a 4 x 4 block each
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    for (int k = 0; k < w; ++k) {
        T lv[4], uv[4];
        lds4<T>(&Ls[k][tr], lv);
        lds4<T>(&Us[k][tc], uv);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += lv[a] * uv[b];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int gr = r0 + tr + a;
        if (gr >= n) continue;
        T* row = A + (long long)gr * ld;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int gc = c0 + tc + b;
            if (gc < n) row[gc] -= acc[a][b];
        }
    }
}

}  // namespace

template <class T>
static int launch_update(const EngItem<T>* items_dev, int count, int maxn, int p, T* dscr, int* err, cudaStream_t st,
                         bool tc);
template <>
int launch_update<double>(const EngItem<double>* items_dev, int count, int maxn, int p, double* dscr, int* err,
                          cudaStream_t st, bool tc) {
    (void)tc;
    (void)err;
    const int nt = (maxn - p + TILE - 1) / TILE;
    k_update<double, 32><<<dim3(count, 1 + nt * nt), UPD_THREADS, 0, st>>>(items_dev, p, dscr);
    bddc_note_launches(1);
    return BDDC_OK;
}
template <>
int launch_update<float>(const EngItem<float>* items_dev, int count, int maxn, int p, float* dscr, int* err,
                         cudaStream_t st, bool tc) {
    if (tc) return tc_update_run(items_dev, count, maxn, p, dscr, err, st);
    const int nt = (maxn - p + TILE - 1) / TILE;
    k_update<float, 32><<<dim3(count, 1 + nt * nt), UPD_THREADS, 0, st>>>(items_dev, p, dscr);
    bddc_note_launches(1);
    return BDDC_OK;
}

template <class T>
int engine_run(const EngItem<T>* items_dev, int count, int maxn, int maxk, T* dscr, int* err,
               cudaStream_t st, const int* hn, const int* hk, bool tc) {
    constexpr int NB = 32;
    if (count <= 0 || maxk <= 0) return BDDC_OK;
    for (int p = 0; p < maxk; p += NB) {
        int mrem = maxn - p;                 // upper bound of the trailing size
        int nch = (mrem + CHUNK - 1) / CHUNK;
        int nt = (mrem + TILE - 1) / TILE;
        // algorithmic work of this panel: trailing update 2 m^2 w, panel solves ~ 2 w^2 m
        double fu = 0.0, fp = 0.0, bu = 0.0;
        if (hn && (ktimer_on(KT_ENGINE_UPDATE) || ktimer_on(KT_ENGINE_PANEL)))
            for (int i = 0; i < count; ++i) {
                if (p >= hk[i]) continue;
                double w = std::min(NB, hk[i] - p), m = hn[i] - p - w;
                fu += 2.0 * m * m * w;
                fp += 2.0 * w * w * m;
                bu += sizeof(T) * (2.0 * m * m + 2.0 * m * w);   // read + write M22, read L21, U12
            }
        ktimer_begin(KT_ENGINE_PANEL, st);
        k_panel<T, NB><<<dim3(count, 1 + 2 * nch), PANEL_THREADS, 0, st>>>(items_dev, p, dscr, err);
        bddc_note_launches(1);
        ktimer_end(KT_ENGINE_PANEL, st, fp, 0.0);
        ktimer_begin(KT_ENGINE_UPDATE, st);
        BDDC_TRY(launch_update<T>(items_dev, count, maxn, p, dscr, err, st, tc));
        ktimer_end(KT_ENGINE_UPDATE, st, fu, bu);
        (void)nt;
    }
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

template int engine_run<double>(const EngItem<double>*, int, int, int, double*, int*, cudaStream_t,
                                const int*, const int*, bool);
template int engine_run<float>(const EngItem<float>*, int, int, int, float*, int*, cudaStream_t,
                               const int*, const int*, bool);
