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
// pivoting exists.  Zero / non-finite pivots are flagged (and replaced by 1),
// not trapped.
//
// Right-looking blocked algorithm, panel width NB (128 in FP32, 64 in FP64).
// Per panel three kinds of task, each batched over all items:
//   diagonal  one CTA factors the NB x NB diagonal block in shared memory, 32
//             columns at a time (one warp factors the 32 x 32 sub-block in
//             registers, one thread per row / column solves the strips, a
//             register-tiled rank-32 update), writes L11\U11 back and the pivot
//             reciprocals to a scratch; on the tensor-core path it also forms
//             U11^{-1} and L11^{-1} (packed in one NB x NB scratch block);
//   strip     L21 = M21 U11^{-1} and U12 = L11^{-1} M12: on the tensor-core path
//             as products with the inverses on 128-row / -column chunks; on the
//             CUDA cores by substitution in 64-row / -column chunks (U12 solved
//             transposed, so both run the same code: per 32-column block a
//             thread-per-row substitution, then a right-looking update of the
//             later columns);
//   update    M22 -= L21 U12 in TILE x TILE tiles: on the tensor cores (tcgen05,
//             split TF32, FP32 path by default) or on the CUDA cores (register
//             tiles, K staged through shared memory in chunks of 32).
// One persistent task kernel runs all panels of all items (below); with the
// kernel timer on, per-panel launches k_diag, k_trsm, k_update (or the
// tensor-core k_tc_update) run the same bodies.  A wider panel divides the passes
// over the trailing matrices (the HBM traffic of the update) by the width:
// NB = 128 does a quarter of the passes of a 32-wide panel.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "bddc_internal.h"
#include "tc_common.cuh"
#include <cuda_bf16.h>

namespace {

template <class T>
struct EngCfg;
template <>
struct EngCfg<float> {
    static constexpr int NB = 128, TILE = 128;
};
template <>
struct EngCfg<double> {
    static constexpr int NB = 64, TILE = 64;
};

constexpr int DIAG_THREADS = 256;     // small, so that it fits beside an update CTA (look-ahead)
constexpr int TRSM_THREADS = 256;
constexpr int UPD_THREADS = 256;
constexpr int CH = 64;      // rows (columns) of L21 (U12) per k_trsm CTA
constexpr int KC = 32;      // K chunk of the update
constexpr int IB = 32;      // inner block of the diagonal factorisation

__device__ __forceinline__ bool bad_pivot(double v) { return !(fabs(v) > 1e-300) || !isfinite(v); }
__device__ __forceinline__ bool bad_pivot(float v) { return !(fabsf(v) > 0.f) || !isfinite(v); }

// 16-byte shared-memory load into out[0 .. 16 / sizeof(T) - 1]
template <class T>
__device__ __forceinline__ void lds16(const T* p, T* out);
template <>
__device__ __forceinline__ void lds16<float>(const float* p, float* out) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <>
__device__ __forceinline__ void lds16<double>(const double* p, double* out) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    out[0] = v.x; out[1] = v.y;
}

// Per-item scratch: the reciprocal pivots of every panel (NB per panel, so that
// a panel's pivots stay valid while the next panel is factored in the task
// kernel); `stride` elements per item.

constexpr int TS = IB + 4;          // row length of the shifted triangle copies (16-byte rows, conflict-free writes)

// One warp factors the bw x bw block Db (bw <= 32, leading dimension LD) in
// registers: lane c holds column c.  Step j broadcasts the pivot and the
// unscaled column j from lane j (all 32 shuffles first, off the pivot's
// dependency chain); the lanes right of j subtract x(j + r, j) * (U(j, c) /
// pivot), one FMA per entry.  Column j itself stays unscaled in registers: each
// lane keeps its pivot reciprocal and scales its L entries when they are
// written out.  The rows are shifted down one register per step (row j + 1
// moves to x[0]), so every register index is static inside a compact loop.
// Row j is final after step j: it is written back to Db and, shifted so that
// the distance from the diagonal is the column index, to Us[j][c - j] = U(j, c)
// (c > j) and Ls[c][j - c] = L(j, c) (j > c); the strip solves read those rows
// as 16-byte vectors.  Rows and columns past bw are padded with the identity (no
// effect on the real part).
template <class T>
__device__ __forceinline__ void lu_warp32(T* __restrict__ Db, int LD, int bw, T* __restrict__ dv,
                                          T* __restrict__ Us, T* __restrict__ Ls, int* __restrict__ err,
                                          int lane) {
    T x[IB];
#pragma unroll
    for (int r = 0; r < IB; ++r) x[r] = (r < bw && lane < bw) ? Db[r * LD + lane] : (r == lane ? (T)1 : (T)0);
    T myri = (T)1;
#pragma unroll 1
    for (int j = 0; j < IB; ++j) {
        // FP32: all shuffles up front (32 more registers); FP64: next to their FMAs
        constexpr int NS = sizeof(T) == 4 ? IB : 1;
        T sv[NS];
#pragma unroll
        for (int r = 0; r < NS; ++r) sv[r] = __shfl_sync(0xffffffffu, x[r], j);
        T piv = sv[0];
        const bool bad = bad_pivot(piv);
        if (bad) piv = (T)1;
        const T ri = (T)1 / piv;
        myri = lane == j ? ri : myri;
        // row j: L(j, c) for c < j (scaled now), the pivot, U(j, c) for c > j
        const T rowv = lane < j ? x[0] * myri : (lane == j ? piv : x[0]);
        const T m = lane > j ? x[0] * ri : (T)0;
#pragma unroll
        for (int r = 1; r < IB; ++r)
            x[r - 1] = x[r] - (NS == IB ? sv[r % NS] : __shfl_sync(0xffffffffu, x[r], j)) * m;
        x[IB - 1] = (T)0;
        if (j < bw && lane < bw) Db[j * LD + lane] = rowv;
        if (lane == j && j < bw) {
            dv[j] = ri;
            if (bad) atomicOr(err, ERR_PIVOT);
        }
        if (lane > j) Us[j * TS + lane - j] = rowv;
        if (lane < j) Ls[lane * TS + j - lane] = rowv;
    }
}

// Rank-32 update of the trailing block of the diagonal block (rows and columns
// b0 + 32 .. w - 1): 16 x 16 threads, thread (ty, tx) owns rows b0 + 32 + ty + 16 i
// and columns b0 + 32 + tx + 16 j, i, j < MR (MR = the stage's ceil(rem / 16),
// rounded up to the instantiated sizes).
template <class T, int MR>
__device__ __forceinline__ void diag_rank32(T* __restrict__ D, int LD, int b0, int w, int t) {
    const int base = b0 + IB;
    const int ty = t >> 4, tx = t & 15;
    T acc[MR][MR];
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int j = 0; j < MR; ++j) acc[i][j] = (T)0;
#pragma unroll 2
    for (int l = 0; l < IB; ++l) {
        T a[MR], b[MR];
#pragma unroll
        for (int i = 0; i < MR; ++i) {
            const int r = base + ty + 16 * i, c = base + tx + 16 * i;
            a[i] = r < w ? D[r * LD + b0 + l] : (T)0;
            b[i] = c < w ? D[(b0 + l) * LD + c] : (T)0;
        }
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MR; ++j) acc[i][j] += a[i] * b[j];
    }
#pragma unroll
    for (int i = 0; i < MR; ++i) {
        const int r = base + ty + 16 * i;
#pragma unroll
        for (int j = 0; j < MR; ++j) {
            const int c = base + tx + 16 * j;
            if (r < w && c < w) D[r * LD + c] -= acc[i][j];
        }
    }
}

// LU of the w x w diagonal block in shared memory, 32 columns at a time.  Per
// 32-column stage b0:
//   (1) one warp factors the 32 x 32 block (lu_warp32);
//   (2) the rows below it solve y <- y U^{-1} and the columns right of it
//       z <- L^{-1} z, one thread per row / column with the 32 values in
//       registers (same shift-down scheme: the value finished in step c leaves
//       through y[0], U(c, c + l) / L(c + l, c) come from the shifted triangle
//       copies, 16 bytes per load; the slots past the block hold stale values
//       that never reach a real one);
//   (3) the rank-32 update of the trailing block, 16 x 16 threads with register
//       tiles.
// Three barriers per stage instead of one per pivot; the loops stay compact
// (this body runs once per launch: straight-line code would be fetched from
// beyond the instruction cache).
// In-place inverses of the factors of the w x w diagonal block in shared memory
// (after its LU; w <= 4 * 32, leading dimension LD): afterwards the upper
// triangle with the diagonal holds U11^{-1} and the strict lower triangle the
// strict lower part of L11^{-1} (whose diagonal is 1).  Blocked by 32:
//   (1) the diagonal blocks: warp 2b inverts U_bb, warp 2b + 1 the unit lower
//       L_bb, lane c computing column c in registers (U_bb^{-1} from the pivot
//       reciprocals dinv);
//   (2) the off-diagonal blocks from the block rows of X U = I and Y L = I,
//       X_ab = -(sum_{a <= c < b} X_ac U_cb) X_bb   (a < b),
//       Y_ab = -(sum_{b < c <= a} Y_ac L_cb) Y_bb   (a > b),
//       one block column per step and factor (X: columns left to right, Y: right
//       to left), all blocks of the column at once: the products read only blocks
//       of finished columns and the column's own factor blocks, which are
//       overwritten after a barrier.  Threads 0..127 take X, 128..255 Y, each 8
//       entries per block (row tid / 4, columns 8 (tid % 4) ..); the sums and a
//       masked copy of the column's diagonal inverse block go through tmp
//       (8 blocks of 32 x 33).
// The padding of the last 32-block is zeroed first, so that no stale value
// enters a product.
template <class T>
__device__ void diag_inverse(T* __restrict__ D, int LD, int w, const T* __restrict__ dinv, T* __restrict__ tmp,
                             int t) {
    const int nbk = (w + IB - 1) / IB, W32 = nbk * IB;
    for (int q = t; q < W32 * W32; q += DIAG_THREADS) {
        const int r = q / W32, c = q - r * W32;
        if (r >= w || c >= w) D[r * LD + c] = (T)0;
    }
    __syncthreads();
    const int wid = t >> 5, lane = t & 31;
    if ((wid >> 1) < nbk) {
        const int b0 = IB * (wid >> 1), bw = min(IB, w - b0);
        T* Bk = D + b0 * LD + b0;
        T x[IB];
        if ((wid & 1) == 0) {
#pragma unroll
            for (int i = IB - 1; i >= 0; --i) {
                T s = (T)0;
#pragma unroll
                for (int l = i + 1; l < IB; ++l) s += Bk[i * LD + l] * x[l];
                const T di = i < bw ? dinv[b0 + i] : (T)0;
                x[i] = i == lane ? di : (i < lane ? -s * di : (T)0);
            }
            __syncwarp();
            if (lane < bw)
#pragma unroll
                for (int i = 0; i < IB; ++i)
                    if (i <= lane) Bk[i * LD + lane] = x[i];
        } else {
#pragma unroll
            for (int i = 0; i < IB; ++i) {
                T s = (T)0;
#pragma unroll
                for (int l = 0; l < i; ++l) s += Bk[i * LD + l] * x[l];
                x[i] = i == lane ? (T)1 : ((i > lane && i < bw) ? -s : (T)0);
            }
            __syncwarp();
            if (lane < bw)
#pragma unroll
                for (int i = 0; i < IB; ++i)
                    if (i > lane && i < bw) Bk[i * LD + lane] = x[i];
        }
    }
    __syncthreads();
    // off-diagonal blocks from X U = I and Y L = I, one block column per step and
    // factor, all its blocks at once (reads of the column's factor blocks precede
    // the writes of its inverse blocks):
    //   X_ab = -(sum_{a <= c < b} X_ac U_cb) X_bb   (a < b, columns b = 1 .. nbk-1),
    //   Y_ab = -(sum_{b < c <= a} Y_ac L_cb) Y_bb   (a > b, columns b = nbk-2 .. 0)
    const bool up = t < DIAG_THREADS / 2;
    const int tu = up ? t : t - DIAG_THREADS / 2;
    const int r = tu >> 2, j0 = (tu & 3) * 8;
    constexpr int BS = IB * (IB + 1);
    T* Tb = tmp + (up ? 0 : 4 * BS);          // up to 3 product blocks and the masked diagonal block
    T* Db = Tb + 3 * BS;
#pragma unroll 1
    for (int s = 0; s + 1 < nbk; ++s) {
        const int b = up ? s + 1 : nbk - 2 - s;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const int j = j0 + jj;
            const T v = D[(IB * b + r) * LD + IB * b + j];
            Db[r * (IB + 1) + j] = up ? (r <= j ? v : (T)0) : (r > j ? v : (r == j ? (T)1 : (T)0));
        }
#pragma unroll 1
        for (int q = 0; q <= s; ++q) {
            const int a = up ? q : b + 1 + q;
            const int c0 = up ? a : b + 1, c1 = up ? b - 1 : a;
            T acc[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) acc[jj] = (T)0;
#pragma unroll 1
            for (int c = c0; c <= c1; ++c) {
                const T* F = D + (IB * a + r) * LD + IB * c;    // X_ac / Y_ac, row r
                const T* G = D + (IB * c) * LD + IB * b + j0;   // U_cb / L_cb
                if (c == a) {
                    // the diagonal inverse block: X_aa upper with its diagonal, Y_aa unit lower
#pragma unroll 4
                    for (int k = 0; k < IB; ++k) {
                        T f = F[k];
                        f = up ? (k >= r ? f : (T)0) : (k < r ? f : (k == r ? (T)1 : (T)0));
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) acc[jj] += f * G[k * LD + jj];
                    }
                } else {
#pragma unroll 4
                    for (int k = 0; k < IB; ++k) {
                        const T f = F[k];
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) acc[jj] += f * G[k * LD + jj];
                    }
                }
            }
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) Tb[q * BS + r * (IB + 1) + j0 + jj] = acc[jj];
        }
        __syncthreads();
#pragma unroll 1
        for (int q = 0; q <= s; ++q) {
            const int a = up ? q : b + 1 + q;
            T acc[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) acc[jj] = (T)0;
#pragma unroll 4
            for (int k = 0; k < IB; ++k) {
                const T f = Tb[q * BS + r * (IB + 1) + k];
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) acc[jj] += f * Db[k * (IB + 1) + j0 + jj];
            }
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) D[(IB * a + r) * LD + IB * b + j0 + jj] = -acc[jj];
        }
        __syncthreads();
    }
}

template <class T, int NB, bool INV = false>
__device__ __noinline__ void diag_body(const EngItem<T>& it, int p, T* __restrict__ out, int* __restrict__ err,
                          unsigned char* dsm, T* __restrict__ inv = nullptr) {
    static_assert(NB - IB <= DIAG_THREADS / 2, "one thread per strip row / column");
    const int w = min(NB, it.k - p);
    const long long ld = it.ld;
    T* A = it.a + (long long)p * ld + p;
    constexpr int LD = NB + 1;
    constexpr int MR = (NB - IB + 15) / 16;  // register tile of the trailing update
    T* D = reinterpret_cast<T*>(dsm);        // NB x LD: L\U of the diagonal block
    T* dinv = D + NB * LD;                    // NB reciprocal pivots
    T* Ut = dinv + NB;                        // IB x TS: Ut[c][l] = U(b0 + c, b0 + c + l)
    T* Lt = Ut + IB * TS;                     // IB x TS: Lt[r][l] = L(b0 + r + l, b0 + r)
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    // thread t reads column t % NB of rows t / NB + RPI u, 16 loads in flight
    constexpr int RPI = DIAG_THREADS / NB;
    const int lc = t % NB, lr = t / NB;
#pragma unroll 1
    for (int r0 = 0; r0 < w; r0 += 16 * RPI) {
        T v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int r = r0 + lr + u * RPI;
            if (r < w && lc < w) v[u] = __ldcg(A + r * ld + lc);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int r = r0 + lr + u * RPI;
            if (r < w && lc < w) D[r * LD + lc] = v[u];
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int b0 = 0; b0 < w; b0 += IB) {
        const int bw = min(IB, w - b0);
        const int rem = w - b0 - bw;
        if (wid == 0) lu_warp32<T>(D + b0 * LD + b0, LD, bw, dinv + b0, Ut, Lt, err, lane);
        __syncthreads();
        if (rem <= 0) break;
        const int base = b0 + IB;
        if (t < DIAG_THREADS / 2) {
            const int r = base + t;
            if (r < w) {
                T y[IB];
#pragma unroll
                for (int l = 0; l < IB; ++l) y[l] = D[r * LD + b0 + l];
#pragma unroll 1
                for (int c = 0; c < IB; ++c) {
                    T u[IB];
#pragma unroll
                    for (int q = 0; q < IB; q += 16 / (int)sizeof(T)) lds16<T>(Ut + c * TS + q, u + q);
                    const T z = y[0] * dinv[b0 + c];
                    D[r * LD + b0 + c] = z;
#pragma unroll
                    for (int l = 1; l < IB; ++l) y[l - 1] = y[l] - z * u[l];
                }
            }
        } else {
            const int cc = base + t - DIAG_THREADS / 2;
            if (cc < w) {
                T y[IB];
#pragma unroll
                for (int l = 0; l < IB; ++l) y[l] = D[(b0 + l) * LD + cc];
#pragma unroll 1
                for (int r = 0; r < IB; ++r) {
                    T lt[IB];
#pragma unroll
                    for (int q = 0; q < IB; q += 16 / (int)sizeof(T)) lds16<T>(Lt + r * TS + q, lt + q);
                    const T v = y[0];
                    D[(b0 + r) * LD + cc] = v;
#pragma unroll
                    for (int l = 1; l < IB; ++l) y[l - 1] = y[l] - v * lt[l];
                }
            }
        }
        __syncthreads();
        {
            const int nr = (rem + 15) / 16;
            if (nr <= 2) diag_rank32<T, 2>(D, LD, b0, w, t);
            else if (MR <= 4 || nr <= 4) diag_rank32<T, (MR < 4 ? MR : 4)>(D, LD, b0, w, t);
            else diag_rank32<T, MR>(D, LD, b0, w, t);
        }
        __syncthreads();
    }
    __syncthreads();
    for (int q = t; q < w; q += DIAG_THREADS) out[q] = dinv[q];
    if (lc < w)
#pragma unroll 4
        for (int r = lr; r < w; r += RPI) A[r * ld + lc] = D[r * LD + lc];
    if constexpr (INV) {
        // the factors' inverses for the strips' tensor-core products, NB x NB row-major
        __syncthreads();
        diag_inverse<T>(D, LD, w, dinv, Ut, t);
        if (lc < w)
#pragma unroll 4
            for (int r = lr; r < w; r += RPI) inv[r * NB + lc] = D[r * LD + lc];
    }
}

template <class T, int NB>
__global__ void __launch_bounds__(DIAG_THREADS, 2) k_diag(const EngItem<T>* __restrict__ items, int p,
                                                          T* __restrict__ scr, long long stride, int* __restrict__ err) {
    const EngItem<T> it = items[blockIdx.x];
    if (p >= it.k) return;
    extern __shared__ __align__(16) unsigned char dsm[];
    diag_body<T, NB>(it, p, scr + (long long)blockIdx.x * stride + (p / NB) * NB, err, dsm);
}

// X[:, b0 + 32 .. w) -= X[:, b0 .. b0 + 32) U[b0 .. b0 + 32, b0 + 32 .. w) on a
// CH-row chunk in shared memory: 16 x 16 threads, thread (ty, tx) owns rows
// ty + 16 i (i < CH / 16) and columns b0 + 32 + tx + 16 j (j < MC).
template <class T, int NB, int MC>
__device__ __forceinline__ void trsm_rank32(T* __restrict__ X, const T* __restrict__ Us, int b0, int w, int t) {
    constexpr int LDX = NB + 1, MR = CH / 16;
    const int ty = t >> 4, tx = t & 15;
    const int base = b0 + IB;
    T acc[MR][MC];
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int j = 0; j < MC; ++j) acc[i][j] = (T)0;
#pragma unroll 2
    for (int l = 0; l < IB; ++l) {
        T a[MR], b[MC];
#pragma unroll
        for (int i = 0; i < MR; ++i) a[i] = X[(ty + 16 * i) * LDX + b0 + l];
#pragma unroll
        for (int j = 0; j < MC; ++j) {
            const int c = base + tx + 16 * j;
            b[j] = c < w ? Us[(b0 + l) * LDX + c] : (T)0;
        }
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MC; ++j) acc[i][j] += a[i] * b[j];
    }
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int j = 0; j < MC; ++j) {
            const int c = base + tx + 16 * j;
            if (c < w) X[(ty + 16 * i) * LDX + c] -= acc[i][j];
        }
}

// Blocked substitution on a chunk of R <= CH rows, X (R x w, in shared memory):
//   X <- X U^{-1}, U upper triangular w x w given by the accessor U(l, c), l <= c.
// L21 chunks use U = U11 (pivot reciprocals from the diagonal task); U12 chunks
// are solved transposed with U = L11^T (unit diagonal).  The chunk and the whole
// triangle are loaded once, up front (a few L2 round trips, several loads in
// flight per thread).  Per 32-column block: substitute within the block (one
// thread per row, the block's triangle rows as 16-byte vector loads), then
// subtract its contribution from all later columns at once (right-looking,
// register tiles of CH/16 x up to 6 per thread).
template <class T, int NB>
__device__ void trsm_body(const EngItem<T>& it, int p, bool colside, int chunk, const T* __restrict__ pinv,
                          unsigned char* tsm_) {
    const int w = min(NB, it.k - p);
    const int n = it.n;
    const long long ld = it.ld;
    const int m0 = p + w;
    const int g0 = m0 + chunk * CH;
    if (g0 >= n) return;
    const int R = min(CH, n - g0);
    constexpr int LDX = NB + 1;
    T* X = reinterpret_cast<T*>(tsm_);        // CH x LDX
    T* Us = X + CH * LDX;                     // NB x LDX: U(l, c)
    T* dv = Us + NB * LDX;                    // NB reciprocal diagonal entries (1 for L11^T)
    const T* A = it.a;
    const int t = threadIdx.x;
    // loads: 16 in flight per thread before their stores, no index divisions
    if (!colside) {
        constexpr int RX = TRSM_THREADS / NB;
        const int xc = t % NB, xr = t / NB;
#pragma unroll 1
        for (int r0 = 0; r0 < CH; r0 += 16 * RX) {
            T v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int r = r0 + xr + u * RX;
                v[u] = (r < R && xc < w) ? __ldcg(A + (long long)(g0 + r) * ld + p + xc) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) X[(r0 + xr + u * RX) * LDX + xc] = v[u];
        }
        // U11: rows of the diagonal block, upper part (the strict lower part is never read)
#pragma unroll 1
        for (int l0 = 0; l0 < w; l0 += 16 * RX) {
            T v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int l = l0 + xr + u * RX;
                v[u] = (l < w && xc < w && xc >= l) ? __ldcg(A + (long long)(p + l) * ld + p + xc) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int l = l0 + xr + u * RX;
                if (l < NB) Us[l * LDX + xc] = v[u];
            }
        }
        if (t < NB) dv[t] = t < w ? __ldcg(pinv + t) : (T)1;
    } else {
        // X[c][k] = M12[k][c]: rows of M12 are contiguous along c
        constexpr int RK = TRSM_THREADS / CH;
        const int xc = t % CH, xk = t / CH;
#pragma unroll 1
        for (int k0 = 0; k0 < NB; k0 += 16 * RK) {
            T v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int k = k0 + xk + u * RK;
                v[u] = (k < w && xc < R) ? __ldcg(A + (long long)(p + k) * ld + g0 + xc) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) X[xc * LDX + k0 + xk + u * RK] = v[u];
        }
        // U(l, c) = L11[c][l] for l < c: rows c of L11, read along l
        constexpr int RC = TRSM_THREADS / NB;
        const int ul = t % NB, uc = t / NB;
#pragma unroll 1
        for (int c0 = 0; c0 < w; c0 += 16 * RC) {
            T v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int c = c0 + uc + u * RC;
                v[u] = (c < w && ul < c) ? __ldcg(A + (long long)(p + c) * ld + p + ul) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int c = c0 + uc + u * RC;
                if (c < NB) Us[ul * LDX + c] = v[u];
            }
        }
        if (t < NB) dv[t] = (T)1;
    }
    T* Sh = dv + NB;                          // IB x TS: Sh[c][l] = U(b0 + c, b0 + c + l)
    __syncthreads();
#pragma unroll 1
    for (int b0 = 0; b0 < w; b0 += IB) {
        const int bw = min(IB, w - b0);
        // the block's triangle, shifted so that its rows load as 16-byte vectors
        for (int q = t; q < IB * IB; q += TRSM_THREADS) {
            const int c = q >> 5, l = q & 31;
            Sh[c * TS + l] = c + l < bw ? Us[(b0 + c) * LDX + b0 + c + l] : (T)0;
        }
        __syncthreads();
        // (1) substitution within the block, one thread per row, the row's 32
        //     entries in registers; the entry finished in step c leaves through y[0]
        if (t < CH) {
            T y[IB];
#pragma unroll
            for (int l = 0; l < IB; ++l) y[l] = X[t * LDX + b0 + l];
#pragma unroll 1
            for (int c = 0; c < bw; ++c) {
                T u[IB];
#pragma unroll
                for (int q = 0; q < IB; q += 16 / (int)sizeof(T)) lds16<T>(Sh + c * TS + q, u + q);
                const T z = y[0] * dv[b0 + c];
                X[t * LDX + b0 + c] = z;
#pragma unroll
                for (int l = 1; l < IB; ++l) y[l - 1] = y[l] - z * u[l];
            }
        }
        __syncthreads();
        // (2) right-looking update of the columns after the block
        const int rem = w - b0 - bw;
        if (rem > 0) {
            const int nc = (rem + 15) / 16;
            if (nc <= 2) trsm_rank32<T, NB, 2>(X, Us, b0, w, t);
            else if (nc <= 4) trsm_rank32<T, NB, (NB >= 96 ? 4 : 2)>(X, Us, b0, w, t);
            else trsm_rank32<T, NB, (NB >= 128 ? 6 : 2)>(X, Us, b0, w, t);
            __syncthreads();
        }
    }
    T* Aw = it.a;
    if (!colside) {
        const int xc = t % NB, xr = t / NB;
        if (xc < w)
#pragma unroll 4
            for (int r = xr; r < R; r += TRSM_THREADS / NB) Aw[(long long)(g0 + r) * ld + p + xc] = X[r * LDX + xc];
    } else {
        const int xc = t % CH, xk = t / CH;
        if (xc < R)
#pragma unroll 4
            for (int k = xk; k < w; k += TRSM_THREADS / CH) Aw[(long long)(p + k) * ld + g0 + xc] = X[xc * LDX + k];
    }
}

template <class T, int NB>
__global__ void __launch_bounds__(TRSM_THREADS, 2) k_trsm(const EngItem<T>* __restrict__ items, int p,
                                                          const T* __restrict__ scr, long long stride, int nch) {
    const EngItem<T> it = items[blockIdx.x];
    if (p >= it.k) return;
    const bool colside = (int)blockIdx.y >= nch;
    const int chunk = colside ? blockIdx.y - nch : blockIdx.y;
    extern __shared__ __align__(16) unsigned char tsm_[];
    trsm_body<T, NB>(it, p, colside, chunk, scr + (long long)blockIdx.x * stride + (p / NB) * NB, tsm_);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <class T, int TILE>
struct UpdLayout {
    static constexpr int VW = 16 / sizeof(T);          // elements per 16-byte copy
    static constexpr int LKP = KC + VW;                // L21 chunk, row-major [r][k]
    static constexpr int UKP = TILE + VW;              // U12 chunk, row-major [k][c]
    static constexpr int BUF = TILE * LKP + KC * UKP;  // elements of one buffer
};

// Load (STORE = false) or store (STORE = true) the thread's 2H x 2H part of a
// TILE x TILE tile at (r0, c0): rows {tr*H + a, TILE/2 + tr*H + a}, columns
// {tc*H + b, TILE/2 + tc*H + b}.  Loads element by element, unconditionally
// (all of them can be in flight at once without extra registers): an
// out-of-range element loads its clamped neighbour and is never stored.  Loads
// go through L2 only (__ldcg).  Stores move runs of H columns
// as one 16-byte access when the tile origin and leading dimension allow it and
// the run is in range (out-of-range elements are not stored).
template <class T, int H, int TILE, bool STORE>
__device__ __forceinline__ void tile_io(T (&acc)[2 * H][2 * H], T* __restrict__ A, long long ld, int r0, int c0,
                                        int n, int tr, int tc, bool vec) {
    static_assert(H * sizeof(T) == 16, "one 16-byte access per run");
#pragma unroll
    for (int a = 0; a < 2 * H; ++a) {
        const int gr = r0 + (a < H ? tr * H + a : TILE / 2 + tr * H + a - H);
        T* row = A + (long long)gr * ld;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int gc = c0 + h * (TILE / 2) + tc * H;
            T* q = row + gc;
            if (STORE && vec && gr < n && gc + H <= n) {
                {
                    if (sizeof(T) == 4) {
                        *reinterpret_cast<float4*>(q) = make_float4((float)acc[a][h * H], (float)acc[a][h * H + 1],
                                                                    (float)acc[a][h * H + 2], (float)acc[a][h * H + 3]);
                    } else {
                        *reinterpret_cast<double2*>(q) = make_double2((double)acc[a][h * H], (double)acc[a][h * H + 1]);
                    }
                }
            } else {
#pragma unroll
                for (int b = 0; b < H; ++b) {
                    if (STORE) {
                        if (gr < n && gc + b < n) q[b] = acc[a][h * H + b];
                    } else {
                        // unconditional load from the clamped position (an out-of-range
                        // accumulator is never stored): no select, no extra registers
                        acc[a][h * H + b] = __ldcg(A + (long long)min(gr, n - 1) * ld + min(gc + b, n - 1));
                    }
                }
            }
        }
    }
}

// M22 -= L21 U12 on one TILE x TILE tile.  Thread (tr, tc) of a 16 x 16 grid owns
// rows {tr*H + a, TILE/2 + tr*H + a} and columns {tc*H + b, TILE/2 + tc*H + b},
// H = TILE/32.  The K-chunks of L21 and U12 are double-buffered in shared memory
// by 16-byte cp.async.cg copies (L2 only: coherent with other CTAs' writes in the
// task kernel), so the next chunk's loads overlap this chunk's FMAs; a trailing
// origin not 16-byte aligned (only a last, narrower panel) takes plain loads.
template <class T, int NB, int TILE>
__device__ void update_body(const EngItem<T>& it, int p, int ti, int tj, unsigned char* usm) {
    const int w = min(NB, it.k - p);
    const int n = it.n;
    const long long ld = it.ld;
    const int m0 = p + w;
    const int r0 = m0 + ti * TILE, c0 = m0 + tj * TILE;
    if (r0 >= n || c0 >= n) return;
    typedef UpdLayout<T, TILE> LY;
    constexpr int H = TILE / 32;              // elements per half per thread (4 in FP32, 2 in FP64)
    constexpr int VW = LY::VW, LKP = LY::LKP, UKP = LY::UKP;
    T* A = it.a;
    const int t = threadIdx.x;
    const int tr = t >> 4, tc = t & 15;
    T acc[2 * H][2 * H];
    T* buf0 = reinterpret_cast<T*>(usm);
    T* buf1 = buf0 + LY::BUF;
    const bool aligned = (m0 % VW) == 0 && (p % VW) == 0 && (ld % VW) == 0 &&
                         (reinterpret_cast<unsigned long long>(A) & 15) == 0;
    auto issue = [&](int k0, T* Lb, T* Ub) {
        const int kw = min(KC, w - k0);
        for (int q = t; q < TILE * (KC / VW); q += UPD_THREADS) {
            const int r = q / (KC / VW), kv = (q - r * (KC / VW)) * VW;
            const int gr = r0 + r;
            int bytes = 0;
            const T* src = A;
            if (gr < n && kv < kw) {
                bytes = min(VW, kw - kv) * (int)sizeof(T);
                src = A + (long long)gr * ld + p + k0 + kv;
            }
            cp_async16(Lb + r * LKP + kv, src, bytes);
        }
        for (int q = t; q < KC * (TILE / VW); q += UPD_THREADS) {
            const int k = q / (TILE / VW), cv = (q - k * (TILE / VW)) * VW;
            const int gc = c0 + cv;
            int bytes = 0;
            const T* src = A;
            if (k < kw && gc < n) {
                bytes = min(VW, n - gc) * (int)sizeof(T);
                src = A + (long long)(p + k0 + k) * ld + gc;
            }
            cp_async16(Ub + k * UKP + cv, src, bytes);
        }
        cp_async_commit();
    };
    auto load_plain = [&](int k0, T* Lb, T* Ub) {
        // PER elements per thread and operand, in batches of 8 loads in flight before their stores
        constexpr int PER = TILE * KC / UPD_THREADS, BT = PER < 8 ? PER : 8;
        const int kw = min(KC, w - k0);
        for (int u0 = 0; u0 < PER; u0 += BT) {
            T v[BT];
#pragma unroll
            for (int u = 0; u < BT; ++u) {
                const int q = t + (u0 + u) * UPD_THREADS, r = q / KC, k = q - r * KC, gr = r0 + r;
                v[u] = (gr < n && k < kw) ? __ldcg(A + (long long)gr * ld + p + k0 + k) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < BT; ++u) {
                const int q = t + (u0 + u) * UPD_THREADS, r = q / KC, k = q - r * KC;
                Lb[r * LKP + k] = v[u];
            }
        }
        for (int u0 = 0; u0 < PER; u0 += BT) {
            T v[BT];
#pragma unroll
            for (int u = 0; u < BT; ++u) {
                const int q = t + (u0 + u) * UPD_THREADS, k = q / TILE, c = q - k * TILE, gc = c0 + c;
                v[u] = (gc < n && k < kw) ? __ldcg(A + (long long)(p + k0 + k) * ld + gc) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < BT; ++u) {
                const int q = t + (u0 + u) * UPD_THREADS, k = q / TILE, c = q - k * TILE;
                Ub[k * UKP + c] = v[u];
            }
        }
    };
    if (aligned) issue(0, buf0, buf0 + TILE * LKP);
    // the accumulators start from the tile of M22 (loads in flight with the first chunk's
    // copies); the K loop subtracts L21 U12 from them and the epilogue only stores
    tile_io<T, H, TILE, false>(acc, A, ld, r0, c0, n, tr, tc, aligned);
    int b = 0;
    for (int k0 = 0; k0 < w; k0 += KC, b ^= 1) {
        T* Lc = b ? buf1 : buf0;
        T* Uc = Lc + TILE * LKP;
        if (aligned) {
            cp_async_wait_all();          // this chunk (issued one iteration earlier)
            __syncthreads();              // ... of every thread; the other buffer is free
            if (k0 + KC < w) {
                T* Ln = b ? buf0 : buf1;
                issue(k0 + KC, Ln, Ln + TILE * LKP);
            }
        } else {
            __syncthreads();
            load_plain(k0, Lc, Uc);
            __syncthreads();
        }
#pragma unroll 4
        for (int k = 0; k < KC; ++k) {
            T lv[2 * H], uv[2 * H];
#pragma unroll
            for (int a = 0; a < H; ++a) {
                lv[a] = Lc[(tr * H + a) * LKP + k];
                lv[H + a] = Lc[(TILE / 2 + tr * H + a) * LKP + k];
            }
            lds16<T>(&Uc[k * UKP + tc * H], uv);
            lds16<T>(&Uc[k * UKP + TILE / 2 + tc * H], uv + H);
#pragma unroll
            for (int a = 0; a < 2 * H; ++a)
#pragma unroll
                for (int bb = 0; bb < 2 * H; ++bb) acc[a][bb] -= lv[a] * uv[bb];
        }
    }
    tile_io<T, H, TILE, true>(acc, A, ld, r0, c0, n, tr, tc, aligned);
}

template <class T, int TILE>
__host__ __device__ constexpr size_t upd_smem() { return 2 * sizeof(T) * UpdLayout<T, TILE>::BUF; }

// M22 -= L21 U12, one TILE x TILE tile per CTA.  part: 0 every tile; 1 the first
// tile row and column (with TILE == NB, the next panel's diagonal block and
// strips); 2 the other tiles.
template <class T, int NB, int TILE>
__global__ void __launch_bounds__(UPD_THREADS) k_update(const EngItem<T>* __restrict__ items, int p, int nt,
                                                        int part) {
    const EngItem<T> it = items[blockIdx.x];
    if (p >= it.k) return;
    const int y = blockIdx.y;
    int ti, tj;
    if (part == 0) {
        ti = y / nt;
        tj = y - ti * nt;
    } else if (part == 1) {
        ti = y < nt ? 0 : y - nt + 1;
        tj = y < nt ? y : 0;
    } else {
        ti = 1 + y / (nt - 1);
        tj = 1 + y % (nt - 1);
    }
    extern __shared__ __align__(16) unsigned char usm[];
    update_body<T, NB, TILE>(it, p, ti, tj, usm);
}

template <class T>
size_t trsm_smem() {
    constexpr int NB = EngCfg<T>::NB;
    return sizeof(T) * ((size_t)CH * (NB + 1) + (size_t)NB * (NB + 1) + NB + IB * TS);
}

template <class T>
size_t diag_smem() {
    constexpr int NB = EngCfg<T>::NB;
    // the LU's shifted triangle copies, then the inverse's 8 blocks of 32 x 33, share one area
    return sizeof(T) * ((size_t)NB * (NB + 1) + NB + std::max(2 * IB * TS, 8 * IB * (IB + 1)));
}

// Shared-memory layout of the tensor-core products: the TF32 hi / lo operand
// parts of one K-chunk of PK = 16 (K-major core matrices: 8 rows x 16 bytes, the
// 8-row groups PK / 4 core matrices apart), then NSTG raw FP32 stages filled by
// cp.async: A as 128 rows x PK (row stride RA floats: conflict-free 16-byte
// reads) and B as PK rows of a 16-byte aligned window of RB columns (the block's
// first column sits delta = 0..3 floats into it).
namespace tcp {
constexpr int PK = 16, NSTG = 4;
constexpr int RA = PK + 4, RB = 132;
constexpr int PART = 128 * PK * 4;                         // bytes of one hi / lo operand part
constexpr int RAW = (128 * RA + PK * RB) * 4;              // bytes of one raw stage
constexpr int SMEM = 4 * PART + NSTG * RAW;
__device__ __forceinline__ int cm(int row, int k) {
    return ((row >> 3) * (PK / 4) + (k >> 2)) * tcx::CORE_BYTES + (row & 7) * 16 + (k & 3) * 4;
}
}  // namespace tcp

// One product on the tensor cores (tcgen05, FP32 accumulation in tensor memory),
// inside the persistent task kernel:
//   C -= A B   (AM = BM = 0: the trailing update M22 -= L21 U12 of one tile), or
//   C  = A B   (the strips: L21 = M21 U11^{-1} with BM = 1, U12 = L11^{-1} M12
//               with AM = 1, in place: every operand load of the block precedes
//               the epilogue's stores),
// on a rows x cols <= 128 x 128 block, K <= 128.  A is rows x K at Ap (element
// (r, k) at Ap[r lda + k]), B is K x cols at Bp (element (k, c) at Bp[k ldb + c]);
// AM = 1 reads A as a unit lower triangle (its strict lower part, 1 on the
// diagonal), BM = 1 reads B as an upper triangle with its diagonal (the packed
// inverses of the diagonal task).  Ap and the rows of A are 16-byte aligned (lda
// a multiple of 4), so is ldb; Bp may sit 0..3 floats past an aligned address.
//
// Pipeline: the operands move global -> shared memory by 16-byte cp.async copies
// (L2 only) in chunks of PK along K, NSTG chunks in flight; per chunk the threads
// split the raw values into TF32 hi / lo parts (KIND = split TF32: hi*hi +
// hi*lo + lo*hi, about FP32 accuracy) or round them to BF16, in the K-major
// core-matrix layout, and one thread issues the MMAs and commits them to the
// mbarrier (bounded wait).  The CTA holds 128 tensor-memory columns (the
// accumulator) and the mbarrier for its whole life; nphase counts the mbarrier
// phases completed so far.  The epilogue reads the accumulator (warp w: rows
// 32 (w % 4) .., columns 64 (w / 4) ..), turns each 32 x 32 block around in shared
// memory and stores (or subtracts) it row by row (coalesced); for C -= A B the
// block's lines were prefetched into L2 when the task started.  Returns false if
// a bounded wait expired (the error is flagged).
template <int KIND, int AM, int BM>
__device__ __noinline__ bool tc_prod_body(const float* __restrict__ Ap, long long lda, const float* __restrict__ Bp,
                                          long long ldb, float* __restrict__ Cp, long long ldc, int rows, int cols,
                                          int K, unsigned char* smem, uint32_t tmem, uint32_t mbar, uint32_t& nphase,
                                          int* __restrict__ err) {
    static_assert(KIND == TC_SPLIT_TF32 || KIND == TC_BF16, "operand kind");
    using namespace tcx;
    using namespace tcp;
    constexpr bool SUB = AM == 0 && BM == 0;
    if (rows <= 0 || cols <= 0 || K <= 0) return true;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    unsigned char* a_hi = smem;
    unsigned char* a_lo = smem + PART;
    unsigned char* b_hi = smem + 2 * PART;
    unsigned char* b_lo = smem + 3 * PART;
    float* raw0 = reinterpret_cast<float*>(smem + 4 * PART);
    if constexpr (SUB) {
        // the block's lines into L2 now: the epilogue reads them after the K loop
        for (int q = t; q < rows * 5; q += UPD_THREADS) {
            const int r = q / 5, l = q - r * 5;
            const int c = min(l * 32, cols - 1);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(Cp + (long long)r * ldc + c));
        }
    }
    const int delta = (int)((reinterpret_cast<unsigned long long>(Bp) >> 2) & 3);
    const float* Bw = Bp - delta;                  // 16-byte aligned window origin
    const int nk = (K + PK - 1) / PK;
    // raw stage of chunk kc: A 128 x 4 groups, B PK x (RB / 4) groups of 16 bytes
    auto issue = [&](int kc) {
        float* ra = raw0 + (kc % NSTG) * (RAW / 4);
        float* rb = ra + 128 * RA;
        const int k0 = kc * PK;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int q = t + u * UPD_THREADS;
            const int row = q & 127, g = q >> 7;
            const int kk = k0 + 4 * g;
            const int bytes = row < rows ? max(0, min(4, K - kk)) * 4 : 0;
            cp_async16(ra + row * RA + 4 * g, bytes ? Ap + (long long)row * lda + kk : Ap, bytes);
        }
        for (int q = t; q < PK * (RB / 4); q += UPD_THREADS) {
            const int kr = q / (RB / 4), g = q - kr * (RB / 4);
            const int c = 4 * g - delta;           // block column of the group's first float
            const int bytes = k0 + kr < K ? max(0, min(4, cols - c)) * 4 : 0;
            cp_async16(rb + kr * RB + 4 * g, bytes ? Bw + (long long)(k0 + kr) * ldb + 4 * g : Bp, bytes);
        }
    };
    // split of chunk kc into the operand parts: thread q -> (row / column q % 128, k group q / 128)
    auto convert = [&](int kc) {
        const float* ra = raw0 + (kc % NSTG) * (RAW / 4);
        const float* rb = ra + 128 * RA;
        const int k0 = kc * PK;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int q = t + u * UPD_THREADS;
            const int row = q & 127, g = q >> 7;
            float a[4], b[4];
            lds16<float>(ra + row * RA + 4 * g, a);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                b[e] = rb[(4 * g + e) * RB + row + delta];
                const int kk = k0 + 4 * g + e;
                if constexpr (AM == 1) a[e] = kk < row ? a[e] : (kk == row && row < rows ? 1.f : 0.f);
                if constexpr (BM == 1) b[e] = kk <= row ? b[e] : 0.f;
            }
            if constexpr (KIND == TC_BF16) {
                // one BF16 operand each, 8 bytes per (row, 4 k): the BF16 layout has 8 k per core-matrix row
                const __nv_bfloat162 a01 = __floats2bfloat162_rn(a[0], a[1]), a23 = __floats2bfloat162_rn(a[2], a[3]);
                const __nv_bfloat162 b01 = __floats2bfloat162_rn(b[0], b[1]), b23 = __floats2bfloat162_rn(b[2], b[3]);
                uint2 pa, pb;
                pa.x = *reinterpret_cast<const uint32_t*>(&a01);
                pa.y = *reinterpret_cast<const uint32_t*>(&a23);
                pb.x = *reinterpret_cast<const uint32_t*>(&b01);
                pb.y = *reinterpret_cast<const uint32_t*>(&b23);
                const int off = ((row >> 3) * (PK / 8) + (g >> 1)) * CORE_BYTES + (row & 7) * 16 + (g & 1) * 8;
                *reinterpret_cast<uint2*>(a_hi + off) = pa;
                *reinterpret_cast<uint2*>(b_hi + off) = pb;
            } else {
                float ah[4], al[4], bh[4], bl[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    ah[e] = tf32_round(a[e]);
                    al[e] = tf32_round(a[e] - ah[e]);
                    bh[e] = tf32_round(b[e]);
                    bl[e] = tf32_round(b[e] - bh[e]);
                }
                const int off = cm(row, 4 * g);
                *reinterpret_cast<float4*>(a_hi + off) = make_float4(ah[0], ah[1], ah[2], ah[3]);
                *reinterpret_cast<float4*>(a_lo + off) = make_float4(al[0], al[1], al[2], al[3]);
                *reinterpret_cast<float4*>(b_hi + off) = make_float4(bh[0], bh[1], bh[2], bh[3]);
                *reinterpret_cast<float4*>(b_lo + off) = make_float4(bl[0], bl[1], bl[2], bl[3]);
            }
        }
    };
    auto mma = [&](int kc) {
        const int kw = min(PK, K - kc * PK);
        if constexpr (KIND == TC_BF16) {
            const uint32_t idesc = instr_desc_bf16(128, 128);
            // 16 BF16 per MMA = two core matrices along K; the 8-row groups PK / 8 core matrices apart
            mma_bf16(tmem, smem_desc(smem_u32(a_hi), CORE_BYTES, (PK / 8) * CORE_BYTES),
                     smem_desc(smem_u32(b_hi), CORE_BYTES, (PK / 8) * CORE_BYTES), idesc, kc > 0 ? 1 : 0);
        } else {
            const uint32_t idesc = instr_desc(128, 128);
            const uint32_t sbo = (PK / 4) * CORE_BYTES;
            for (int kk = 0; kk < (kw + 7) / 8; ++kk) {
                const uint32_t koff = kk * 2 * CORE_BYTES;     // 8 TF32 = two core matrices along K
                const uint64_t ah = smem_desc(smem_u32(a_hi) + koff, CORE_BYTES, sbo);
                const uint64_t al = smem_desc(smem_u32(a_lo) + koff, CORE_BYTES, sbo);
                const uint64_t bh = smem_desc(smem_u32(b_hi) + koff, CORE_BYTES, sbo);
                const uint64_t bl = smem_desc(smem_u32(b_lo) + koff, CORE_BYTES, sbo);
                mma_tf32(tmem, ah, bh, idesc, (kc == 0 && kk == 0) ? 0 : 1);
                mma_tf32(tmem, ah, bl, idesc, 1);
                mma_tf32(tmem, al, bh, idesc, 1);
            }
        }
    };
    bool ok = true;
#pragma unroll 1
    for (int kc = 0; kc < NSTG - 1; ++kc) {
        if (kc < nk) issue(kc);
        cp_async_commit();
    }
#pragma unroll 1
    for (int kc = 0; kc < nk; ++kc) {
        // the stage of chunk kc + NSTG - 1 was converted in the previous iteration
        if (kc + NSTG - 1 < nk) issue(kc + NSTG - 1);
        cp_async_commit();
        asm volatile("cp.async.wait_group %0;\n" ::"n"(NSTG - 1) : "memory");
        if (kc > 0) {
            // the previous chunk's MMAs have read the operand parts
            ok = mbar_wait(mbar, nphase & 1) && ok;
            ++nphase;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        }
        __syncthreads();
        convert(kc);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (t == 0) {
            mma(kc);
            mma_commit(mbar);
        }
    }
    cp_async_wait_all();
    ok = mbar_wait(mbar, nphase & 1) && ok;
    ++nphase;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) {
        if (t == 0) atomicOr(err, ERR_TIMEOUT_TC);
        return false;
    }
    // warp w: accumulator lanes (block rows) 32 (w % 4) .. + 31, columns 64 (w / 4) .. + 63;
    // each 32 x 32 block turns around in shared memory (the raw stages are free
    // now) so that a warp reads and writes 32 consecutive columns of a row
    const int wq = warp & 3, h = warp >> 2;
    float* Tt = raw0 + warp * 32 * 33;
#pragma unroll 1
    for (int cb = 64 * h; cb < 64 * h + 64; cb += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)cb, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) Tt[lane * 33 + j] = v[j];
        __syncwarp();
        const int col = cb + lane;
        const bool cin = col < cols;
        if constexpr (SUB) {
            float c[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int row = 32 * wq + r;
                c[r] = (cin && row < rows) ? __ldcg(Cp + (long long)row * ldc + col) : 0.f;
            }
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int row = 32 * wq + r;
                if (cin && row < rows) Cp[(long long)row * ldc + col] = c[r] - Tt[r * 33 + lane];
            }
        } else {
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int row = 32 * wq + r;
                if (cin && row < rows) Cp[(long long)row * ldc + col] = Tt[r * 33 + lane];
            }
        }
        __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    return true;
}

// ---------------------------------------------------------------------------
// Persistent task kernel.  The host lists the tasks of all panels of all items
// in a topological order (every task after the tasks it depends on, the next
// panel's diagonal block and strips ahead of the bulk of the current update);
// resident CTAs take tasks from an atomic counter, wait for their inputs on
// per-task completion flags and run them.  A CTA only waits for tasks taken
// earlier, which running CTAs hold, so the scheme needs no co-residency.  Every
// wait is bounded: on expiry the kernel flags ERR_TIMEOUT_ENGINE and stops
// waiting (the tasks then finish without their inputs, the error is reported).
// ---------------------------------------------------------------------------
struct EngTask {
    int type;     // 0 diagonal block, 1 L21 row chunk a, 2 U12 column chunk a, 3 tile (a, b)
    int item;
    int panel;
    int a, b;
};
struct EngMeta {
    int off;      // first flag of the item
    int P;        // panels of the item
    int NCH;      // chunk slots per panel
    int NT;       // tile slots per panel and direction
};

__device__ __forceinline__ int flag_diag(const EngMeta& m, int pi) { return m.off + pi; }
__device__ __forceinline__ int flag_row(const EngMeta& m, int pi, int c) { return m.off + m.P + pi * m.NCH + c; }
__device__ __forceinline__ int flag_col(const EngMeta& m, int pi, int c) {
    return m.off + m.P + m.P * m.NCH + pi * m.NCH + c;
}
__device__ __forceinline__ int flag_tile(const EngMeta& m, int pi, int ti, int tj) {
    return m.off + m.P + 2 * m.P * m.NCH + (pi * m.NT + ti) * m.NT + tj;
}

__device__ __forceinline__ int ld_acquire(const int* f) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    return v;
}

constexpr long long ENG_WAIT_LIMIT = 1LL << 24;    // x ~0.1 us sleeps: a few seconds

__device__ void wait_flag(const int* f, int* abort_flag, int* err) {
    long long it = 0;
    while (ld_acquire(f) == 0) {
        if (*(volatile int*)abort_flag) return;
        if (++it > ENG_WAIT_LIMIT) {
            atomicOr(err, ERR_TIMEOUT_ENGINE);
            atomicExch(abort_flag, 1);
            return;
        }
        __nanosleep(100);
    }
}

// wait for every tile of the previous panel overlapping rows [r0, r1) x cols [c0, c1)
// (coordinates relative to the previous panel's trailing origin)
__device__ void wait_prev_tiles(const int* flags, const EngMeta& m, int pi_prev, int ntp, int r0, int r1, int c0,
                                int c1, int tile, int* abort_flag, int* err) {
    const int t0 = r0 / tile, t1 = min((r1 - 1) / tile, ntp - 1);
    const int u0 = c0 / tile, u1 = min((c1 - 1) / tile, ntp - 1);
    for (int a = t0; a <= t1; ++a)
        for (int b = u0; b <= u1; ++b) wait_flag(flags + flag_tile(m, pi_prev, a, b), abort_flag, err);
}

template <class T, int NB, int TILE, int TCK>
__global__ void __launch_bounds__(UPD_THREADS, 2) k_engine_tasks(const EngItem<T>* __restrict__ items,
                                                                 const EngTask* __restrict__ tasks, int ntasks,
                                                                 const EngMeta* __restrict__ meta, int* flags,
                                                                 int* next, int* abort_flag, T* __restrict__ scr,
                                                                 long long stride, T* __restrict__ inv,
                                                                 long long inv_stride, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char esm[];
    __shared__ int s_idx;
    // tensor-core tiles (FP32 only): 128 tensor-memory columns and one mbarrier for
    // the CTA's lifetime
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    uint32_t tmem = 0, nphase = 0;
    // (a separate instantiation: a kernel with tensor-memory allocation gets one CTA per SM)
    constexpr bool tc = TCK != TC_NONE && sizeof(T) == 4;
    // strip chunk: one tensor-core block (128 rows / columns) or CH rows / columns
    constexpr int SCH = tc ? TILE : CH;
    if constexpr (tc) {
        if ((threadIdx.x >> 5) == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(
                tcx::smem_u32(&s_tmem)));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
        }
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tcx::smem_u32(&s_mbar)));
            asm volatile("fence.mbarrier_init.release.cluster;\n");
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        tmem = s_tmem;
    }
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(next, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= ntasks) break;
        const EngTask tk = tasks[idx];
        const EngItem<T> it = items[tk.item];
        const EngMeta m = meta[tk.item];
        const int pi = tk.panel, p = pi * NB;
        const int w = min(NB, it.k - p);
        const int m0 = p + w;
        int own;
        if (threadIdx.x == 0) {
            // inputs: the previous panel's update of the region, and this panel's factors
            const int pp = p - NB;                         // previous panel's trailing origin is p
            const int ntp = (it.n - p + TILE - 1) / TILE;  // its tiles per direction
            if (tk.type == 0) {
                if (pi > 0) wait_prev_tiles(flags, m, pi - 1, ntp, 0, w, 0, w, TILE, abort_flag, err);
            } else if (tk.type == 1 || tk.type == 2) {
                wait_flag(flags + flag_diag(m, pi), abort_flag, err);
                if (pi > 0) {
                    const int g0 = w + tk.a * SCH, g1 = min(it.n - p, g0 + SCH);
                    if (tk.type == 1) wait_prev_tiles(flags, m, pi - 1, ntp, g0, g1, 0, w, TILE, abort_flag, err);
                    else wait_prev_tiles(flags, m, pi - 1, ntp, 0, w, g0, g1, TILE, abort_flag, err);
                }
            } else {
                const int nch = (it.n - m0 + SCH - 1) / SCH;
                const int ca = (tk.a * TILE) / SCH, cb = min(nch - 1, ((tk.a + 1) * TILE - 1) / SCH);
                for (int c = ca; c <= cb; ++c) wait_flag(flags + flag_row(m, pi, c), abort_flag, err);
                const int da = (tk.b * TILE) / SCH, db = min(nch - 1, ((tk.b + 1) * TILE - 1) / SCH);
                for (int c = da; c <= db; ++c) wait_flag(flags + flag_col(m, pi, c), abort_flag, err);
                if (pi > 0) {
                    const int r0 = w + tk.a * TILE, c0 = w + tk.b * TILE;
                    wait_prev_tiles(flags, m, pi - 1, ntp, r0, min(it.n - p, r0 + TILE), c0,
                                    min(it.n - p, c0 + TILE), TILE, abort_flag, err);
                }
            }
            (void)pp;
        }
        __syncthreads();
        T* pv = scr + (long long)tk.item * stride + (long long)pi * NB;
        if (tk.type == 0) {
            if constexpr (tc) diag_body<T, NB, true>(it, p, pv, err, esm, inv + tk.item * inv_stride + (long long)pi * NB * NB);
            else diag_body<T, NB>(it, p, pv, err, esm);
            own = flag_diag(m, pi);
        } else if (tk.type == 1 || tk.type == 2) {
            if constexpr (tc) {
                // L21 = M21 U11^{-1} (128 rows) or U12 = L11^{-1} M12 (128 columns) in place, split TF32
                float* A = reinterpret_cast<float*>(it.a);
                const float* Iv = reinterpret_cast<const float*>(inv) + tk.item * inv_stride + (long long)pi * NB * NB;
                const long long ld = it.ld;
                const int g0 = m0 + tk.a * SCH, len = min(SCH, it.n - g0);
                bool ok = true;
                if (tk.type == 1)
                    ok = tc_prod_body<TC_SPLIT_TF32, 0, 1>(A + (long long)g0 * ld + p, ld, Iv, NB,
                                                          A + (long long)g0 * ld + p, ld, len, w, w, esm, tmem,
                                                          tcx::smem_u32(&s_mbar), nphase, err);
                else
                    ok = tc_prod_body<TC_SPLIT_TF32, 1, 0>(Iv, NB, A + (long long)p * ld + g0, ld,
                                                          A + (long long)p * ld + g0, ld, w, len, w, esm, tmem,
                                                          tcx::smem_u32(&s_mbar), nphase, err);
                if (!ok && threadIdx.x == 0) atomicExch(abort_flag, 1);
            } else {
                trsm_body<T, NB>(it, p, tk.type == 2, tk.a, pv, esm);
            }
            own = tk.type == 1 ? flag_row(m, pi, tk.a) : flag_col(m, pi, tk.a);
        } else {
            if constexpr (tc) {
                float* A = reinterpret_cast<float*>(it.a);
                const long long ld = it.ld;
                const int r0 = m0 + tk.a * TILE, c0 = m0 + tk.b * TILE;
                if (r0 < it.n && c0 < it.n &&
                    !tc_prod_body<(TCK == TC_BF16 ? TC_BF16 : TC_SPLIT_TF32), 0, 0>(
                        A + (long long)r0 * ld + p, ld, A + (long long)p * ld + c0, ld, A + (long long)r0 * ld + c0,
                        ld, min(TILE, it.n - r0), min(TILE, it.n - c0), w, esm, tmem, tcx::smem_u32(&s_mbar), nphase,
                        err) &&
                    threadIdx.x == 0)
                    atomicExch(abort_flag, 1);
            } else {
                update_body<T, NB, TILE>(it, p, tk.a, tk.b, esm);
            }
            own = flag_tile(m, pi, tk.a, tk.b);
        }
        __threadfence();        // every thread's results, before the completion flag
        __syncthreads();
        if (threadIdx.x == 0)
            asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(flags + own), "r"(1) : "memory");
    }
    if constexpr (tc) {
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if ((threadIdx.x >> 5) == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem));
    }
}

template <class T>
size_t task_smem(bool tc) {
    constexpr int TILE = EngCfg<T>::TILE;
    // tensor-core instantiation: the diagonal body and the products' four operand
    // parts (the strips run as products too)
    if (tc) return std::max(diag_smem<T>(), (size_t)tcp::SMEM);
    return std::max(std::max(diag_smem<T>(), trsm_smem<T>()), upd_smem<T, TILE>());
}

}  // namespace

long long engine_scratch_elems(int count, bool dbl, int maxk) {
    const int nb = dbl ? EngCfg<double>::NB : EngCfg<float>::NB;
    const long long np = std::max(1, (maxk + nb - 1) / nb);
    return (long long)count * nb * np;
}

namespace {
// Task list of the persistent kernel (host), in the order described above.
template <class T>
static void build_tasks(const int* hn, const int* hk, int count, int CH, std::vector<EngTask>& tasks,
                        std::vector<EngMeta>& meta, int& nflags) {
    constexpr int NB = EngCfg<T>::NB, TILE = EngCfg<T>::TILE;
    meta.resize(count);
    nflags = 0;
    int Pmax = 0;
    for (int i = 0; i < count; ++i) {
        EngMeta& m = meta[i];
        m.P = hk[i] > 0 ? (hk[i] + NB - 1) / NB : 0;
        m.NCH = std::max(1, (hn[i] + CH - 1) / CH);
        m.NT = std::max(1, (hn[i] + TILE - 1) / TILE);
        m.off = nflags;
        nflags += m.P * (1 + 2 * m.NCH + m.NT * m.NT);
        Pmax = std::max(Pmax, m.P);
    }
    auto geom = [&](int i, int pi, int& nch, int& nt) {
        const int p = pi * NB, w = std::min(NB, hk[i] - p), mrem = hn[i] - p - w;
        nch = (mrem + CH - 1) / CH;
        nt = (mrem + TILE - 1) / TILE;
    };
    const int lo = 0, hi = count;
    auto add_diag = [&](int pi) {
        for (int i = lo; i < hi; ++i)
            if (pi < meta[i].P) tasks.push_back(EngTask{0, i, pi, 0, 0});
    };
    auto add_rc = [&](int pi) {
        for (int i = lo; i < hi; ++i) {
            if (pi >= meta[i].P) continue;
            int nch, nt;
            geom(i, pi, nch, nt);
            for (int c = 0; c < nch; ++c) {
                tasks.push_back(EngTask{1, i, pi, c, 0});
                tasks.push_back(EngTask{2, i, pi, c, 0});
            }
        }
    };
    auto add_tiles = [&](int pi, bool first) {
        for (int i = lo; i < hi; ++i) {
            if (pi >= meta[i].P) continue;
            int nch, nt;
            geom(i, pi, nch, nt);
            for (int a = 0; a < nt; ++a)
                for (int b = 0; b < nt; ++b)
                    if ((a == 0 || b == 0) == first) tasks.push_back(EngTask{3, i, pi, a, b});
        }
    };
    // D(0) RC(0) Uf(0) | D(1) Ur(0) RC(1) Uf(1) | D(2) Ur(1) ...: the next diagonal
    // block starts as soon as its tile is updated, the bulk of the current update
    // fills the GPU meanwhile, and the strips that need the new factors come after.
    // (All items per panel: the diagonal tasks' chain is hidden behind the other
    // items' tiles; a task order by groups of items that fit in L2 made the strips
    // wait for their diagonal blocks.)
    if (Pmax == 0) return;
    add_diag(0);
    add_rc(0);
    add_tiles(0, true);
    for (int pi = 0; pi < Pmax; ++pi) {
        if (pi + 1 < Pmax) add_diag(pi + 1);
        add_tiles(pi, false);
        if (pi + 1 < Pmax) {
            add_rc(pi + 1);
            add_tiles(pi + 1, true);
        }
    }
}
}  // namespace

// Eliminate the leading k_i unknowns of every item.  Default: one persistent
// task kernel per call (update tiles on the tensor cores when tc is set and T is
// float).  With the kernel timer on, the per-panel launches k_diag, k_trsm,
// k_update (k_tc_update) run instead, so that every launch of a kernel class can
// be bracketed by events.
template <class T>
int engine_run(const EngItem<T>* items_dev, int count, int maxn, int maxk, T* dscr, int* err,
               cudaStream_t st, const int* hn, const int* hk, int tc) {
    constexpr int NB = EngCfg<T>::NB, TILE = EngCfg<T>::TILE;
    static_assert(NB == TILE, "the task dependencies assume one tile per panel");
    if (count <= 0 || maxk <= 0) return BDDC_OK;
    const long long stride = (long long)NB * std::max(1, (maxk + NB - 1) / NB);
    const bool timed = ktimer_on(KT_ENGINE_UPDATE) || ktimer_on(KT_ENGINE_PANEL);
    const int tck = sizeof(T) == 4 ? tc : TC_NONE;
    const bool use_tc = tck != TC_NONE;
    // (the BF16 tiles exist only in the task kernel: it runs even with the timer on)
    if ((!timed || tck == TC_BF16) && hn && hk) {
        std::vector<EngTask> tasks;
        std::vector<EngMeta> meta;
        int nflags = 0;
        // tensor-core strips are 128-row / -column products (one flag per tile row / column)
        build_tasks<T>(hn, hk, count, use_tc ? TILE : CH, tasks, meta, nflags);
        if (tasks.empty()) return BDDC_OK;
        // one allocation for the task list, the item table, the flags and (tensor
        // cores) the inverses of the diagonal blocks' factors (NB x NB per item and
        // panel), freed by the stream-ordered allocator after the launch
        const size_t tb = tasks.size() * sizeof(EngTask), mb = meta.size() * sizeof(EngMeta);
        const size_t fb = sizeof(int) * ((size_t)nflags + 2);
        const size_t o1 = (tb + 255) & ~size_t(255), o2 = o1 + ((mb + 255) & ~size_t(255));
        const size_t o3 = o2 + ((fb + 255) & ~size_t(255));
        const long long inv_stride = use_tc ? (long long)NB * stride : 0;
        const size_t ib = sizeof(T) * (size_t)inv_stride * (size_t)count;
        std::vector<unsigned char> host(o2);
        memcpy(host.data(), tasks.data(), tb);
        memcpy(host.data() + o1, meta.data(), mb);
        unsigned char* dev = nullptr;
        BDDC_CUDA_TRY(cudaMallocAsync((void**)&dev, o3 + ib, st));
        BDDC_TRY(staged_upload(dev, host.data(), o2, st));
        int* flags = reinterpret_cast<int*>(dev + o2);
        T* inv = use_tc ? reinterpret_cast<T*>(dev + o3) : nullptr;
        BDDC_CUDA_TRY(cudaMemsetAsync(flags, 0, fb, st));
        const size_t sm = task_smem<T>(use_tc);
        auto kern = !use_tc ? k_engine_tasks<T, NB, TILE, TC_NONE>
                    : (tck == TC_BF16 ? k_engine_tasks<T, NB, TILE, TC_BF16> : k_engine_tasks<T, NB, TILE, TC_SPLIT_TF32>);
        BDDC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        // all of the SM's configurable memory as shared memory: two CTAs of this size per SM
        BDDC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        int dev_id = 0, nsm = 0, occ = 0;
        BDDC_CUDA_TRY(cudaGetDevice(&dev_id));
        BDDC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev_id));
        // residency from the CUDA-core instantiation (same registers and shared memory):
        // the occupancy calculator reports one CTA per SM for a kernel that allocates
        // tensor memory, but two CTAs of 128 columns each (of 512) run side by side
        auto kcc = k_engine_tasks<T, NB, TILE, TC_NONE>;
        BDDC_CUDA_TRY(cudaFuncSetAttribute(kcc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        BDDC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kcc, UPD_THREADS, sm));
        const int grid = (int)std::min<long long>((long long)nsm * std::max(occ, 1), (long long)tasks.size());
        double fl = 0.0, by = 0.0;
        if (ktimer_on(KT_ENGINE_TASKS))
            for (int i = 0; i < count; ++i)
                for (int p = 0; p < hk[i]; p += NB) {
                    // trailing update 2 m^2 w, substitutions 2 w^2 m, diagonal block (2/3) w^3;
                    // bytes: the trailing matrix read and written once per panel
                    const double w = std::min(NB, hk[i] - p), m = hn[i] - p - w;
                    fl += 2.0 * m * m * w + 2.0 * w * w * m + 2.0 * w * w * w / 3.0;
                    by += sizeof(T) * (2.0 * m * m + 4.0 * m * w + 2.0 * w * w);
                }
        ktimer_begin(KT_ENGINE_TASKS, st);
        kern<<<grid, UPD_THREADS, sm, st>>>(items_dev, reinterpret_cast<const EngTask*>(dev), (int)tasks.size(),
                                             reinterpret_cast<const EngMeta*>(dev + o1), flags, flags + nflags,
                                             flags + nflags + 1, dscr, stride, inv, inv_stride, err);
        ktimer_end(KT_ENGINE_TASKS, st, fl, by);
        bddc_note_launches(1);
        BDDC_CUDA_TRY(cudaGetLastError());
        BDDC_CUDA_TRY(cudaFreeAsync(dev, st));
        return BDDC_OK;
    }
    const size_t dsm = diag_smem<T>();
    const size_t tsm = trsm_smem<T>();
    const size_t usm_b = upd_smem<T, TILE>();
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_diag<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_trsm<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_update<T, NB, TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usm_b));
    auto panel = [&](int p, cudaStream_t s) -> int {
        const int nch = (std::max(maxn - p, 1) + CH - 1) / CH;
        k_diag<T, NB><<<count, DIAG_THREADS, dsm, s>>>(items_dev, p, dscr, stride, err);
        k_trsm<T, NB><<<dim3(count, 2 * nch), TRSM_THREADS, tsm, s>>>(items_dev, p, dscr, stride, nch);
        bddc_note_launches(2);
        return BDDC_OK;
    };
    for (int p = 0; p < maxk; p += NB) {
        const int mrem = std::max(maxn - p, 1);          // bound of the trailing size
        const int nt = (mrem + TILE - 1) / TILE;
        // algorithmic work of this panel: trailing update 2 m^2 w; diagonal block
        // (2/3) w^3 and substitutions 2 w^2 m
        double fu = 0.0, fp = 0.0, bu = 0.0;
        if (hn && timed)
            for (int i = 0; i < count; ++i) {
                if (p >= hk[i]) continue;
                double w = std::min(NB, hk[i] - p), m = hn[i] - p - w;
                fu += 2.0 * m * m * w;
                fp += 2.0 * w * w * w / 3.0 + 2.0 * w * w * m;
                bu += sizeof(T) * (2.0 * m * m + 2.0 * m * w);   // read + write M22, read L21, U12
            }
        ktimer_begin(KT_ENGINE_PANEL, st);
        BDDC_TRY(panel(p, st));
        ktimer_end(KT_ENGINE_PANEL, st, fp, 0.0);
        ktimer_begin(KT_ENGINE_UPDATE, st);
        if constexpr (sizeof(T) == 4) {
            if (use_tc) {
                BDDC_TRY(tc_update_run(reinterpret_cast<const EngItem<float>*>(items_dev), count, maxn, p, NB,
                                       err, st));
            } else {
                k_update<T, NB, TILE><<<dim3(count, nt * nt), UPD_THREADS, usm_b, st>>>(items_dev, p, nt, 0);
                bddc_note_launches(1);
            }
        } else {
            k_update<T, NB, TILE><<<dim3(count, nt * nt), UPD_THREADS, usm_b, st>>>(items_dev, p, nt, 0);
            bddc_note_launches(1);
        }
        ktimer_end(KT_ENGINE_UPDATE, st, fu, bu);
    }
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

template int engine_run<double>(const EngItem<double>*, int, int, int, double*, int*, cudaStream_t,
                                const int*, const int*, int);
template int engine_run<float>(const EngItem<float>*, int, int, int, float*, int*, cudaStream_t,
                               const int*, const int*, int);
