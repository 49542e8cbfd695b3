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
// Per panel three launches, each batched over all items:
//   k_diag    one CTA per item factors the NB x NB diagonal block in shared
//             memory, 32 columns at a time (the 32 pivot steps restricted to
//             the column panel and the row strip, one barrier each, then a
//             rank-32 update of the rest), writes L11\U11 back and the pivot
//             reciprocals to a scratch;
//   k_trsm    L21 = M21 U11^{-1} in 64-row chunks and U12 = L11^{-1} M12 in
//             64-column chunks (the latter solved transposed, so both run the
//             same blocked substitution: per 32-column block subtract the
//             solved blocks, then substitute within the block);
//   k_update  M22 -= L21 U12 in TILE x TILE tiles, K staged through shared
//             memory in chunks of 32, register-blocked (8 x 8 per thread in
//             FP32, 4 x 4 in FP64).  The FP32 update can run on the tensor
//             cores instead (tc_update.cu).
// A wider panel divides the passes over the trailing matrices (the HBM
// traffic of the update) by the width: NB = 128 does a quarter of the
// passes of a 32-wide panel.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "bddc_internal.h"

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

// Per-item scratch: the reciprocal pivots of every panel (NB per panel, so that
// a panel's pivots stay valid while the next panel is factored in the task
// kernel); `stride` elements per item.

// Solve x U = b within one 32-column block for NR vectors held by a group of 8
// lanes (lane cg of the group owns entries cg, cg+8, cg+16, cg+24 of every
// vector in acc[.][0..3]).  U(c, c') = U[c*s1 + c'*s2] for c < c' < bw; its
// diagonal enters through the reciprocals d (nullptr: unit diagonal).  Column
// c is final once the update from columns < c is in: its owner scales it and
// broadcasts it by shuffle, and every lane updates its later columns, so the
// dependent chain is 32 short steps instead of a 32 x 32 triangle per thread.
// All 32 lanes of the warp must call it (the shuffles are warp-wide).
template <class T, int NR>
__device__ __forceinline__ void subst8(T (&acc)[NR][4], const T* __restrict__ U, int s1, int s2,
                                       const T* __restrict__ d, int bw, int cg) {
#pragma unroll
    for (int ec = 0; ec < 4; ++ec) {
        for (int gc = 0; gc < 8; ++gc) {
            const int c = gc + 8 * ec;
            if (c >= bw) break;
            const T dc = d ? d[c] : (T)1;
            T x[NR];
#pragma unroll
            for (int a = 0; a < NR; ++a) {
                x[a] = __shfl_sync(0xffffffffu, acc[a][ec] * dc, gc, 8);
                if (cg == gc) acc[a][ec] = x[a];
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int cp = cg + 8 * e;
                if (cp > c && cp < bw) {
                    const T u = U[c * s1 + cp * s2];
#pragma unroll
                    for (int a = 0; a < NR; ++a) acc[a][e] -= x[a] * u;
                }
            }
        }
    }
}

// LU of the w x w diagonal block in shared memory, 32 columns at a time.  The
// code is kept compact (loops over shared memory, no long unrolled chains): it
// runs once per launch, so straight-line code would be fetched from beyond the
// instruction cache for every instruction.
// (global loads of matrix data go through L2, __ldcg: in the persistent task
// kernel other CTAs write it during the launch)
template <class T, int NB>
__device__ void diag_body(const EngItem<T>& it, int p, T* __restrict__ out, int* __restrict__ err,
                          unsigned char* dsm) {
    const int w = min(NB, it.k - p);
    const long long ld = it.ld;
    T* A = it.a + (long long)p * ld + p;
    constexpr int LD = NB + 1;
    T* D = reinterpret_cast<T*>(dsm);        // NB x LD: L\U of the diagonal block
    T* dinv = D + NB * LD;                    // NB reciprocal pivots
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int q = t; q < w * w; q += DIAG_THREADS) {
        const int r = q / w, c = q - r * w;
        D[r * LD + c] = __ldcg(A + r * ld + c);
    }
    __syncthreads();
    for (int b0 = 0; b0 < w; b0 += IB) {
        const int bw = min(IB, w - b0);
        // (a) the block's 32 pivots, all threads, one barrier per pivot: step jj
        //     updates the column panel (rows below jj, columns jj+1 .. b0+bw-1) and
        //     the row strip (rows jj+1 .. b0+bw-1, columns b0+bw .. w-1) with the
        //     unscaled column jj; the column is scaled after the barrier (no later
        //     step of the block reads it).
        const int rem = w - b0 - bw;
        {
            const int ty = t >> 5;                 // 16 row lanes
            constexpr int NRL = DIAG_THREADS / 32;
            for (int jj = b0; jj < b0 + bw; ++jj) {
                T piv = D[jj * LD + jj];
                const bool bad = bad_pivot(piv);
                if (bad) piv = (T)1;
                const T ri = (T)1 / piv;
                const int cend = b0 + bw;
                // column panel: c = jj + 1 + lane (< cend), rows jj+1+ty, stepping NRL
                {
                    const int c = jj + 1 + lane;
                    if (c < cend) {
                        const T u = D[jj * LD + c] * ri;
                        for (int r = jj + 1 + ty; r < w; r += NRL) D[r * LD + c] -= D[r * LD + jj] * u;
                    }
                }
                // row strip: rows jj+1 .. cend-1, columns cend .. w-1
                for (int r = jj + 1 + ty; r < cend; r += NRL) {
                    const T l = D[r * LD + jj] * ri;
                    for (int c = cend + lane; c < w; c += 32) D[r * LD + c] -= l * D[jj * LD + c];
                }
                __syncthreads();
                for (int r = jj + 1 + t; r < w; r += DIAG_THREADS) D[r * LD + jj] *= ri;
                if (t == 0) {
                    if (bad) {
                        D[jj * LD + jj] = piv;
                        atomicOr(err, ERR_PIVOT);
                    }
                    dinv[jj] = ri;
                }
            }
        }
        __syncthreads();
        // (c) rank-bw update of the remaining rem x rem block; lane = column within a
        //     32-column group, four rows per thread
        if (rem > 0) {
            const int ncg = (rem + 31) / 32, nrg = (rem + 3) / 4;
            const int base = b0 + bw;
            for (int job = wid; job < ncg * nrg; job += DIAG_THREADS / 32) {
                const int cg = job % ncg, rg = job / ncg;
                const int c = base + cg * 32 + lane;
                const int r0 = base + rg * 4;
                if (c < w) {
                    T acc[4] = {0, 0, 0, 0};
                    for (int l = 0; l < bw; ++l) {
                        const T u = D[(b0 + l) * LD + c];
#pragma unroll
                        for (int a = 0; a < 4; ++a)
                            if (r0 + a < w) acc[a] += D[(r0 + a) * LD + b0 + l] * u;
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
                        if (r0 + a < w) D[(r0 + a) * LD + c] -= acc[a];
                }
            }
        }
        __syncthreads();
    }
    for (int q = t; q < w; q += DIAG_THREADS) out[q] = dinv[q];
    for (int q = t; q < w * w; q += DIAG_THREADS) {
        const int r = q / w, c = q - r * w;
        A[r * ld + c] = D[r * LD + c];
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

// Blocked substitution on a chunk of R <= CH rows, X (R x w, in shared memory):
//   X <- X U^{-1}, U upper triangular w x w given by the accessor U(l, c), l <= c.
// L21 chunks use U = U11 (pivot reciprocals from k_diag); U12 chunks are solved
// transposed with U = L11^T (unit diagonal).  Per 32-column block: subtract the
// solved blocks (register-blocked, 2 rows x 4 columns per thread), then
// substitute within the block (subst8: 8 lanes per row pair).
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
    T* Us = X + CH * LDX;                     // NB x 33: U(l, b0 + c) for l < b0 + 32
    T* dv = Us + NB * (IB + 1);               // 32 reciprocal diagonal entries of the block
    const T* A = it.a;
    const int t = threadIdx.x;
    if (!colside) {
        for (int q = t; q < CH * w; q += TRSM_THREADS) {
            const int r = q / w, c = q - r * w;
            X[r * LDX + c] = r < R ? __ldcg(A + (long long)(g0 + r) * ld + p + c) : (T)0;
        }
    } else {
        // X[c][k] = M12[k][c]: rows of M12 are contiguous along c
        for (int q = t; q < CH * w; q += TRSM_THREADS) {
            const int k = q / CH, c = q - k * CH;
            X[c * LDX + k] = c < R ? __ldcg(A + (long long)(p + k) * ld + g0 + c) : (T)0;
        }
    }
    const int rg = t >> 3, cg = t & 7;        // rows 2rg, 2rg+1; columns cg + 8e
    for (int b0 = 0; b0 < w; b0 += IB) {
        const int bw = min(IB, w - b0);
        const int nl = b0 + bw;
        if (!colside) {
            for (int q = t; q < nl * IB; q += TRSM_THREADS) {
                const int l = q / IB, c = q - l * IB;
                Us[l * (IB + 1) + c] = c < bw ? __ldcg(A + (long long)(p + l) * ld + p + b0 + c) : (T)0;
            }
            if (t < IB) dv[t] = t < bw ? __ldcg(pinv + b0 + t) : (T)1;
        } else {
            // U(l, b0 + c) = L11[b0 + c][l]: rows of L11, read along l
            for (int q = t; q < nl * IB; q += TRSM_THREADS) {
                const int c = q / nl, l = q - c * nl;
                Us[l * (IB + 1) + c] = c < bw ? __ldcg(A + (long long)(p + b0 + c) * ld + p + l) : (T)0;
            }
            if (t < IB) dv[t] = (T)1;
        }
        __syncthreads();
        T acc[2][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[a][e] = X[(2 * rg + a) * LDX + b0 + cg + 8 * e];
        for (int l = 0; l < b0; ++l) {
            const T x0 = X[(2 * rg) * LDX + l], x1 = X[(2 * rg + 1) * LDX + l];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const T u = Us[l * (IB + 1) + cg + 8 * e];
                acc[0][e] -= x0 * u;
                acc[1][e] -= x1 * u;
            }
        }
        subst8<T, 2>(acc, Us + b0 * (IB + 1), IB + 1, 1, dv, bw, cg);
        __syncthreads();        // every read of this block's X and of Us is done
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int e = 0; e < 4; ++e) X[(2 * rg + a) * LDX + b0 + cg + 8 * e] = acc[a][e];
        __syncthreads();
    }
    T* Aw = it.a;
    if (!colside) {
        for (int q = t; q < R * w; q += TRSM_THREADS) {
            const int r = q / w, c = q - r * w;
            Aw[(long long)(g0 + r) * ld + p + c] = X[r * LDX + c];
        }
    } else {
        for (int q = t; q < R * w; q += TRSM_THREADS) {
            const int k = q / R, c = q - k * R;
            Aw[(long long)(p + k) * ld + g0 + c] = X[c * LDX + k];
        }
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
#pragma unroll
    for (int a = 0; a < 2 * H; ++a)
#pragma unroll
        for (int b = 0; b < 2 * H; ++b) acc[a][b] = (T)0;
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
        const int kw = min(KC, w - k0);
        for (int q = t; q < TILE * KC; q += UPD_THREADS) {
            const int r = q / KC, k = q - r * KC;
            const int gr = r0 + r;
            Lb[r * LKP + k] = (gr < n && k < kw) ? __ldcg(A + (long long)gr * ld + p + k0 + k) : (T)0;
        }
        for (int q = t; q < TILE * KC; q += UPD_THREADS) {
            const int k = q / TILE, c = q - k * TILE;
            const int gc = c0 + c;
            Ub[k * UKP + c] = (gc < n && k < kw) ? __ldcg(A + (long long)(p + k0 + k) * ld + gc) : (T)0;
        }
    };
    if (aligned) issue(0, buf0, buf0 + TILE * LKP);
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
                for (int bb = 0; bb < 2 * H; ++bb) acc[a][bb] += lv[a] * uv[bb];
        }
    }
#pragma unroll
    for (int a = 0; a < 2 * H; ++a) {
        const int gr = r0 + (a < H ? tr * H + a : TILE / 2 + tr * H + a - H);
        if (gr >= n) continue;
        T* row = A + (long long)gr * ld;
#pragma unroll
        for (int bb = 0; bb < 2 * H; ++bb) {
            const int gc = c0 + (bb < H ? tc * H + bb : TILE / 2 + tc * H + bb - H);
            if (gc < n) row[gc] = __ldcg(row + gc) - acc[a][bb];
        }
    }
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
    return sizeof(T) * ((size_t)CH * (NB + 1) + (size_t)NB * (IB + 1) + IB);
}

template <class T>
size_t diag_smem() {
    constexpr int NB = EngCfg<T>::NB;
    return sizeof(T) * ((size_t)NB * (NB + 1) + NB);
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

template <class T, int NB, int TILE>
__global__ void __launch_bounds__(UPD_THREADS, 2) k_engine_tasks(const EngItem<T>* __restrict__ items,
                                                                 const EngTask* __restrict__ tasks, int ntasks,
                                                                 const EngMeta* __restrict__ meta, int* flags,
                                                                 int* next, int* abort_flag, T* __restrict__ scr,
                                                                 long long stride, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char esm[];
    __shared__ int s_idx;
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
                    const int g0 = w + tk.a * CH, g1 = min(it.n - p, g0 + CH);
                    if (tk.type == 1) wait_prev_tiles(flags, m, pi - 1, ntp, g0, g1, 0, w, TILE, abort_flag, err);
                    else wait_prev_tiles(flags, m, pi - 1, ntp, 0, w, g0, g1, TILE, abort_flag, err);
                }
            } else {
                const int nch = (it.n - m0 + CH - 1) / CH;
                const int ca = (tk.a * TILE) / CH, cb = min(nch - 1, ((tk.a + 1) * TILE - 1) / CH);
                for (int c = ca; c <= cb; ++c) wait_flag(flags + flag_row(m, pi, c), abort_flag, err);
                const int da = (tk.b * TILE) / CH, db = min(nch - 1, ((tk.b + 1) * TILE - 1) / CH);
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
            diag_body<T, NB>(it, p, pv, err, esm);
            own = flag_diag(m, pi);
        } else if (tk.type == 1 || tk.type == 2) {
            trsm_body<T, NB>(it, p, tk.type == 2, tk.a, pv, esm);
            own = tk.type == 1 ? flag_row(m, pi, tk.a) : flag_col(m, pi, tk.a);
        } else {
            update_body<T, NB, TILE>(it, p, tk.a, tk.b, esm);
            own = flag_tile(m, pi, tk.a, tk.b);
        }
        __threadfence();        // every thread's results, before the completion flag
        __syncthreads();
        if (threadIdx.x == 0)
            asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(flags + own), "r"(1) : "memory");
    }
}

template <class T>
size_t task_smem() {
    constexpr int TILE = EngCfg<T>::TILE;
    return std::max(std::max(diag_smem<T>(), trsm_smem<T>()), upd_smem<T, TILE>());
}

}  // namespace

long long engine_scratch_elems(int count, bool dbl, int maxk) {
    const int nb = dbl ? EngCfg<double>::NB : EngCfg<float>::NB;
    const long long np = std::max(1, (maxk + nb - 1) / nb);
    return (long long)count * nb * np;
}

namespace {
// Side stream and events of the look-ahead (one set per host thread).
struct LookAhead {
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int dev = -1;
    int init() {
        int d = 0;
        BDDC_CUDA_TRY(cudaGetDevice(&d));
        if (side && d == dev) return BDDC_OK;
        dev = d;                              // (a stream of another device is left alive)
        int lo = 0, hi = 0;
        BDDC_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        // highest priority: the next panel's CTAs take SM slots as update CTAs retire
        BDDC_CUDA_TRY(cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, hi));
        BDDC_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        BDDC_CUDA_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        return BDDC_OK;
    }
};
thread_local LookAhead g_la;

// Task list of the persistent kernel (host), in the order described above.
template <class T>
static void build_tasks(const int* hn, const int* hk, int count, std::vector<EngTask>& tasks,
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
    auto add_diag = [&](int pi) {
        for (int i = 0; i < count; ++i)
            if (pi < meta[i].P) tasks.push_back(EngTask{0, i, pi, 0, 0});
    };
    auto add_rc = [&](int pi) {
        for (int i = 0; i < count; ++i) {
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
        for (int i = 0; i < count; ++i) {
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
    // fills the GPU meanwhile, and the strips that need the new factors come after
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
// task kernel per call.  With the kernel timer on (or the tensor-core update)
// the per-panel launches k_diag, k_trsm, k_update run instead, so that every
// launch of a kernel class can be bracketed by events.
template <class T>
int engine_run(const EngItem<T>* items_dev, int count, int maxn, int maxk, T* dscr, int* err,
               cudaStream_t st, const int* hn, const int* hk, bool tc) {
    constexpr int NB = EngCfg<T>::NB, TILE = EngCfg<T>::TILE;
    static_assert(NB == TILE, "the task dependencies assume one tile per panel");
    if (count <= 0 || maxk <= 0) return BDDC_OK;
    const long long stride = (long long)NB * std::max(1, (maxk + NB - 1) / NB);
    const bool timed = ktimer_on(KT_ENGINE_UPDATE) || ktimer_on(KT_ENGINE_PANEL);
    const bool use_tc = tc && sizeof(T) == 4;
    if (!timed && !use_tc && hn && hk) {
        std::vector<EngTask> tasks;
        std::vector<EngMeta> meta;
        int nflags = 0;
        build_tasks<T>(hn, hk, count, tasks, meta, nflags);
        if (tasks.empty()) return BDDC_OK;
        // one allocation for the task list, the item table and the flags, freed by
        // the stream-ordered allocator after the launch
        const size_t tb = tasks.size() * sizeof(EngTask), mb = meta.size() * sizeof(EngMeta);
        const size_t fb = sizeof(int) * ((size_t)nflags + 2);
        const size_t o1 = (tb + 255) & ~size_t(255), o2 = o1 + ((mb + 255) & ~size_t(255));
        std::vector<unsigned char> host(o2);
        memcpy(host.data(), tasks.data(), tb);
        memcpy(host.data() + o1, meta.data(), mb);
        unsigned char* dev = nullptr;
        BDDC_CUDA_TRY(cudaMallocAsync((void**)&dev, o2 + fb, st));
        BDDC_CUDA_TRY(cudaMemcpyAsync(dev, host.data(), o2, cudaMemcpyHostToDevice, st));
        int* flags = reinterpret_cast<int*>(dev + o2);
        BDDC_CUDA_TRY(cudaMemsetAsync(flags, 0, fb, st));
        const size_t sm = task_smem<T>();
        auto kern = k_engine_tasks<T, NB, TILE>;
        BDDC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int dev_id = 0, nsm = 0, occ = 0;
        BDDC_CUDA_TRY(cudaGetDevice(&dev_id));
        BDDC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev_id));
        BDDC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, UPD_THREADS, sm));
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
                                             flags + nflags + 1, dscr, stride, err);
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
                                const int*, const int*, bool);
template int engine_run<float>(const EngItem<float>*, int, int, int, float*, int*, cudaStream_t,
                               const int*, const int*, bool);
