// Adaptive primal constraints: deluxe scaling, face GEP and the edge GEP on
// prior-selected primal constraints (Sect. 3), one CTA per face / edge, FP64.
//
// Face F, n(F) = {i, j} (eqs. conv-proof-key-F ... primal-constraints-F):
//   D^(i) = (S_FF^(i) + S_FF^(j))^{-1} S_FF^(i)                 (deluxe scaling)
//   B_F   = D^(j)T B_FF^(i) D^(j) + D^(i)T B_FF^(j) D^(i)
//   B~_F  = B~_F^(i) : B~_F^(j)                                 (parallel sum)
//   B_F v = lambda B~_F v, select lambda >= Theta_F, constraints (B_F v_l)^T (w_i,F - w_j,F) = 0.
// Edge E, n(E) = {k_1 < ... < k_m} (eqs. equ-5-19 ... equ-5-22, m = 4 here):
//   w_check_k = w_k,E - w_k1,E, w^_E = sum_k D^(k) w_k,E, w_k,E = T^(k) (w_check; w^_E)
//   M_E  = Tbar^T diag(B_E^(k)) Tbar
//   B~_E = sum_k J_k^T B~^(k) J_k with B~^(k) the Schur complement of B^(k) onto
//          E and the prior primal unknowns H_k (vertices, face primal coordinates),
//          shared primal unknowns identified
//   B~~_E = B~_E with (w^_E, w^_H) eliminated;  M_E v = lambda B~~_E v,
//   select lambda >= Theta_E, Q_E = orthonormal basis of the span of the n_E-blocks
//   of M_E v_l (order n_E; the remark after eq. equ-5-22).
// The pencils X v = lambda Y v (X, Y symmetric positive semi-definite) are
// solved as X v = sigma (X+Y) v: eigen-decompose K = X+Y (cyclic Jacobi), drop
// its null directions (<= 1e-12 max), reduce, eigen-decompose again;
// lambda = sigma / (1 - sigma).  Pseudo-inverse Schur complements use
// symmetric diagonal pivoting and stop at pivots <= 1e-12 of the largest
// diagonal.  The constraint span uses Householder QR with column pivoting and
// relative rank tolerance 1e-10; its full Q is the change of basis
// T_X = [Q_X, Q_X^perp] used by the constrained local solvers.
#include <cuda_runtime.h>

#include "bddc_internal.h"
#include "gep.h"

namespace {

constexpr int GT = 512;                 // threads per GEP CTA
// Tolerances per precision: the FP64 values are the readings of the paper
// (1e-12 null-space drop, 1e-10 rank); FP32 uses values above its noise floor.
template <class T> struct Tol;
template <> struct Tol<double> {
    static constexpr double drop = 1e-12, rank = 1e-10, slack = 1e-12, tiny = 1e-300;
    static constexpr double rot_rel = 1e-14, rot_abs = 1e-15, chol = 1e-12;
};
template <> struct Tol<float> {
    static constexpr double drop = 1e-6, rank = 1e-5, slack = 1e-6, tiny = 1e-30;
    static constexpr double rot_rel = 1e-6, rot_abs = 1e-7, chol = 1e-5;
};
constexpr int JACOBI_MAX_SWEEPS = 60;

__device__ __forceinline__ void bar() { __syncthreads(); }

// Visit every (i, j) of an m x n index space with the CTA's threads; one
// integer division per thread instead of one per element (integer division
// by a run-time value is a long instruction sequence on this GPU).  An empty
// extent (m <= 0 or n <= 0) visits nothing.
#define CTA_FOR_2D(i, j, m, n)                                                             \
    for (int i##_n = (n) > 0 ? (n) : 1, i = (n) > 0 ? (int)threadIdx.x / i##_n : (m),      \
             j = (int)threadIdx.x % i##_n, i##_st = GT / i##_n, j##_st = GT % i##_n;       \
         i < (m); i += i##_st, j += j##_st, i += (j >= i##_n), j -= (j >= i##_n) ? i##_n : 0)

template <class T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA (every thread gets the result).
template <class T>
__device__ T block_sum(T v) {
    __shared__ T red[GT / 32];
    v = wsum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    bar();
    T tot = 0;
#pragma unroll
    for (int q = 0; q < GT / 32; ++q) tot += red[q];
    bar();
    return tot;
}

// Arg-max over the CTA of (value, index); ties keep the smaller index.
template <class T>
__device__ void block_argmax(T v, int i, T* vout, int* iout) {
    __shared__ T rv[GT / 32];
    __shared__ int ri[GT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
    }
    if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = v; ri[threadIdx.x >> 5] = i; }
    bar();
    T bv = rv[0];
    int bi = ri[0];
    for (int q = 1; q < GT / 32; ++q)
        if (rv[q] > bv || (rv[q] == bv && ri[q] < bi)) { bv = rv[q]; bi = ri[q]; }
    *vout = bv;
    *iout = bi;
    bar();
}

// Arg-max over a warp of (value, index); ties keep the smaller index.
template <class T>
__device__ __forceinline__ void warp_argmax(T& v, int& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
    }
}

// Arg-max of per-warp partial results (rv, ri)[0 .. GT / 32), read by every thread.
template <class T>
__device__ __forceinline__ void argmax_of(const T* rv, const int* ri, T* vout, int* iout) {
    T bv = rv[0];
    int bi = ri[0];
#pragma unroll
    for (int q = 1; q < GT / 32; ++q)
        if (rv[q] > bv || (rv[q] == bv && ri[q] < bi)) { bv = rv[q]; bi = ri[q]; }
    *vout = bv;
    *iout = bi;
}

// Row updates of the step loops below: with g = GT / rows threads per row (at
// least 1), thread t takes the rows t / g + (GT / g) u and, within a row, the
// columns t % g + g v, so that a row's multiplier stays in a register and the
// threads of a row touch consecutive columns.
struct RowMap {
    int g, tr, tq, rs;
    __device__ explicit RowMap(int rows, int gmax = GT) {
        g = min(gmax, rows > 0 ? max(1, GT / rows) : GT);
        tr = (int)threadIdx.x / g;
        tq = (int)threadIdx.x - tr * g;
        rs = GT / g;
    }
};

// C = alpha * op(A) * op(B) + beta * C ; row-major; transA/transB flags
template <class T, class TA, class TB, class TC>
__device__ void mm(const TA* A, int lda, bool ta, const TB* B, int ldb, bool tb, TC* C,
                   int ldc, int m, int n, int k, T alpha, T beta) {
    CTA_FOR_2D(i, j, m, n) {
        T s = 0;
        for (int l = 0; l < k; ++l) {
            T a = ta ? (T)A[l * lda + i] : (T)A[i * lda + l];
            T b = tb ? (T)B[j * ldb + l] : (T)B[l * ldb + j];
            s += a * b;
        }
        C[i * ldc + j] = (TC)(alpha * s + (beta == (T)0 ? (T)0 : beta * (T)C[i * ldc + j]));
    }
    bar();
}

template <class TA, class TB>
__device__ void copy_mat(const TA* A, int lda, TB* B, int ldb, int m, int n) {
    CTA_FOR_2D(i, j, m, n) B[i * ldb + j] = (TB)A[i * lda + j];
    bar();
}

template <class T>
__device__ void symmetrize(T* A, int ld, int n) {
    CTA_FOR_2D(i, j, n, n) {
        if (i < j) {
            T v = (T)0.5 * (A[i * ld + j] + A[j * ld + i]);
            A[i * ld + j] = v;
            A[j * ld + i] = v;
        }
    }
    bar();
}

// Solve A X = B in place (A n x n overwritten by its U factor, B n x nr
// overwritten by X); Gaussian elimination with partial pivoting on [A | B], then
// back substitution.  Row updates per thread row (GQ threads per row, the
// multiplier in a register); the back substitution uses x_c = B(c, :) / U(c, c)
// on the fly (row c is final by then) and divides every row at the end.
template <class T>
__device__ void lu_solve(T* A, int lda, T* B, int ldb, int n, int nr, int* err) {
    __shared__ int piv_s;
    __shared__ T pv_s[32];
    __shared__ int pi_s[32];
    const RowMap rm(n);
    const int tr = rm.tr, tq = rm.tq, GQ = rm.g, RS = rm.rs;
    for (int c = 0; c < n; ++c) {
        // pivot search by warp 0
        if (threadIdx.x < 32) {
            T best = -1.0;
            int bi = c;
            for (int r = c + threadIdx.x; r < n; r += 32) {
                T v = fabs(A[r * lda + c]);
                if (v > best) { best = v; bi = r; }
            }
            pv_s[threadIdx.x] = best;
            pi_s[threadIdx.x] = bi;
            __syncwarp();
            if (threadIdx.x == 0) {
                T b = -1.0;
                int ii = c;
                for (int q = 0; q < 32; ++q)
                    if (pv_s[q] > b) { b = pv_s[q]; ii = pi_s[q]; }
                piv_s = ii;
                if (!(b > 0.0)) atomicOr(err, ERR_PIVOT);
            }
        }
        bar();
        const int p = piv_s;
        if (p != c) {
            for (int q = threadIdx.x; q < n; q += GT) {
                T t = A[c * lda + q]; A[c * lda + q] = A[p * lda + q]; A[p * lda + q] = t;
            }
            for (int q = threadIdx.x; q < nr; q += GT) {
                T t = B[c * ldb + q]; B[c * ldb + q] = B[p * ldb + q]; B[p * ldb + q] = t;
            }
            bar();
        }
        T d = A[c * lda + c];
        if (d == (T)0) d = (T)Tol<T>::tiny;
        const int rem = n - c - 1;
        for (int r = c + 1 + tr; r < n; r += RS) {
            const T l = A[r * lda + c] / d;
#pragma unroll 4
            for (int j = tq; j < rem; j += GQ) A[r * lda + c + 1 + j] -= l * A[c * lda + c + 1 + j];
#pragma unroll 4
            for (int j = tq; j < nr; j += GQ) B[r * ldb + j] -= l * B[c * ldb + j];
        }
        bar();
    }
    // back substitution
    for (int c = n - 1; c > 0; --c) {
        T d = A[c * lda + c];
        if (d == (T)0) d = (T)Tol<T>::tiny;
        for (int r = tr; r < c; r += RS) {
            const T a = A[r * lda + c];
#pragma unroll 4
            for (int j = tq; j < nr; j += GQ) B[r * ldb + j] -= a * (B[c * ldb + j] / d);
        }
        bar();
    }
    for (int r = tr; r < n; r += RS) {
        T d = A[r * lda + r];
        if (d == (T)0) d = (T)Tol<T>::tiny;
        for (int j = tq; j < nr; j += GQ) B[r * ldb + j] /= d;
    }
    bar();
}

// Generalised Schur complement of a symmetric PSD matrix: eliminate the
// indices [r0, n) by symmetric diagonal pivoting; pivots <= tol * (largest
// initial diagonal among them) are left (their directions carry no energy).
// The leading r0 x r0 block then holds M_ww - M_wr M_rr^+ M_rw.
template <class T>
__device__ void pinv_schur_tail(T* M, int ld, int n, int r0, unsigned char* done) {
    // One barrier per pivot: the threads that update a diagonal entry of the
    // tail also reduce the next pivot's arg-max, per warp, into a double-buffered
    // array that every thread reads after the barrier (ties to the smaller index).
    __shared__ T dmax0_s;
    __shared__ T rv[2][GT / 32];
    __shared__ int ri[2][GT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const RowMap rm(n, 4);      // (more threads per row measured slower on the 2n x 2n sums)
    const int tr = rm.tr, tq = rm.tq, GQ = rm.g, RS = rm.rs;
    for (int q = threadIdx.x; q < n; q += GT) done[q] = q < r0 ? 1 : 0;
    if (threadIdx.x == 0) {
        T d = 0.0;
        for (int q = r0; q < n; ++q) d = fmax(d, M[q * ld + q]);
        dmax0_s = d;
    }
    {
        T b = (T)-1;
        int bi = n;
        for (int q = r0 + threadIdx.x; q < n; q += GT)
            if (M[q * ld + q] > b) { b = M[q * ld + q]; bi = q; }
        warp_argmax(b, bi);
        if (lane == 0) { rv[0][wid] = b; ri[0][wid] = bi; }
    }
    bar();
    const T tol = (T)Tol<T>::drop * dmax0_s;
    int buf = 0;
    for (int step = r0; step < n; ++step) {
        T bv;
        int p;
        argmax_of(rv[buf], ri[buf], &bv, &p);
        if (p >= n || !(bv > tol)) break;        // the same decision in every thread
        done[p] = 1;                             // same value from every thread; p is skipped below
        const T rdp = (T)1 / M[p * ld + p];
        T b = (T)-1;
        int bi = n;
        // update all not-yet-eliminated rows/cols (including the kept block)
        for (int i = tr; i < n; i += RS) {
            if (i == p || (i >= r0 && done[i])) continue;
            const T l = M[i * ld + p] * rdp;
#pragma unroll 4
            for (int j = tq; j < n; j += GQ) {
                // branch-free body (predicated store): the loads of several columns in flight
                const bool act = j != p && !(j >= r0 && done[j]);
                const T v = M[i * ld + j] - l * M[p * ld + j];
                if (act) M[i * ld + j] = v;
                if (act && j == i && i >= r0 && v > b) { b = v; bi = i; }
            }
        }
        warp_argmax(b, bi);
        if (lane == 0) { rv[buf ^ 1][wid] = b; ri[buf ^ 1][wid] = bi; }
        bar();
        buf ^= 1;
    }
}

// Cyclic parallel Jacobi (round-robin pairs) on a symmetric positive
// semi-definite n x n matrix in shared memory, row stride ld (odd: no bank
// conflicts on column access), np = n rounded up to even.  A rotation is
// applied only when |a_pq| exceeds both rot_rel * sqrt|a_pp a_qq| and
// rot_abs * max_k a_kk; the sweep in which no rotation was applied ends the
// iteration.  On exit diag(A) = eigenvalues, V = eigenvectors (columns).
template <class T>
__device__ int jacobi(T* A, T* V, int n, int np, int ld, T* cs, T* sn, int* pp, int* qq, int* err) {
    CTA_FOR_2D(i, j, np, np) {
        V[i * ld + j] = i == j ? (T)1 : (T)0;
        if (i >= n || j >= n) A[i * ld + j] = 0;
    }
    __shared__ T amax_s;
    __shared__ int rotated_s;
    bar();
    if (threadIdx.x == 0) {
        T m = 0;
        for (int i = 0; i < n; ++i) m = fmax(m, fabs(A[i * ld + i]));
        amax_s = m;
    }
    bar();
    const T floor_abs = (T)Tol<T>::rot_abs * amax_s;
    const int half = np / 2;
    if (threadIdx.x == 0) rotated_s = 0;
    bar();
    for (int sweep = 0; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
        for (int r = 0; r < np - 1; ++r) {
            for (int k = threadIdx.x; k < half; k += GT) {
                int p = (r + k) % (np - 1);
                int q = k == 0 ? np - 1 : (r - k + np - 1) % (np - 1);
                if (p > q) { int t = p; p = q; q = t; }
                pp[k] = p;
                qq[k] = q;
                T c = 1, s = 0;
                T apq = A[p * ld + q];
                if (q < n) {
                    T app = A[p * ld + p], aqq = A[q * ld + q];
                    T lim = fmax((T)Tol<T>::rot_rel * sqrt(fabs(app * aqq)), floor_abs);
                    if (fabs(apq) > lim && fabs(apq) > (T)Tol<T>::tiny) {
                        T th = (aqq - app) / ((T)2 * apq);
                        T t = (th >= 0 ? (T)1 : (T)-1) / (fabs(th) + sqrt((T)1 + th * th));
                        c = (T)1 / sqrt((T)1 + t * t);
                        s = t * c;
                        rotated_s = 1;
                    }
                }
                cs[k] = c;
                sn[k] = s;
            }
            bar();
            CTA_FOR_2D(k, col, half, np) {                             // rows p, q
                T s = sn[k];
                if (s == (T)0) continue;
                int p = pp[k], qi = qq[k];
                T c = cs[k];
                T a = A[p * ld + col], b = A[qi * ld + col];
                A[p * ld + col] = c * a - s * b;
                A[qi * ld + col] = s * a + c * b;
            }
            bar();
            CTA_FOR_2D(k, row, half, np) {                             // columns p, q
                T s = sn[k];
                if (s == (T)0) continue;
                int p = pp[k], qi = qq[k];
                T c = cs[k];
                T a = A[row * ld + p], b = A[row * ld + qi];
                A[row * ld + p] = c * a - s * b;
                A[row * ld + qi] = s * a + c * b;
                T va = V[row * ld + p], vb = V[row * ld + qi];
                V[row * ld + p] = c * va - s * vb;
                V[row * ld + qi] = s * va + c * vb;
            }
            bar();
            for (int k = threadIdx.x; k < half; k += GT) {          // the rotated pair is zero
                if (sn[k] != (T)0) {
                    A[pp[k] * ld + qq[k]] = 0;
                    A[qq[k] * ld + pp[k]] = 0;
                }
            }
        }
        bar();
        const int any = rotated_s;      // every thread reads the flag before it is reset
        bar();
        if (threadIdx.x == 0) rotated_s = 0;
        bar();                          // and the reset lands before the next sweep sets it
        if (!any) return sweep + 1;
    }
    if (threadIdx.x == 0) atomicOr(err, ERR_JACOBI);
    return JACOBI_MAX_SWEEPS;
}

// Sort (val, vec columns) by decreasing value (n small; thread 0 computes the order).
template <class T>
__device__ void sort_desc(const T* A, int ld, int n, int* order) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) order[i] = i;
        for (int i = 1; i < n; ++i) {
            int v = order[i];
            T key = A[v * ld + v];
            int j = i - 1;
            while (j >= 0 && A[order[j] * ld + order[j]] < key) { order[j + 1] = order[j]; --j; }
            order[j + 1] = v;
        }
    }
    bar();
}

// In-place Cholesky K = L L^T (lower triangle, shared memory, stride ld);
// returns false when a pivot falls to <= tol * (largest initial diagonal).
// Step k subtracts A(i, k) A(j, k) / d_k from the trailing lower triangle with
// column k still unscaled (it is not written in the step), so one barrier per
// step suffices; the columns are scaled by 1 / sqrt(d_k) at the end.
template <class T>
__device__ bool cholesky(T* A, int n, int ld, T tol) {
    __shared__ T dmax_s;
    const RowMap rm(n);
    const int tr = rm.tr, tq = rm.tq, GQ = rm.g, RS = rm.rs;
    if (threadIdx.x == 0) {
        T m = 0;
        for (int i = 0; i < n; ++i) m = fmax(m, A[i * ld + i]);
        dmax_s = m;
    }
    bar();
    const T dmax = dmax_s;
    if (!(dmax > (T)0)) return false;
    for (int k = 0; k < n; ++k) {
        const T d = A[k * ld + k];
        if (!(d > tol * dmax)) return false;     // the same decision in every thread
        const T rd = (T)1 / d;
        for (int i = k + 1 + tr; i < n; i += RS) {
            const T l = A[i * ld + k] * rd;
#pragma unroll 4
            for (int j = k + 1 + tq; j <= i; j += GQ) A[i * ld + j] -= l * A[j * ld + k];
        }
        bar();
    }
    for (int i = tr; i < n; i += RS)
        for (int k = tq; k < i; k += GQ) A[i * ld + k] /= sqrt(A[k * ld + k]);
    bar();
    for (int k = threadIdx.x; k < n; k += GT) A[k * ld + k] = sqrt(A[k * ld + k]);
    bar();
    return true;
}

// X <- L^{-1} X for an n x m block X (row stride ldx), L lower in (Ls, ldl).
// Step k subtracts L(i, k) (X(k, :) / L(k, k)) from the rows below, X(k, :) being
// final by then; every row is divided by its diagonal entry at the end.  One
// barrier per step, thread rows as in the eliminations.
template <class T>
__device__ void trsm_lower(const T* Ls, int ldl, T* X, int ldx, int n, int m) {
    const RowMap rm(n);
    const int tr = rm.tr, tq = rm.tq, GQ = rm.g, RS = rm.rs;
    for (int k = 0; k + 1 < n; ++k) {
        const T inv = (T)1 / Ls[k * ldl + k];
        for (int i = k + 1 + tr; i < n; i += RS) {
            const T l = Ls[i * ldl + k];
#pragma unroll 4
            for (int c = tq; c < m; c += GQ) X[i * ldx + c] -= l * (X[k * ldx + c] * inv);
        }
        bar();
    }
    for (int k = tr; k < n; k += RS) {
        const T inv = (T)1 / Ls[k * ldl + k];
        for (int c = tq; c < m; c += GQ) X[k * ldx + c] *= inv;
    }
    bar();
}

// X <- L^{-T} X for an n x m block X (as above, from the last row up).
template <class T>
__device__ void trsm_lower_t(const T* Ls, int ldl, T* X, int ldx, int n, int m) {
    const RowMap rm(n);
    const int tr = rm.tr, tq = rm.tq, GQ = rm.g, RS = rm.rs;
    for (int k = n - 1; k > 0; --k) {
        const T inv = (T)1 / Ls[k * ldl + k];
        for (int i = tr; i < k; i += RS) {
            const T l = Ls[k * ldl + i];
#pragma unroll 4
            for (int c = tq; c < m; c += GQ) X[i * ldx + c] -= l * (X[k * ldx + c] * inv);
        }
        bar();
    }
    for (int k = tr; k < n; k += RS) {
        const T inv = (T)1 / Ls[k * ldl + k];
        for (int c = tq; c < m; c += GQ) X[k * ldx + c] *= inv;
    }
    bar();
}

// Largest order the tridiagonal eigen-solver handles (shared-memory vectors).
constexpr int TRI_EIG_MAX = FACE_NMAX;

// Sturm count: eigenvalues of the symmetric tridiagonal (d, e) below x.
template <class T>
__device__ __forceinline__ int sturm_count(const T* d, const T* e2, int n, T x, T pivmin) {
    int c = 0;
    T q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < (T)0;
    for (int i = 1; i < n; ++i) {
        q = d[i] - x - e2[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        c += q < (T)0;
    }
    return c;
}

// Eigen-decomposition of the symmetric n x n matrix A (shared memory, stride ld;
// destroyed) for the eigenvalues >= thr only: every eigenvalue goes to sig[0..n)
// in decreasing order; the eigenvectors of the first s (those >= thr) to the
// columns 0..s-1 of V (row stride ldv); s is returned.  Steps: Householder
// reduction to tridiagonal form (reflectors kept in A's lower part), all
// eigenvalues by parallel multisection on Sturm counts (8 lanes per eigenvalue),
// inverse iteration with partial pivoting on the tridiagonal for the selected
// ones (re-orthogonalised within clusters), back-transformation by the
// reflectors.  work: 5 n elements per selected eigenvalue, cap of them; when more
// than cap eigenvalues are selected no vector is computed and -s is returned.
template <class T>
__device__ int tridiag_eig_sel(T* A, int ld, int n, T thr, T* sig, T* V, int ldv, T* work, int cap) {
    __shared__ T td[TRI_EIG_MAX], te[TRI_EIG_MAX], te2[TRI_EIG_MAX], tb[TRI_EIG_MAX], tv[TRI_EIG_MAX],
        tp[TRI_EIG_MAX];
    __shared__ T sc_s[2];
    __shared__ int s_sel;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    // ---- 1. tridiagonalisation: step k zeroes A[k+2.., k]
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        if (wid == 0) {
            T sg = 0;
            for (int i = 1 + lane; i < m; i += 32) {
                const T x = A[(k + 1 + i) * ld + k];
                sg += x * x;
            }
            sg = wsum(sg);
            if (lane == 0) {
                const T x0 = A[(k + 1) * ld + k];
                if (sg == (T)0) {
                    sc_s[0] = 0;          // beta: column already reduced
                    te[k] = x0;
                    tv[0] = 0;
                } else {
                    const T nrm = sqrt(x0 * x0 + sg);
                    const T alpha = x0 >= (T)0 ? -nrm : nrm;
                    const T v0 = x0 - alpha;
                    tv[0] = v0;
                    sc_s[0] = (T)2 / (v0 * v0 + sg);
                    te[k] = alpha;
                }
                td[k] = A[k * ld + k];
            }
            __syncwarp();
            for (int i = 1 + lane; i < m; i += 32) tv[i] = A[(k + 1 + i) * ld + k];
        }
        bar();
        const T beta = sc_s[0];
        if (beta != (T)0) {
            // p = beta A_sub v
            for (int i = t; i < m; i += GT) {
                const T* row = A + (k + 1 + i) * ld + k + 1;
                T acc = 0;
                for (int j = 0; j < m; ++j) acc += row[j] * tv[j];
                tp[i] = beta * acc;
            }
            bar();
            if (wid == 0) {
                T kk = 0;
                for (int i = lane; i < m; i += 32) kk += tp[i] * tv[i];
                kk = wsum(kk);
                if (lane == 0) sc_s[1] = (T)0.5 * beta * kk;
            }
            bar();
            const T K = sc_s[1];
            for (int i = t; i < m; i += GT) tp[i] -= K * tv[i];      // w = p - K v
            bar();
            CTA_FOR_2D(i, j, m, m) A[(k + 1 + i) * ld + k + 1 + j] -= tv[i] * tp[j] + tp[i] * tv[j];
        }
        // keep the reflector (v, beta) for the back-transformation
        for (int i = t; i < m; i += GT) A[(k + 1 + i) * ld + k] = tv[i];
        if (t == 0) tb[k] = beta;
        bar();
    }
    if (t == 0) {
        if (n >= 2) {
            td[n - 2] = A[(n - 2) * ld + n - 2];
            te[n - 2] = A[(n - 1) * ld + n - 2];
        }
        td[n - 1] = A[(n - 1) * ld + n - 1];
    }
    bar();
    for (int i = t; i + 1 < n; i += GT) te2[i] = te[i] * te[i];
    // Gershgorin interval
    if (t == 0) {
        T lo = td[0], hi = td[0], amax = 0;
        for (int i = 0; i < n; ++i) {
            const T r = (i > 0 ? fabs(te[i - 1]) : (T)0) + (i + 1 < n ? fabs(te[i]) : (T)0);
            lo = fmin(lo, td[i] - r);
            hi = fmax(hi, td[i] + r);
            amax = fmax(amax, fmax(fabs(td[i]), r));
        }
        sc_s[0] = lo - (T)1e-6 * (amax + (T)1e-30);
        sc_s[1] = hi + (T)1e-6 * (amax + (T)1e-30);
    }
    bar();
    // ---- 2. all eigenvalues: 8 lanes per eigenvalue, 9-section per round
    {
        const T lo0 = sc_s[0], hi0 = sc_s[1];
        const T pivmin = (T)1e-30 + (T)4 * (T)Tol<T>::tiny;
        const int sub = lane & 7;
        for (int g0 = 0; g0 < n; g0 += GT / 8) {
            const int g = g0 + (t >> 3);                // ascending index j
            const bool act = g < n;
            T a = lo0, b = hi0;
            for (int round = 0; round < 12; ++round) {
                const T x = a + (b - a) * (T)(sub + 1) / (T)9;
                const int c = act ? sturm_count(td, te2, n, x, pivmin) : n;
                const unsigned ok = __ballot_sync(0xffffffffu, c <= g) >> (lane & 24);
                const int cnt = __popc(ok & 0xffu);    // points (increasing) at or below lambda_g
                const T xa = __shfl_sync(0xffffffffu, x, (lane & 24) + max(cnt - 1, 0));
                const T xb = __shfl_sync(0xffffffffu, x, (lane & 24) + min(cnt, 7));
                const T na = cnt > 0 ? xa : a;
                const T nb = cnt < 8 ? xb : b;
                a = na;
                b = nb;
            }
            if (act && sub == 0) sig[n - 1 - g] = (T)0.5 * (a + b);
        }
    }
    bar();
    if (t == 0) {
        int c = 0;
        while (c < n && sig[c] >= thr) ++c;
        s_sel = c;
    }
    bar();
    const int s = s_sel;
    if (s == 0) return 0;
    if (s > cap) return -s;
    // ---- 3. inverse iteration on T - lambda I (thread per selected eigenvalue)
    T amax = 0;
    for (int i = 0; i < n; ++i) amax = fmax(amax, fabs(td[i]) + (i + 1 < n ? fabs(te[i]) : (T)0));
    const T eps = sizeof(T) == 4 ? (T)1.2e-7 : (T)2.3e-16;
    for (int it = 0; it < 3; ++it) {
        for (int q = t; q < s; q += GT) {
            T* x = V + q;                                    // column q, stride ldv
            T* u0 = work + (size_t)q * 5 * n;
            T* u1 = u0 + n;
            T* u2 = u1 + n;
            T* ml = u2 + n;
            T* sw = ml + n;
            const T lam = sig[q];
            if (it == 0)
                for (int i = 0; i < n; ++i)                  // a start vector particular to q
                    x[i * ldv] = (T)1 + (T)0.25 * sin((T)(0.7 + 0.37 * q) * (T)(i + 1));
            // factor T - lam I with partial pivoting (rows i, i+1)
            T a = td[0] - lam, b = n > 1 ? te[0] : (T)0, c2 = 0;
            for (int i = 0; i < n; ++i) {
                if (i + 1 < n) {
                    const T cdn = te[i];                     // subdiagonal of row i+1
                    const T an = td[i + 1] - lam;
                    const T bn = i + 2 < n ? te[i + 1] : (T)0;
                    if (fabs(a) >= fabs(cdn)) {
                        const T mlt = a != (T)0 ? cdn / a : (T)0;
                        u0[i] = a; u1[i] = b; u2[i] = c2; ml[i] = mlt; sw[i] = 0;
                        a = an - mlt * b;
                        b = bn;
                        c2 = 0;
                    } else {
                        const T mlt = a / cdn;
                        u0[i] = cdn; u1[i] = an; u2[i] = bn; ml[i] = mlt; sw[i] = 1;
                        a = b - mlt * an;
                        b = -mlt * bn;
                        c2 = 0;
                    }
                } else {
                    u0[i] = a; u1[i] = 0; u2[i] = 0;
                }
                if (fabs(u0[i]) < eps * amax) u0[i] = u0[i] >= (T)0 ? eps * amax : -eps * amax;
            }
            // forward: apply the row operations to x
            for (int i = 0; i + 1 < n; ++i) {
                T xi = x[i * ldv], xn = x[(i + 1) * ldv];
                if (sw[i] != (T)0) {
                    const T tmp = xi;
                    xi = xn;
                    xn = tmp;
                }
                x[i * ldv] = xi;
                x[(i + 1) * ldv] = xn - ml[i] * xi;
            }
            // back substitution with the banded U (diagonal u0, superdiagonals u1, u2)
            for (int i = n - 1; i >= 0; --i) {
                T v = x[i * ldv];
                if (i + 1 < n) v -= u1[i] * x[(i + 1) * ldv];
                if (i + 2 < n) v -= u2[i] * x[(i + 2) * ldv];
                x[i * ldv] = v / u0[i];
            }
            T nn = 0;
            for (int i = 0; i < n; ++i) nn += x[i * ldv] * x[i * ldv];
            nn = (T)1 / sqrt(fmax(nn, (T)1e-300));
            for (int i = 0; i < n; ++i) x[i * ldv] *= nn;
        }
        bar();
        // re-orthogonalise within clusters (eigenvalues closer than 1e-3 of the spread)
        if (t == 0) {
            const T gap = (T)1e-3 * fmax(amax, (T)1e-30);
            for (int q = 1; q < s; ++q) {
                for (int r = 0; r < q; ++r) {
                    if (fabs(sig[r] - sig[q]) > gap) continue;
                    T dp = 0;
                    for (int i = 0; i < n; ++i) dp += V[i * ldv + r] * V[i * ldv + q];
                    for (int i = 0; i < n; ++i) V[i * ldv + q] -= dp * V[i * ldv + r];
                }
                T nn = 0;
                for (int i = 0; i < n; ++i) nn += V[i * ldv + q] * V[i * ldv + q];
                nn = (T)1 / sqrt(fmax(nn, (T)1e-300));
                for (int i = 0; i < n; ++i) V[i * ldv + q] *= nn;
            }
        }
        bar();
    }
    // ---- 4. back-transformation: x <- H_0 ... H_{n-3} x, one warp per vector
    for (int q = wid; q < s; q += GT / 32) {
        for (int k = n - 3; k >= 0; --k) {
            const T beta = tb[k];
            if (beta == (T)0) continue;
            const int m = n - k - 1;
            T dp = 0;
            for (int i = lane; i < m; i += 32) dp += A[(k + 1 + i) * ld + k] * V[(k + 1 + i) * ldv + q];
            dp = wsum(dp) * beta;
            for (int i = lane; i < m; i += 32) V[(k + 1 + i) * ldv + q] -= dp * A[(k + 1 + i) * ld + k];
            __syncwarp();
        }
    }
    bar();
    return s;
}

// Solve X v = sigma (X + Y) v for symmetric PSD X, Y (n x n in global scratch).
// On exit: sig[0..r) decreasing, Vout (n x r, row stride r) = eigenvectors
// with Vout^T (X+Y) Vout = I, r returned.  FP64 (the oracle's reading):
// eigen-decompose K = X + Y, drop its null directions, reduce, eigen-decompose.
// FP32: when K is safely positive definite, reduce by its Cholesky factor
// instead of the first eigen-decomposition.
template <class T>
__device__ int sigma_pencil(const T* X, const T* Y, int n, T* Ash, T* Vsh, int np, int ld,
                            T* work1, T* work2, T* sig, T* Vout, T* cs,
                            T* sn, int* pp, int* qq, int* order, int* err, int* sweeps, T thr) {
    __shared__ int r_s;
    CTA_FOR_2D(i, j, n, n) {
        Ash[i * ld + j] = (T)0.5 * (X[i * n + j] + X[j * n + i]) + (T)0.5 * (Y[i * n + j] + Y[j * n + i]);
    }
    bar();
    if (sizeof(T) == 4 && cholesky(Ash, n, ld, (T)Tol<T>::chol)) {
        // L -> work1 (n x n), C = L^{-1} X L^{-T} -> Ash
        CTA_FOR_2D(i, j, n, n) work1[i * n + j] = j <= i ? Ash[i * ld + j] : (T)0;
        bar();
        CTA_FOR_2D(i, j, n, n) work2[i * n + j] = X[i * n + j];
        bar();
        trsm_lower(work1, n, work2, n, n, n);                     // Z = L^{-1} X
        CTA_FOR_2D(i, j, n, n) Ash[i * ld + j] = work2[j * n + i];  // Z^T
        bar();
        trsm_lower(work1, n, Ash, ld, n, n);                      // L^{-1} Z^T = C
        CTA_FOR_2D(i, j, n, n) {
            if (i < j) {
                T v = (T)0.5 * (Ash[i * ld + j] + Ash[j * ld + i]);
                Ash[i * ld + j] = v;
                Ash[j * ld + i] = v;
            }
        }
        bar();
        if (n <= TRI_EIG_MAX) {
            // eigenvectors are needed for the selected eigenvalues only: tridiagonal
            // route; the matrix is kept in work2 in case more are selected than fit
            CTA_FOR_2D(i, j, n, n) work2[i * n + j] = Ash[i * ld + j];
            bar();
            const int cap = (np * ld) / (5 * n);
            const int s = tridiag_eig_sel(Ash, ld, n, thr, sig, Vout, n, Vsh, cap);
            if (s >= 0) {
                if (s > 0) trsm_lower_t(work1, n, Vout, n, n, s);        // V = L^{-T} Y
                return n;
            }
            CTA_FOR_2D(i, j, n, n) Ash[i * ld + j] = work2[i * n + j];
            bar();
        }
        int sw = jacobi(Ash, Vsh, n, np, ld, cs, sn, pp, qq, err);
        if (threadIdx.x == 0) atomicMax(sweeps, sw);
        sort_desc(Ash, ld, n, order);
        for (int q = threadIdx.x; q < n; q += GT) sig[q] = Ash[order[q] * ld + order[q]];
        CTA_FOR_2D(i, c, n, n) Vout[i * n + c] = Vsh[i * ld + order[c]];
        bar();
        trsm_lower_t(work1, n, Vout, n, n, n);                    // V = L^{-T} Y
        return n;
    }
    // eigen-decomposition route (also the fallback of the FP32 path)
    CTA_FOR_2D(i, j, n, n) {
        Ash[i * ld + j] = (T)0.5 * (X[i * n + j] + X[j * n + i]) + (T)0.5 * (Y[i * n + j] + Y[j * n + i]);
    }
    bar();
    int sw = jacobi(Ash, Vsh, n, np, ld, cs, sn, pp, qq, err);
    if (threadIdx.x == 0) {
        atomicMax(sweeps, sw);
        T m = 0;
        for (int i = 0; i < n; ++i) m = fmax(m, Ash[i * ld + i]);
        int r = 0;
        for (int i = 0; i < n; ++i)
            if (m > (T)0 && Ash[i * ld + i] > (T)Tol<T>::drop * m) order[r++] = i;
        r_s = r;
    }
    bar();
    const int r = r_s;
    if (r == 0) return 0;
    // W = U_keep / sqrt(kappa)  (n x r) -> work1
    CTA_FOR_2D(i, c, n, r) {
        int col = order[c];
        work1[i * r + c] = Vsh[i * ld + col] / sqrt(Ash[col * ld + col]);
    }
    bar();
    // C = W^T X W -> shared A (r x r)
    mm(X, n, false, work1, r, false, work2, r, n, r, n, (T)1, (T)0);        // X W  (n x r)
    mm(work1, r, true, work2, r, false, Ash, ld, r, r, n, (T)1, (T)0);     // W^T (X W)
    CTA_FOR_2D(i, j, r, r) {
        if (i < j) {
            T v = (T)0.5 * (Ash[i * ld + j] + Ash[j * ld + i]);
            Ash[i * ld + j] = v;
            Ash[j * ld + i] = v;
        }
    }
    bar();
    const int rp = (r + 1) & ~1;
    sw = jacobi(Ash, Vsh, r, rp, ld, cs, sn, pp, qq, err);
    if (threadIdx.x == 0) atomicMax(sweeps, sw);
    sort_desc(Ash, ld, r, order);
    for (int q = threadIdx.x; q < r; q += GT) sig[q] = Ash[order[q] * ld + order[q]];
    // Vout = W Y(:, order)
    CTA_FOR_2D(i, c, n, r) {
        int col = order[c];
        T s = 0;
        for (int l = 0; l < r; ++l) s += work1[i * r + l] * Vsh[l * ld + col];
        Vout[i * r + c] = s;
    }
    bar();
    return r;
}

// Householder QR with column pivoting of C (n x m, ld m, destroyed).  Returns
// the numerical rank k and writes Q (n x n, ld n): its first k columns span
// range(C), the rest its orthogonal complement.
template <class T>
__device__ int qr_basis(T* C, int n, int m, T* Q, T* vbuf /* n*n */, T* norms,
                        T* tau) {
    __shared__ int k_s, piv_s;
    __shared__ T n0_s, alpha_s;
    for (int q = threadIdx.x; q < n * n; q += GT) Q[q] = (q % (n + 1) == 0) ? (T)1 : (T)0;
    if (threadIdx.x == 0) k_s = 0;
    bar();
    int steps = min(n, m);
    for (int j = 0; j < steps; ++j) {
        // column norms of the trailing part
        for (int c = threadIdx.x; c < m; c += GT) {
            T s = 0.0;
            if (c >= j)
                for (int i = j; i < n; ++i) s += C[i * m + c] * C[i * m + c];
            norms[c] = s;
        }
        bar();
        if (threadIdx.x == 0) {
            T b = -1.0;
            int bi = j;
            for (int c = j; c < m; ++c)
                if (norms[c] > b) { b = norms[c]; bi = c; }
            piv_s = bi;
            T nb = sqrt(b > (T)0 ? b : (T)0);
            if (j == 0) n0_s = nb;
            alpha_s = nb;
        }
        bar();
        const T al = alpha_s, n0 = n0_s;
        const int p = piv_s;
        bar();
        if (!(al > (T)Tol<T>::rank * n0) || n0 == 0.0) break;
        if (p != j) {
            for (int i = threadIdx.x; i < n; i += GT) {
                T t = C[i * m + j]; C[i * m + j] = C[i * m + p]; C[i * m + p] = t;
            }
            bar();
        }
        // Householder vector for column j, rows j..n-1
        if (threadIdx.x == 0) {
            T x0 = C[j * m + j];
            T a = x0 >= 0 ? -al : al;       // reflect to a e_j
            T v0 = x0 - a;
            T vn2 = al * al - x0 * x0 + v0 * v0;
            tau[j] = vn2 > 0 ? 2.0 / vn2 : 0.0;
            vbuf[j * n + j] = v0;
        }
        bar();
        for (int i = j + 1 + threadIdx.x; i < n; i += GT) vbuf[j * n + i] = C[i * m + j];
        bar();
        // apply H = I - tau v v^T to columns j..m-1
        for (int c = j + threadIdx.x; c < m; c += GT) {
            T s = 0.0;
            for (int i = j; i < n; ++i) s += vbuf[j * n + i] * C[i * m + c];
            s *= tau[j];
            for (int i = j; i < n; ++i) C[i * m + c] -= s * vbuf[j * n + i];
        }
        bar();
        if (threadIdx.x == 0) k_s = j + 1;
        bar();
    }
    const int k = k_s;
    // Q = H_0 H_1 ... H_{k-1} I
    for (int j = k - 1; j >= 0; --j) {
        for (int c = threadIdx.x; c < n; c += GT) {
            T s = 0.0;
            for (int i = j; i < n; ++i) s += vbuf[j * n + i] * Q[i * n + c];
            s *= tau[j];
            for (int i = j; i < n; ++i) Q[i * n + c] -= s * vbuf[j * n + i];
        }
        bar();
    }
    return k;
}

// ------------------------------------------------------------------- face
// ash_global: the two eigen-work matrices (A, V of the Jacobi / tridiagonal steps)
// live in the job's global workspace after its face_work_doubles(n) elements
// instead of shared memory (faces too large for shared memory).
template <class T>
__global__ void __launch_bounds__(GT) k_face(const FaceJob* __restrict__ jobs, int* __restrict__ err,
                                             long long work_off, int ash_global) {
    const FaceJob J = jobs[blockIdx.x];
    const int n = J.n, np = (n + 1) & ~1;
    extern __shared__ __align__(16) unsigned char shm_raw[];
    T* shm = reinterpret_cast<T*>(shm_raw);
    const int ldj = np + 1;                    // odd row stride (no bank conflicts in shared memory)
    T* Ash = ash_global ? (T*)J.work + face_work_doubles(n) : shm;
    T* Vsh = Ash + np * ldj;
    __shared__ T cs[FACE_NMAX / 2], sn[FACE_NMAX / 2];
    __shared__ int pp[FACE_NMAX / 2], qq[FACE_NMAX / 2];
    __shared__ int order[FACE_NMAX];
    __shared__ unsigned char done[2 * FACE_NMAX];
    T* w = work_off >= 0 ? shm + work_off : (T*)J.work;   // workspace in shared memory when it fits
    const int nn = n * n;
    // Workspace of 8 n^2 elements (units of n^2), reused as the steps go:
    //   [0,2) Dij = [D^(i) | D^(j)] (kept to the end)   [2,3) B_F (kept)
    //   deluxe:      [3,4) S_FF^(i)  [4,5) S_FF^(j)  [5,6) their sum
    //   B_F:         [3,4) sym S^(i) [4,5) sym S^(j) [5,6) product scratch
    //   parallel sum [3,7) the 2n x 2n matrix        [7,8) B~_F (kept)
    //   pencil:      [3,4) [4,5) scratch  [5,6) eigenvectors
    //   basis:       [3,4) constraint vectors  [4,5) reflectors  [6,7) Q
    T *Dij = w, *BF = w + 2 * nn, *Bt = w + 7 * nn;
    T *Si = w + 3 * nn, *Sj = w + 4 * nn, *Ssum = w + 5 * nn;
    T *T1 = Si, *T2 = Sj, *W1 = w + 5 * nn;
    T* PS = w + 3 * nn;  // 4 nn
    T *P1 = w + 3 * nn, *P2 = w + 4 * nn, *V = w + 5 * nn;
    T *Cm = w + 3 * nn, *vb = w + 4 * nn, *Qo = w + 6 * nn;
    T* aux = w + 8 * nn;   // 3n
    // gather S_FF blocks
    CTA_FOR_2D(a, b, n, n) {
        Si[a * n + b] = J.Si[(long long)J.pi[a] * J.ldi + J.pi[b]];
        Sj[a * n + b] = J.Sj[(long long)J.pj[a] * J.ldj + J.pj[b]];
    }
    bar();
    for (int q = threadIdx.x; q < nn; q += GT) {
        Ssum[q] = Si[q] + Sj[q];
        int a = q / n, b = q % n;
        Dij[a * 2 * n + b] = Si[q];
        Dij[a * 2 * n + n + b] = Sj[q];
    }
    bar();
    lu_solve(Ssum, n, Dij, 2 * n, n, 2 * n, err);              // [D^(i) | D^(j)]
    // B_F = D_j^T B_FF^(i) D_j + D_i^T B_FF^(j) D_i   (B_FF = sym(S_FF), in place)
    symmetrize(T1, n, n);
    symmetrize(T2, n, n);
    const T* Di = Dij;
    const T* Dj = Dij + n;
    mm(T1, n, false, Dj, 2 * n, false, W1, n, n, n, n, (T)1, (T)0);
    mm(Dj, 2 * n, true, W1, n, false, BF, n, n, n, n, (T)1, (T)0);
    mm(T2, n, false, Di, 2 * n, false, W1, n, n, n, n, (T)1, (T)0);
    mm(Di, 2 * n, true, W1, n, false, BF, n, n, n, n, (T)1, (T)1);
    symmetrize(BF, n, n);
    // parallel sum B~_i : B~_j = B~_i - B~_i (B~_i + B~_j)^+ B~_i (the symmetric
    // parts of the two Schur complements, read from global memory)
    const int n2 = 2 * n;
    CTA_FOR_2D(a, b, n2, n2) {
        const int ra = a < n ? a : a - n, rb = b < n ? b : b - n;
        T v = (T)0.5 * ((T)J.Bti[(long long)ra * J.ldbi + rb] + (T)J.Bti[(long long)rb * J.ldbi + ra]);
        if (a >= n && b >= n)
            v += (T)0.5 * ((T)J.Btj[(long long)ra * J.ldbj + rb] + (T)J.Btj[(long long)rb * J.ldbj + ra]);
        PS[a * n2 + b] = v;        // order [B~_i, B~_i; B~_i, B~_i + B~_j]: eliminate the tail
    }
    bar();
    pinv_schur_tail(PS, n2, n2, n, done);
    copy_mat(PS, n2, Bt, n, n, n);
    symmetrize(Bt, n, n);
    int k = 0;
    T* T1o = Qo;                   // the constraint basis Q (identity when nothing is selected)
    if (J.mode == 0) {
        const T sth = (T)(J.theta / (1.0 + J.theta) - Tol<T>::slack);
        int r = sigma_pencil(BF, Bt, n, Ash, Vsh, np, ldj, P1, P2, aux, V, cs, sn, pp, qq, order, err, err + 1, sth);
        __shared__ int nsel_s;
        if (threadIdx.x == 0) {
            int c = 0;
            for (int q = 0; q < r; ++q) {
                T sg = aux[q];
                J.lambda[q] = (1.0 - (double)sg <= Tol<T>::slack) ? INFINITY : (double)sg / (1.0 - (double)sg);
                if (sg >= sth) ++c;
            }
            for (int q = r; q < n; ++q) J.lambda[q] = NAN;
            *J.neig = r;
            nsel_s = c;
        }
        bar();
        const int s = nsel_s;
        if (s > 0) {
            // Cm = B_F V(:, 0..s)   (n x s)
            mm(BF, n, false, V, r, false, Cm, s, n, s, n, (T)1, (T)0);
            k = qr_basis(Cm, n, s, T1o, vb, aux + n, aux + 2 * n);
        } else {
            for (int q = threadIdx.x; q < nn; q += GT) T1o[q] = (q % (n + 1) == 0) ? (T)1 : (T)0;
            bar();
        }
    } else {
        for (int q = threadIdx.x; q < nn; q += GT) T1o[q] = (q % (n + 1) == 0) ? (T)1 : (T)0;
        if (threadIdx.x == 0) *J.neig = 0;
        bar();
        k = J.mode == 1 ? n : 0;
    }
    // outputs: Q (row-major n x n), D^(i) Q, D^(j) Q
    for (int q = threadIdx.x; q < nn; q += GT) J.Q[q] = T1o[q];
    mm(Di, 2 * n, false, T1o, n, false, J.DQi, n, n, n, n, (T)1, (T)0);
    mm(Dj, 2 * n, false, T1o, n, false, J.DQj, n, n, n, n, (T)1, (T)0);
    if (threadIdx.x == 0) *J.k = k;
}

// ------------------------------------------------------------------- edge
template <class T>
__global__ void __launch_bounds__(GT) k_edge(const EdgeJob* __restrict__ jobs, int* __restrict__ err,
                                             long long work_off) {
    const EdgeJob J = jobs[blockIdx.x];
    const int n = J.n, m = J.m, nw = (m - 1) * n, mn = m * n;
    const int nz = mn + J.nH;
    const int np = (nw + 1) & ~1;
    extern __shared__ __align__(16) unsigned char shm_raw[];
    T* shm = reinterpret_cast<T*>(shm_raw);
    T* Ash = shm;
    const int ldj = np + 1;                    // odd shared-memory row stride
    T* Vsh = shm + np * ldj;
    __shared__ T cs[64], sn[64];
    __shared__ int pp[64], qq[64];
    __shared__ int order[128];
    __shared__ unsigned char done[1024];
    T* w = work_off >= 0 ? shm + work_off : (T*)J.work;   // workspace in shared memory when it fits
    const int nn = n * n;
    T* Ssum = w;                     // n x n
    T* Dall = Ssum + nn;             // n x (m n): [D^(k_1) ... D^(k_m)]
    T* Tk = Dall + n * mn;           // m blocks of n x (m n)
    T* BE = Tk + m * n * mn;         // m blocks n x n (sym S_EE)
    T* ME = BE + m * nn;             // nw x nw
    T* T1 = ME + nw * nw;            // scratch  (max(n x mn, nz x nz))
    T* Bt = T1 + (size_t)nz * nz;    // nz x nz
    T* BB = Bt + (size_t)nz * nz;    // nw x nw
    T* W1 = BB + nw * nw;            // nw x nw
    T* W2 = W1 + nw * nw;
    T* V = W2 + nw * nw;
    T* Cm = V + nw * nw;             // n x (m-1) nw
    T* vb = Cm + n * nw * (m - 1) + nw;
    T* Qo = vb + nn;
    T* aux = Qo + nn;                // sigma (nw), QR norms ((m-1) nw), tau (n)
    // deluxe scaling D^(k) = (sum_l S_EE^(l))^{-1} S_EE^(k)
    CTA_FOR_2D(a, b, n, n) {
        T s = 0.0;
        for (int t = 0; t < m; ++t) {
            T v = J.S[t][(long long)J.pos[t][a] * J.ldS[t] + J.pos[t][b]];
            s += v;
            Dall[a * mn + t * n + b] = v;
        }
        Ssum[a * n + b] = s;
    }
    bar();
    for (int q = threadIdx.x; q < m * nn; q += GT) {
        int t = q / nn, a = (q % nn) / n, b = q % n;
        const double* St = J.S[t];
        T v1 = St[(long long)J.pos[t][a] * J.ldS[t] + J.pos[t][b]];
        T v2 = St[(long long)J.pos[t][b] * J.ldS[t] + J.pos[t][a]];
        BE[q] = (T)0.5 * (v1 + v2);
    }
    bar();
    lu_solve(Ssum, n, Dall, mn, n, mn, err);
    // T^(k): block l (l = 1..m-1, subdomain k_l): (I - D^(k_l)) when k == k_l else -D^(k_l); last block I
    for (int q = threadIdx.x; q < m * n * mn; q += GT) {
        int t = q / (n * mn), a = (q % (n * mn)) / mn, col = q % mn;
        int blk = col / n, b = col % n;
        T v;
        if (blk == m - 1) v = (a == b) ? 1.0 : 0.0;
        else {
            int l = blk + 1;
            v = -Dall[a * mn + l * n + b];
            if (t == l && a == b) v += 1.0;
        }
        Tk[q] = v;
    }
    bar();
    // M_E = sum_k Tbar_k^T B_E^(k) Tbar_k
    for (int q = threadIdx.x; q < nw * nw; q += GT) ME[q] = 0.0;
    bar();
    for (int t = 0; t < m; ++t) {
        mm(BE + t * nn, n, false, Tk + t * n * mn, mn, false, T1, nw, n, nw, n, (T)1, (T)0);
        mm(Tk + t * n * mn, mn, true, T1, nw, false, ME, nw, nw, nw, n, (T)1, (T)1);
    }
    symmetrize(ME, nw, nw);
    if (J.mode == 0) {
    // B~_E = sum_k J_k^T B~^(k) J_k  (z = [w_check (nw), w^_E (n), w^_H (nH)])
    for (int q = threadIdx.x; q < nz * nz; q += GT) Bt[q] = 0.0;
    bar();
    for (int t = 0; t < m; ++t) {
        const T* G = (const T*)J.Bt[t];
        const int ldg = J.ldBt[t];
        const int h = J.h[t];
        const int* hm = J.hmap[t];
        const T* Tm = Tk + t * n * mn;
        // EE: T^T G_EE T  ->  Bt[0:mn, 0:mn]
        for (int q = threadIdx.x; q < n * mn; q += GT) {        // T1 = G_EE T  (n x mn)
            int a = q / mn, c = q % mn;
            T s = 0.0;
            for (int l = 0; l < n; ++l) s += G[a * ldg + l] * Tm[l * mn + c];
            T1[q] = s;
        }
        bar();
        CTA_FOR_2D(a, c, mn, mn) {
            T s = 0.0;
            for (int l = 0; l < n; ++l) s += Tm[l * mn + a] * T1[l * mn + c];
            Bt[a * nz + c] += s;
        }
        bar();
        // EH and HE: T^T G_EH
        CTA_FOR_2D(a, u, mn, h) {
            T s = 0.0;
            for (int l = 0; l < n; ++l) s += Tm[l * mn + a] * G[l * ldg + n + u];
            Bt[a * nz + mn + hm[u]] += s;
            T s2 = 0.0;
            for (int l = 0; l < n; ++l) s2 += G[(n + u) * ldg + l] * Tm[l * mn + a];
            Bt[(mn + hm[u]) * nz + a] += s2;
        }
        bar();
        CTA_FOR_2D(u, v, h, h) {
            Bt[(mn + hm[u]) * nz + mn + hm[v]] += G[(n + u) * ldg + n + v];
        }
        bar();
    }
    symmetrize(Bt, nz, nz);
    // B~~_E: eliminate (w^_E, w^_H) with the pseudo-inverse
    pinv_schur_tail(Bt, nz, nz, nw, done);
    copy_mat(Bt, nz, BB, nw, nw, nw);
    symmetrize(BB, nw, nw);
    for (int q = threadIdx.x; q < nw * nw; q += GT) J.BBout[q] = BB[q];
    bar();
    }
    int k = 0;
    for (int q = threadIdx.x; q < nn; q += GT) Qo[q] = (q % (n + 1) == 0) ? (T)1 : (T)0;
    bar();
    if (J.mode == 3) {
        // conventional edge GEP (Sect. 3, eq. equ-4-8-E):
        //   B_E = sum_i sum_{k != i} D^(k)T B_E^(i) D^(k),  B~_E = B~_E^(1) : ... : B~_E^(m),
        // B~_E^(k) the Schur complement of B^(k) onto E alone: the [E, H_k] complement
        // with H_k eliminated in turn (symmetric pivoting; B^(k)_HH is definite).
        T* BEo = BB;                   // n x n
        T* P = ME;                     // running parallel sum, n x n
        T* At = Cm;                    // n x n
        for (int q = threadIdx.x; q < nn; q += GT) BEo[q] = 0.0;
        bar();
        for (int i = 0; i < m; ++i)
            for (int t = 0; t < m; ++t) {
                if (t == i) continue;
                mm(BE + i * nn, n, false, Dall + t * n, mn, false, W1, n, n, n, n, (T)1, (T)0);
                mm(Dall + t * n, mn, true, W1, n, false, BEo, n, n, n, n, (T)1, (T)1);
            }
        symmetrize(BEo, n, n);
        const int n2 = 2 * n;
        for (int t = 0; t < m; ++t) {
            const int g = n + J.h[t];
            copy_mat((const T*)J.Bt[t], J.ldBt[t], T1, g, g, g);
            symmetrize(T1, g, g);
            pinv_schur_tail(T1, g, g, n, done);
            copy_mat(T1, g, t == 0 ? P : At, n, n, n);
            if (t == 0) {
                symmetrize(P, n, n);
                continue;
            }
            // P : A = P - P (P + A)^+ P: eliminate the tail of [[P, P], [P, P + A]]
            CTA_FOR_2D(a, b, n2, n2) {
                const int ra = a < n ? a : a - n, rb = b < n ? b : b - n;
                T v = P[ra * n + rb];
                if (a >= n && b >= n) v += At[ra * n + rb];
                Bt[a * n2 + b] = v;
            }
            bar();
            pinv_schur_tail(Bt, n2, n2, n, done);
            copy_mat(Bt, n2, P, n, n, n);
            symmetrize(P, n, n);
        }
        const int npn = (n + 1) & ~1;
        const T sth = (T)(J.theta / (1.0 + J.theta) - Tol<T>::slack);
        int r = sigma_pencil(BEo, P, n, Ash, Vsh, npn, npn + 1, W1, W2, aux, V, cs, sn, pp, qq, order, err, err + 1,
                             sth);
        __shared__ int nsel_o;
        if (threadIdx.x == 0) {
            int c = 0;
            for (int q = 0; q < r; ++q) {
                T sg = aux[q];
                J.lambda[q] = (1.0 - (double)sg <= Tol<T>::slack) ? INFINITY : (double)sg / (1.0 - (double)sg);
                if (sg >= sth) ++c;
            }
            for (int q = r; q < nw; ++q) J.lambda[q] = NAN;
            *J.neig = r;
            nsel_o = c;
        }
        bar();
        const int so = nsel_o;
        if (so > 0) {
            mm(BEo, n, false, V, r, false, Cm, so, n, so, n, (T)1, (T)0);     // B_E V(:, 0..so)
            k = qr_basis(Cm, n, so, Qo, vb, aux + nw, aux + nw + (m - 1) * nw);
        }
    } else if (J.mode == 0) {
        const T sth = (T)(J.theta / (1.0 + J.theta) - Tol<T>::slack);
        int r = sigma_pencil(ME, BB, nw, Ash, Vsh, np, ldj, W1, W2, aux, V, cs, sn, pp, qq, order, err, err + 1, sth);
        __shared__ int nsel_s;
        if (threadIdx.x == 0) {
            int c = 0;
            for (int q = 0; q < r; ++q) {
                T sg = aux[q];
                J.lambda[q] = (1.0 - (double)sg <= Tol<T>::slack) ? INFINITY : (double)sg / (1.0 - (double)sg);
                if (sg >= sth) ++c;
            }
            for (int q = r; q < nw; ++q) J.lambda[q] = NAN;
            *J.neig = r;
            nsel_s = c;
        }
        bar();
        const int s = nsel_s;
        if (s > 0) {
            // c_l = M_E v_l (nw); Cm columns = its n-blocks: col (l * (m-1) + b)
            const int nc = s * (m - 1);
            CTA_FOR_2D(a, cidx, n, nc) {
                int l = cidx / (m - 1), b = cidx % (m - 1);
                int row = b * n + a;
                T acc = 0.0;
                for (int t = 0; t < nw; ++t) acc += ME[row * nw + t] * V[t * r + l];
                Cm[a * nc + cidx] = acc;
            }
            bar();
            k = qr_basis(Cm, n, nc, Qo, vb, aux + nw, aux + nw + (m - 1) * nw);
        }
    } else {
        if (threadIdx.x == 0) *J.neig = 0;
        k = J.mode == 1 ? n : 0;
    }
    for (int q = threadIdx.x; q < nn; q += GT) J.Q[q] = Qo[q];
    bar();
    for (int t = 0; t < m; ++t)
        mm(Dall + t * n, mn, false, Qo, n, false, J.DQ[t], n, n, n, n, (T)1, (T)0);
    if (threadIdx.x == 0) *J.k = k;
}

}  // namespace

__host__ __device__ size_t face_work_doubles(int n) { return (size_t)8 * n * n + 3 * n + 64; }
size_t face_eig_doubles(int n) {
    const size_t np = (size_t)((n + 1) & ~1);
    return 2 * np * (np + 1);
}
size_t edge_work_doubles(int n, int m, int nH) {
    size_t nw = (size_t)(m - 1) * n, mn = (size_t)m * n, nz = mn + nH;
    return (size_t)n * n * (3 + m) + (size_t)n * mn * (1 + m) + 6 * nw * nw + 2 * nz * nz +
           (size_t)n * nw * (m - 1) + nw + (size_t)m * nw + n + 64;
}

// Dynamic shared memory of a GEP launch: the Jacobi pair (base bytes) and, when
// the device allows it, the per-job workspace too (returned offset in elements;
// -1 keeps the workspace in the jobs' global buffers).
template <class T>
static int gep_smem(const void* fn, size_t base, size_t work_elems, size_t* smem, long long* off) {
    cudaFuncAttributes fa;
    BDDC_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
    int dev = 0, optin = 0;
    BDDC_CUDA_TRY(cudaGetDevice(&dev));
    BDDC_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t want = base + work_elems * sizeof(T);
    if (fa.sharedSizeBytes + want <= (size_t)optin) {
        *smem = want;
        *off = (long long)(base / sizeof(T));
    } else {
        *smem = base;
        *off = -1;
    }
    return BDDC_OK;
}

template <class T>
bool face_eig_global(int maxn) {
    return (size_t)face_eig_doubles(maxn) * sizeof(T) > 160 * 1024;
}
template bool face_eig_global<double>(int);
template bool face_eig_global<float>(int);

template <class T>
int face_run(const FaceJob* jobs_dev, int count, int maxn, int* err, cudaStream_t st) {
    if (count <= 0) return BDDC_OK;
    if (maxn > FACE_NMAX) {
        bddc_set_last_error("a face has more dofs than the face GEP kernel handles (256)", __FILE__, __LINE__);
        return BDDC_EINVAL;
    }
    // the eigen-work matrices in shared memory when they fit, else in each job's
    // workspace (allocated with face_eig_doubles(n) more elements by the caller)
    const int glob = face_eig_global<T>(maxn) ? 1 : 0;
    const size_t base = glob ? 0 : face_eig_doubles(maxn) * sizeof(T);
    size_t smem = 0;
    long long off = -1;
    BDDC_TRY(gep_smem<T>((const void*)k_face<T>, base, face_work_doubles(maxn), &smem, &off));
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_face<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_face<T><<<count, GT, smem, st>>>(jobs_dev, err, off, glob);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

template <class T>
int edge_run(const EdgeJob* jobs_dev, int count, int maxnw, int maxnz, size_t max_work, int* err, cudaStream_t st) {
    if (count <= 0) return BDDC_OK;
    int np = (maxnw + 1) & ~1;
    const size_t base = (size_t)2 * np * (np + 1) * sizeof(T);
    if (np > 128 || base > 200 * 1024 || maxnz > 1024) {
        bddc_set_last_error("an edge GEP larger than the edge kernel handles ((m-1) n_E <= 128, n_z <= 1024)",
                            __FILE__, __LINE__);
        return BDDC_EINVAL;
    }
    size_t smem = 0;
    long long off = -1;
    BDDC_TRY(gep_smem<T>((const void*)k_edge<T>, base, max_work, &smem, &off));
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_edge<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_edge<T><<<count, GT, smem, st>>>(jobs_dev, err, off);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

template int face_run<double>(const FaceJob*, int, int, int*, cudaStream_t);
template int face_run<float>(const FaceJob*, int, int, int*, cudaStream_t);
template int edge_run<double>(const EdgeJob*, int, int, int, size_t, int*, cudaStream_t);
template int edge_run<float>(const EdgeJob*, int, int, int, size_t, int*, cudaStream_t);
