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

constexpr int GT = 256;                 // threads per GEP CTA
constexpr double EIG_DROP = 1e-12;
constexpr double RANK_TOL = 1e-10;
constexpr int JACOBI_MAX_SWEEPS = 60;

__device__ __forceinline__ void bar() { __syncthreads(); }

// C = alpha * op(A) * op(B) + beta * C ; row-major; transA/transB flags
__device__ void mm(const double* A, int lda, bool ta, const double* B, int ldb, bool tb, double* C,
                   int ldc, int m, int n, int k, double alpha, double beta) {
    for (int q = threadIdx.x; q < m * n; q += GT) {
        int i = q / n, j = q % n;
        double s = 0.0;
        for (int l = 0; l < k; ++l) {
            double a = ta ? A[l * lda + i] : A[i * lda + l];
            double b = tb ? B[j * ldb + l] : B[l * ldb + j];
            s += a * b;
        }
        C[i * ldc + j] = alpha * s + (beta == 0.0 ? 0.0 : beta * C[i * ldc + j]);
    }
    bar();
}

__device__ void copy_mat(const double* A, int lda, double* B, int ldb, int m, int n) {
    for (int q = threadIdx.x; q < m * n; q += GT) B[(q / n) * ldb + q % n] = A[(q / n) * lda + q % n];
    bar();
}

__device__ void symmetrize(double* A, int ld, int n) {
    for (int q = threadIdx.x; q < n * n; q += GT) {
        int i = q / n, j = q % n;
        if (i < j) {
            double v = 0.5 * (A[i * ld + j] + A[j * ld + i]);
            A[i * ld + j] = v;
            A[j * ld + i] = v;
        }
    }
    bar();
}

// Solve A X = B in place (A n x n overwritten by its LU, B n x nr overwritten by X);
// Gaussian elimination with partial pivoting.
__device__ void lu_solve(double* A, int lda, double* B, int ldb, int n, int nr, int* err) {
    __shared__ int piv_s;
    __shared__ double pv_s[32];
    __shared__ int pi_s[32];
    for (int c = 0; c < n; ++c) {
        // pivot search by warp 0
        if (threadIdx.x < 32) {
            double best = -1.0;
            int bi = c;
            for (int r = c + threadIdx.x; r < n; r += 32) {
                double v = fabs(A[r * lda + c]);
                if (v > best) { best = v; bi = r; }
            }
            pv_s[threadIdx.x] = best;
            pi_s[threadIdx.x] = bi;
            __syncwarp();
            if (threadIdx.x == 0) {
                double b = -1.0;
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
                double t = A[c * lda + q]; A[c * lda + q] = A[p * lda + q]; A[p * lda + q] = t;
            }
            for (int q = threadIdx.x; q < nr; q += GT) {
                double t = B[c * ldb + q]; B[c * ldb + q] = B[p * ldb + q]; B[p * ldb + q] = t;
            }
        }
        bar();
        double d = A[c * lda + c];
        if (d == 0.0) d = 1e-300;
        for (int r = c + 1 + threadIdx.x; r < n; r += GT) A[r * lda + c] /= d;
        bar();
        const int rem = n - c - 1;
        for (int q = threadIdx.x; q < rem * (rem + nr); q += GT) {
            int r = c + 1 + q / (rem + nr), j = q % (rem + nr);
            double l = A[r * lda + c];
            if (j < rem) A[r * lda + c + 1 + j] -= l * A[c * lda + c + 1 + j];
            else B[r * ldb + (j - rem)] -= l * B[c * ldb + (j - rem)];
        }
        bar();
    }
    // back substitution, column-parallel over the right-hand sides
    for (int c = n - 1; c >= 0; --c) {
        double d = A[c * lda + c];
        if (d == 0.0) d = 1e-300;
        for (int q = threadIdx.x; q < nr; q += GT) B[c * ldb + q] /= d;
        bar();
        for (int q = threadIdx.x; q < c * nr; q += GT) {
            int r = q / nr, j = q % nr;
            B[r * ldb + j] -= A[r * lda + c] * B[c * ldb + j];
        }
        bar();
    }
}

// Generalised Schur complement of a symmetric PSD matrix: eliminate the
// indices [r0, n) by symmetric diagonal pivoting; pivots <= tol * (largest
// initial diagonal among them) are left (their directions carry no energy).
// The leading r0 x r0 block then holds M_ww - M_wr M_rr^+ M_rw.
__device__ void pinv_schur_tail(double* M, int ld, int n, int r0, unsigned char* done) {
    __shared__ double dmax0_s, best_s;
    __shared__ int bi_s;
    for (int q = threadIdx.x; q < n; q += GT) done[q] = q < r0 ? 1 : 0;
    if (threadIdx.x == 0) {
        double d = 0.0;
        for (int q = r0; q < n; ++q) d = fmax(d, M[q * ld + q]);
        dmax0_s = d;
    }
    bar();
    const double tol = EIG_DROP * dmax0_s;
    for (int step = r0; step < n; ++step) {
        if (threadIdx.x == 0) {
            double b = -1.0;
            int bi = -1;
            for (int q = r0; q < n; ++q)
                if (!done[q] && M[q * ld + q] > b) { b = M[q * ld + q]; bi = q; }
            best_s = b;
            bi_s = bi;
        }
        bar();
        if (bi_s < 0 || !(best_s > tol)) break;
        const int p = bi_s;
        const double dp = M[p * ld + p];
        // update all not-yet-eliminated rows/cols (including the kept block)
        for (int q = threadIdx.x; q < n * n; q += GT) {
            int i = q / n, j = q % n;
            if (i == p || j == p) continue;
            if ((i >= r0 && done[i]) || (j >= r0 && done[j])) continue;
            M[i * ld + j] -= M[i * ld + p] * M[p * ld + j] / dp;
        }
        bar();
        if (threadIdx.x == 0) done[p] = 1;
        bar();
    }
}

// Cyclic parallel Jacobi on a symmetric n x n matrix held in shared memory
// (ld = np = n rounded up to even).  On exit diag(A) = eigenvalues, V = eigenvectors.
__device__ void jacobi(double* A, double* V, int n, int np, double* cs, double* sn, int* pp, int* qq,
                       int* err) {
    const int ld = np;
    for (int q = threadIdx.x; q < np * np; q += GT) {
        int i = q / np, j = q % np;
        V[q] = i == j ? 1.0 : 0.0;
        if (i >= n || j >= n) A[i * ld + j] = 0.0;
    }
    bar();
    __shared__ double off_s, tot_s;
    const int half = np / 2;
    for (int sweep = 0; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
        if (threadIdx.x == 0) {
            double off = 0.0, tot = 0.0;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    double v = A[i * ld + j] * A[i * ld + j];
                    tot += v;
                    if (i != j) off += v;
                }
            off_s = off;
            tot_s = tot;
        }
        bar();
        if (off_s <= 1e-26 * tot_s || tot_s == 0.0) return;
        if (sweep == JACOBI_MAX_SWEEPS - 1) {
            if (threadIdx.x == 0) atomicOr(err, ERR_JACOBI);
            return;
        }
        for (int r = 0; r < np - 1; ++r) {
            for (int k = threadIdx.x; k < half; k += GT) {
                int p = (r + k) % (np - 1);
                int q = k == 0 ? np - 1 : (r - k + np - 1) % (np - 1);
                if (p > q) { int t = p; p = q; q = t; }
                pp[k] = p;
                qq[k] = q;
                double c = 1.0, s = 0.0;
                double apq = A[p * ld + q];
                if (q < n && fabs(apq) > 1e-300) {
                    double app = A[p * ld + p], aqq = A[q * ld + q];
                    double th = (aqq - app) / (2.0 * apq);
                    double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
                cs[k] = c;
                sn[k] = s;
            }
            bar();
            for (int q = threadIdx.x; q < half * np; q += GT) {       // rows p, q
                int k = q / np, col = q % np;
                int p = pp[k], qi = qq[k];
                double c = cs[k], s = sn[k];
                double a = A[p * ld + col], b = A[qi * ld + col];
                A[p * ld + col] = c * a - s * b;
                A[qi * ld + col] = s * a + c * b;
            }
            bar();
            for (int q = threadIdx.x; q < half * np; q += GT) {       // columns p, q
                int k = q / np, row = q % np;
                int p = pp[k], qi = qq[k];
                double c = cs[k], s = sn[k];
                double a = A[row * ld + p], b = A[row * ld + qi];
                A[row * ld + p] = c * a - s * b;
                A[row * ld + qi] = s * a + c * b;
                double va = V[row * ld + p], vb = V[row * ld + qi];
                V[row * ld + p] = c * va - s * vb;
                V[row * ld + qi] = s * va + c * vb;
            }
            bar();
            for (int k = threadIdx.x; k < half; k += GT) {          // the rotated pair is zero
                if (sn[k] != 0.0) {
                    A[pp[k] * ld + qq[k]] = 0.0;
                    A[qq[k] * ld + pp[k]] = 0.0;
                }
            }
            bar();
        }
    }
}

// Sort (val, vec columns) by decreasing value (n small; thread 0 computes the order).
__device__ void sort_desc(const double* A, int ld, int n, int* order) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) order[i] = i;
        for (int i = 1; i < n; ++i) {
            int v = order[i];
            double key = A[v * ld + v];
            int j = i - 1;
            while (j >= 0 && A[order[j] * ld + order[j]] < key) { order[j + 1] = order[j]; --j; }
            order[j + 1] = v;
        }
    }
    bar();
}

// Solve X v = sigma (X + Y) v for symmetric PSD X, Y (n x n in global scratch).
// On exit: sig[0..r) decreasing, Vout (n x r, ld n) = eigenvectors, r returned.
__device__ int sigma_pencil(const double* X, const double* Y, int n, double* Ash, double* Vsh, int np,
                            double* work1, double* work2, double* sig, double* Vout, double* cs,
                            double* sn, int* pp, int* qq, int* order, int* err) {
    __shared__ int r_s;
    __shared__ double kmax_s;
    for (int q = threadIdx.x; q < n * n; q += GT) {
        int i = q / n, j = q % n;
        Ash[i * np + j] = 0.5 * (X[i * n + j] + X[j * n + i]) + 0.5 * (Y[i * n + j] + Y[j * n + i]);
    }
    bar();
    jacobi(Ash, Vsh, n, np, cs, sn, pp, qq, err);
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < n; ++i) m = fmax(m, Ash[i * np + i]);
        kmax_s = m;
        int r = 0;
        for (int i = 0; i < n; ++i)
            if (m > 0.0 && Ash[i * np + i] > EIG_DROP * m) order[r++] = i;
        r_s = r;
    }
    bar();
    const int r = r_s;
    if (r == 0) return 0;
    // W = U_keep / sqrt(kappa)  (n x r) -> work1
    for (int q = threadIdx.x; q < n * r; q += GT) {
        int i = q / r, c = q % r;
        int col = order[c];
        work1[i * r + c] = Vsh[i * np + col] / sqrt(Ash[col * np + col]);
    }
    bar();
    // C = W^T X W -> shared A (r x r)
    mm(X, n, false, work1, r, false, work2, r, n, r, n, 1.0, 0.0);        // X W  (n x r)
    for (int q = threadIdx.x; q < np * np; q += GT) Ash[q] = 0.0;
    bar();
    mm(work1, r, true, work2, r, false, Ash, np, r, r, n, 1.0, 0.0);     // W^T (X W)
    // symmetrize in shared
    for (int q = threadIdx.x; q < r * r; q += GT) {
        int i = q / r, j = q % r;
        if (i < j) {
            double v = 0.5 * (Ash[i * np + j] + Ash[j * np + i]);
            Ash[i * np + j] = v;
            Ash[j * np + i] = v;
        }
    }
    bar();
    const int rp = (r + 1) & ~1;
    // repack to ld rp for the second Jacobi (in place is unsafe: copy through work2)
    for (int q = threadIdx.x; q < r * r; q += GT) work2[q] = Ash[(q / r) * np + q % r];
    bar();
    for (int q = threadIdx.x; q < rp * rp; q += GT) {
        int i = q / rp, j = q % rp;
        Ash[q] = (i < r && j < r) ? work2[i * r + j] : 0.0;
    }
    bar();
    jacobi(Ash, Vsh, r, rp, cs, sn, pp, qq, err);
    sort_desc(Ash, rp, r, order);
    for (int q = threadIdx.x; q < r; q += GT) sig[q] = Ash[order[q] * rp + order[q]];
    // Vout = W Y(:, order)
    for (int q = threadIdx.x; q < n * r; q += GT) {
        int i = q / r, c = q % r;
        int col = order[c];
        double s = 0.0;
        for (int l = 0; l < r; ++l) s += work1[i * r + l] * Vsh[l * rp + col];
        Vout[i * r + c] = s;
    }
    bar();
    return r;
}

// Householder QR with column pivoting of C (n x m, ld m, destroyed).  Returns
// the numerical rank k and writes Q (n x n, ld n): its first k columns span
// range(C), the rest its orthogonal complement.
__device__ int qr_basis(double* C, int n, int m, double* Q, double* vbuf /* n*n */, double* norms,
                        double* tau) {
    __shared__ int k_s, piv_s;
    __shared__ double n0_s, alpha_s;
    for (int q = threadIdx.x; q < n * n; q += GT) Q[q] = (q / n == q % n) ? 1.0 : 0.0;
    if (threadIdx.x == 0) k_s = 0;
    bar();
    int steps = min(n, m);
    for (int j = 0; j < steps; ++j) {
        // column norms of the trailing part
        for (int c = threadIdx.x; c < m; c += GT) {
            double s = 0.0;
            if (c >= j)
                for (int i = j; i < n; ++i) s += C[i * m + c] * C[i * m + c];
            norms[c] = s;
        }
        bar();
        if (threadIdx.x == 0) {
            double b = -1.0;
            int bi = j;
            for (int c = j; c < m; ++c)
                if (norms[c] > b) { b = norms[c]; bi = c; }
            piv_s = bi;
            double nb = sqrt(fmax(b, 0.0));
            if (j == 0) n0_s = nb;
            alpha_s = nb;
        }
        bar();
        const double al = alpha_s, n0 = n0_s;
        const int p = piv_s;
        bar();
        if (!(al > RANK_TOL * n0) || n0 == 0.0) break;
        if (p != j) {
            for (int i = threadIdx.x; i < n; i += GT) {
                double t = C[i * m + j]; C[i * m + j] = C[i * m + p]; C[i * m + p] = t;
            }
            bar();
        }
        // Householder vector for column j, rows j..n-1
        if (threadIdx.x == 0) {
            double x0 = C[j * m + j];
            double a = x0 >= 0 ? -al : al;       // reflect to a e_j
            double v0 = x0 - a;
            double vn2 = al * al - x0 * x0 + v0 * v0;
            tau[j] = vn2 > 0 ? 2.0 / vn2 : 0.0;
            vbuf[j * n + j] = v0;
        }
        bar();
        for (int i = j + 1 + threadIdx.x; i < n; i += GT) vbuf[j * n + i] = C[i * m + j];
        bar();
        // apply H = I - tau v v^T to columns j..m-1
        for (int c = j + threadIdx.x; c < m; c += GT) {
            double s = 0.0;
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
            double s = 0.0;
            for (int i = j; i < n; ++i) s += vbuf[j * n + i] * Q[i * n + c];
            s *= tau[j];
            for (int i = j; i < n; ++i) Q[i * n + c] -= s * vbuf[j * n + i];
        }
        bar();
    }
    return k;
}

// ------------------------------------------------------------------- face
__global__ void __launch_bounds__(GT) k_face(const FaceJob* __restrict__ jobs, int* __restrict__ err) {
    const FaceJob J = jobs[blockIdx.x];
    const int n = J.n, np = (n + 1) & ~1;
    extern __shared__ double shm[];
    double* Ash = shm;
    double* Vsh = shm + np * np;
    __shared__ double cs[64], sn[64];
    __shared__ int pp[64], qq[64];
    __shared__ int order[128];
    __shared__ unsigned char done[256];
    double* w = J.work;
    const int nn = n * n;
    double *Si = w, *Sj = w + nn, *Ssum = w + 2 * nn, *Dij = w + 3 * nn /* n x 2n */;
    double *BF = w + 5 * nn, *Bti = w + 6 * nn, *Btj = w + 7 * nn, *Bt = w + 8 * nn;
    double *T1 = w + 9 * nn, *T2 = w + 10 * nn, *V = w + 11 * nn, *W1 = w + 12 * nn,
           *W2 = w + 13 * nn, *Cm = w + 14 * nn, *vb = w + 15 * nn, *PS = w + 16 * nn /* 4 nn */;
    double* aux = w + 20 * nn;   // 3n
    // gather S_FF blocks
    for (int q = threadIdx.x; q < nn; q += GT) {
        int a = q / n, b = q % n;
        Si[q] = J.Si[(long long)J.pi[a] * J.ldi + J.pi[b]];
        Sj[q] = J.Sj[(long long)J.pj[a] * J.ldj + J.pj[b]];
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
    // B_F = D_j^T B_FF^(i) D_j + D_i^T B_FF^(j) D_i   (B_FF = sym(S_FF))
    for (int q = threadIdx.x; q < nn; q += GT) {
        int a = q / n, b = q % n;
        T1[q] = 0.5 * (Si[a * n + b] + Si[b * n + a]);
        T2[q] = 0.5 * (Sj[a * n + b] + Sj[b * n + a]);
    }
    bar();
    const double* Di = Dij;
    const double* Dj = Dij + n;
    mm(T1, n, false, Dj, 2 * n, false, W1, n, n, n, n, 1.0, 0.0);
    mm(Dj, 2 * n, true, W1, n, false, BF, n, n, n, n, 1.0, 0.0);
    mm(T2, n, false, Di, 2 * n, false, W1, n, n, n, n, 1.0, 0.0);
    mm(Di, 2 * n, true, W1, n, false, BF, n, n, n, n, 1.0, 1.0);
    symmetrize(BF, n, n);
    // parallel sum B~_i : B~_j = B~_i - B~_i (B~_i + B~_j)^+ B~_i
    copy_mat(J.Bti, J.ldbi, Bti, n, n, n);
    copy_mat(J.Btj, J.ldbj, Btj, n, n, n);
    symmetrize(Bti, n, n);
    symmetrize(Btj, n, n);
    const int n2 = 2 * n;
    for (int q = threadIdx.x; q < n2 * n2; q += GT) {
        int a = q / n2, b = q % n2;
        double v;
        if (a < n && b < n) v = Bti[a * n + b];
        else if (a < n) v = Bti[a * n + b - n];
        else if (b < n) v = Bti[(a - n) * n + b];
        else v = Bti[(a - n) * n + b - n] + Btj[(a - n) * n + b - n];
        PS[q] = v;        // order [B~_i, B~_i; B~_i, B~_i + B~_j]: eliminate the tail
    }
    bar();
    pinv_schur_tail(PS, n2, n2, n, done);
    copy_mat(PS, n2, Bt, n, n, n);
    symmetrize(Bt, n, n);
    int k = 0;
    if (J.mode == 0) {
        int r = sigma_pencil(BF, Bt, n, Ash, Vsh, np, W1, W2, aux, V, cs, sn, pp, qq, order, err);
        const double sth = J.theta / (1.0 + J.theta) - 1e-12;
        __shared__ int nsel_s;
        if (threadIdx.x == 0) {
            int c = 0;
            for (int q = 0; q < r; ++q) {
                double sg = aux[q];
                J.lambda[q] = (1.0 - sg <= 1e-12) ? INFINITY : sg / (1.0 - sg);
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
            mm(BF, n, false, V, r, false, Cm, s, n, s, n, 1.0, 0.0);
            k = qr_basis(Cm, n, s, T1, vb, aux + n, aux + 2 * n);
        } else {
            for (int q = threadIdx.x; q < nn; q += GT) T1[q] = (q / n == q % n) ? 1.0 : 0.0;
            bar();
        }
    } else {
        for (int q = threadIdx.x; q < nn; q += GT) T1[q] = (q / n == q % n) ? 1.0 : 0.0;
        if (threadIdx.x == 0) *J.neig = 0;
        bar();
        k = J.mode == 1 ? n : 0;
    }
    // outputs: Q (row-major n x n), D^(i) Q, D^(j) Q
    for (int q = threadIdx.x; q < nn; q += GT) J.Q[q] = T1[q];
    mm(Di, 2 * n, false, T1, n, false, J.DQi, n, n, n, n, 1.0, 0.0);
    mm(Dj, 2 * n, false, T1, n, false, J.DQj, n, n, n, n, 1.0, 0.0);
    if (threadIdx.x == 0) *J.k = k;
}

// ------------------------------------------------------------------- edge
__global__ void __launch_bounds__(GT) k_edge(const EdgeJob* __restrict__ jobs, int* __restrict__ err) {
    const EdgeJob J = jobs[blockIdx.x];
    const int n = J.n, m = J.m, nw = (m - 1) * n, mn = m * n;
    const int nz = mn + J.nH;
    const int np = (nw + 1) & ~1;
    extern __shared__ double shm[];
    double* Ash = shm;
    double* Vsh = shm + np * np;
    __shared__ double cs[64], sn[64];
    __shared__ int pp[64], qq[64];
    __shared__ int order[128];
    __shared__ unsigned char done[1024];
    double* w = J.work;
    const int nn = n * n;
    double* Ssum = w;                     // n x n
    double* Dall = Ssum + nn;             // n x (m n): [D^(k_1) ... D^(k_m)]
    double* Tk = Dall + n * mn;           // m blocks of n x (m n)
    double* BE = Tk + m * n * mn;         // m blocks n x n (sym S_EE)
    double* ME = BE + m * nn;             // nw x nw
    double* T1 = ME + nw * nw;            // scratch  (max(n x mn, nz x nz))
    double* Bt = T1 + (size_t)nz * nz;    // nz x nz
    double* BB = Bt + (size_t)nz * nz;    // nw x nw
    double* W1 = BB + nw * nw;            // nw x nw
    double* W2 = W1 + nw * nw;
    double* V = W2 + nw * nw;
    double* Cm = V + nw * nw;             // n x (m-1) nw
    double* vb = Cm + n * nw * (m - 1) + nw;
    double* Qo = vb + nn;
    double* aux = Qo + nn;                // sigma (nw), QR norms ((m-1) nw), tau (n)
    // deluxe scaling D^(k) = (sum_l S_EE^(l))^{-1} S_EE^(k)
    for (int q = threadIdx.x; q < nn; q += GT) {
        int a = q / n, b = q % n;
        double s = 0.0;
        for (int t = 0; t < m; ++t) {
            double v = J.S[t][(long long)J.pos[t][a] * J.ldS[t] + J.pos[t][b]];
            s += v;
            Dall[a * mn + t * n + b] = v;
        }
        Ssum[q] = s;
    }
    bar();
    for (int q = threadIdx.x; q < m * nn; q += GT) {
        int t = q / nn, a = (q % nn) / n, b = q % n;
        const double* St = J.S[t];
        double v1 = St[(long long)J.pos[t][a] * J.ldS[t] + J.pos[t][b]];
        double v2 = St[(long long)J.pos[t][b] * J.ldS[t] + J.pos[t][a]];
        BE[q] = 0.5 * (v1 + v2);
    }
    bar();
    lu_solve(Ssum, n, Dall, mn, n, mn, err);
    // T^(k): block l (l = 1..m-1, subdomain k_l): (I - D^(k_l)) when k == k_l else -D^(k_l); last block I
    for (int q = threadIdx.x; q < m * n * mn; q += GT) {
        int t = q / (n * mn), a = (q % (n * mn)) / mn, col = q % mn;
        int blk = col / n, b = col % n;
        double v;
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
        mm(BE + t * nn, n, false, Tk + t * n * mn, mn, false, T1, nw, n, nw, n, 1.0, 0.0);
        mm(Tk + t * n * mn, mn, true, T1, nw, false, ME, nw, nw, nw, n, 1.0, 1.0);
    }
    symmetrize(ME, nw, nw);
    if (J.mode == 0) {
    // B~_E = sum_k J_k^T B~^(k) J_k  (z = [w_check (nw), w^_E (n), w^_H (nH)])
    for (int q = threadIdx.x; q < nz * nz; q += GT) Bt[q] = 0.0;
    bar();
    for (int t = 0; t < m; ++t) {
        const double* G = J.Bt[t];
        const int ldg = J.ldBt[t];
        const int h = J.h[t];
        const int* hm = J.hmap[t];
        const double* T = Tk + t * n * mn;
        // EE: T^T G_EE T  ->  Bt[0:mn, 0:mn]
        for (int q = threadIdx.x; q < n * mn; q += GT) {        // T1 = G_EE T  (n x mn)
            int a = q / mn, c = q % mn;
            double s = 0.0;
            for (int l = 0; l < n; ++l) s += G[a * ldg + l] * T[l * mn + c];
            T1[q] = s;
        }
        bar();
        for (int q = threadIdx.x; q < mn * mn; q += GT) {
            int a = q / mn, c = q % mn;
            double s = 0.0;
            for (int l = 0; l < n; ++l) s += T[l * mn + a] * T1[l * mn + c];
            Bt[a * nz + c] += s;
        }
        bar();
        // EH and HE: T^T G_EH
        for (int q = threadIdx.x; q < mn * h; q += GT) {
            int a = q / h, u = q % h;
            double s = 0.0;
            for (int l = 0; l < n; ++l) s += T[l * mn + a] * G[l * ldg + n + u];
            Bt[a * nz + mn + hm[u]] += s;
            double s2 = 0.0;
            for (int l = 0; l < n; ++l) s2 += G[(n + u) * ldg + l] * T[l * mn + a];
            Bt[(mn + hm[u]) * nz + a] += s2;
        }
        bar();
        for (int q = threadIdx.x; q < h * h; q += GT) {
            int u = q / h, v = q % h;
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
    for (int q = threadIdx.x; q < nn; q += GT) Qo[q] = (q / n == q % n) ? 1.0 : 0.0;
    bar();
    if (J.mode == 0) {
        int r = sigma_pencil(ME, BB, nw, Ash, Vsh, np, W1, W2, aux, V, cs, sn, pp, qq, order, err);
        const double sth = J.theta / (1.0 + J.theta) - 1e-12;
        __shared__ int nsel_s;
        if (threadIdx.x == 0) {
            int c = 0;
            for (int q = 0; q < r; ++q) {
                double sg = aux[q];
                J.lambda[q] = (1.0 - sg <= 1e-12) ? INFINITY : sg / (1.0 - sg);
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
            for (int q = threadIdx.x; q < n * nc; q += GT) {
                int a = q / nc, cidx = q % nc;
                int l = cidx / (m - 1), b = cidx % (m - 1);
                int row = b * n + a;
                double acc = 0.0;
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
        mm(Dall + t * n, mn, false, Qo, n, false, J.DQ[t], n, n, n, n, 1.0, 0.0);
    if (threadIdx.x == 0) *J.k = k;
}

}  // namespace

size_t face_work_doubles(int n) { return (size_t)21 * n * n + 3 * n + 64; }
size_t edge_work_doubles(int n, int m, int nH) {
    size_t nw = (size_t)(m - 1) * n, mn = (size_t)m * n, nz = mn + nH;
    return (size_t)n * n * (3 + m) + (size_t)n * mn * (1 + m) + 6 * nw * nw + 2 * nz * nz +
           (size_t)n * nw * (m - 1) + nw + (size_t)m * nw + n + 64;
}

int face_run(const FaceJob* jobs_dev, int count, int maxn, int* err, cudaStream_t st) {
    if (count <= 0) return BDDC_OK;
    int np = (maxn + 1) & ~1;
    size_t smem = (size_t)2 * np * np * sizeof(double);
    if (np > 128 || smem > 200 * 1024) return BDDC_EINVAL;
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_face, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_face<<<count, GT, smem, st>>>(jobs_dev, err);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

int edge_run(const EdgeJob* jobs_dev, int count, int maxnw, int maxnz, int* err, cudaStream_t st) {
    if (count <= 0) return BDDC_OK;
    int np = (maxnw + 1) & ~1;
    size_t smem = (size_t)2 * np * np * sizeof(double);
    if (np > 128 || smem > 200 * 1024 || maxnz > 1024) return BDDC_EINVAL;
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_edge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_edge<<<count, GT, smem, st>>>(jobs_dev, err);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
