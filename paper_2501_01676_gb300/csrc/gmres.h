// Device-resident scalar state of one GMRES cycle.
#pragma once
#include <cuda_runtime.h>

// Column strides of batched GMRES arrays (elements): column c of an array is
// base + c * stride; the GmState of column c is S[c].  ncol = 1 with zero
// strides is the single-column solver.
struct GmBatch {
    int ncol;
    long long sV;    // Krylov basis V ((m+1) x ld)
    long long sW;    // n-vectors (w, vcur, r, t, x, b)
    long long sH;    // Hessenberg
    long long sSm;   // per-column scalar arrays (cs, sn, g, h, h2, y)
    long long sP;    // partial sums of the reductions
};
inline GmBatch gm_single() { return GmBatch{1, 0, 0, 0, 0, 0}; }

struct GmState {
    int j;           // Arnoldi index within the cycle (number of columns done)
    int m;           // cycle length (restart, or the iteration cap)
    int stop;        // 1: converged, cycle full or cap reached
    int converged;
    int total;       // iterations over all cycles
    int max_iter;
    int need_norm;
    int cnt;         // CTAs of a fused pass that have stored their partial sums
    double tol;      // absolute residual target rtol * ||b||
    double beta;     // initial residual norm of the cycle
    double res;      // current residual estimate |g_{j}|
    double nrm2;     // squared norm of the new Krylov vector
    double scale;    // 1 / norm used to normalise it
    int done;        // batched solves: the column has finished (no new cycle)
    int pad_;
};

int gm_nchunk(long long n);
int gm_dots(const double* V, long long ldv, const double* w, long long n, GmState* S, double* partial,
            double* h, int mode, int max_rows, cudaStream_t st, GmBatch B = gm_single());
int gm_norm2(const double* w, long long n, GmState* S, double* partial, cudaStream_t st, GmBatch B = gm_single());
int gm_orth_update(const double* V, long long ldv, double* w, long long n, const GmState* S,
                   const double* c, cudaStream_t st, GmBatch B = gm_single());
int gm_givens(GmState* S, double* H, double* cs, double* sn, double* gv, const double* h,
              const double* h2, cudaStream_t st, GmBatch B = gm_single());
int gm_normalize(double* V, long long ldv, const double* w, long long n, GmState* S, double* vcur,
                 cudaStream_t st, GmBatch B = gm_single());
// One fused CGS2 pass over the Krylov basis V[0..j] (one launch, last-CTA reduction):
//   mode 0: hout = V^T w;  1: w -= V hin, then hout = V^T w;  2: w -= V hin, then S->nrm2 = w.w
int gm_pass(int mode, const double* V, long long ldv, double* w, long long n, GmState* S, const double* hin,
            double* hout, double* partial, cudaStream_t st, GmBatch B = gm_single());
int gm_copy_row(const double* V, long long ldv, double* out, long long n, const GmState* S,
                cudaStream_t st, GmBatch B = gm_single());
// Start a cycle from r: beta = ||r|| (reduced with the private states Sspare),
// V[0] = vcur = r / beta; a column whose GmState has `done` set stays stopped.
int gm_cycle_start(const double* r, long long n, GmState* S, GmState* Sspare, double* gv, double* partial,
                   double* V0, double* vcur, cudaStream_t st, GmBatch B = gm_single());
int gm_finish(const double* V, long long ldv, const GmState* S, const double* H, const double* gv,
              double* y, double* t, long long n, cudaStream_t st, GmBatch B = gm_single());
int vec_axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t st,
              GmBatch B = gm_single());
// Condition estimate sigma_max / sigma_min of the cycle's Hessenberg (the
// triangular factor left by the Givens rotations); *kmax = max(*kmax, estimate)
// over the columns.  mmax: the cycle length the Hessenberg was allocated for;
// cycles longer than 128 columns are not estimated.
int gm_cond(const GmState* S, const double* H, int mmax, double* kmax, cudaStream_t st, GmBatch B = gm_single());
// *flag = 1 when every column's GmState has stopped, else 0.
int gm_all_stopped(const GmState* S, int ncol, int* flag, cudaStream_t st);
// y[:, c] = a x[:, c] + b y[:, c], c < ncol, column strides ldy / ldx.
int vec_axpby_cols(double* y, long long ldy, const double* x, long long ldx, double a, double b, long long n,
                   int ncol, cudaStream_t st);
