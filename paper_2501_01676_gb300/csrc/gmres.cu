// FP64 Arnoldi / Givens kernels of right-preconditioned GMRES (Sect. 4: the
// iteration stops when the residual falls below the tolerance or after 300
// iterations).  Classical Gram-Schmidt applied twice (CGS2) in three fused
// passes (dots; update + dots; update + norm), each one launch whose last CTA
// reduces the per-chunk partial sums in a fixed order.
// All scalars of the iteration (Hessenberg column, rotations, residual
// estimate, stop flag) stay on the device so a fixed block of iterations can
// be replayed as one CUDA graph; every kernel returns at once when the stop
// flag is set.
#include <cuda_runtime.h>

#include <algorithm>

#include "bddc_internal.h"
#include "gmres.h"

namespace {

constexpr int DOT_THREADS = 256;
constexpr int DOT_ROWS = 8;      // rows per block of the dot kernel
constexpr int DOT_CHUNK = 1024;  // vector elements per block (several CTAs per row group)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// partial[row * nchunk + chunk] = sum_{e in chunk} V[row][e] * w[e], rows 0..nrows-1
__global__ void __launch_bounds__(DOT_THREADS) k_dots(const double* __restrict__ V, long long ldv,
                                                      const double* __restrict__ w, long long n,
                                                      const GmState* __restrict__ S, int rows_mode,
                                                      double* __restrict__ partial, int nchunk, GmBatch B) {
    const int col = blockIdx.z;
    S += col;
    if (V) V += col * B.sV;
    w += col * B.sW;
    partial += col * B.sP;
    if (S->stop) return;
    const int nrows = rows_mode == 0 ? S->j + 1 : 1;   // 0: rows 0..j; 1: w.w
    const int r0 = blockIdx.y * DOT_ROWS;
    if (r0 >= nrows) return;
    const int nr = min(DOT_ROWS, nrows - r0);
    const long long e0 = (long long)blockIdx.x * DOT_CHUNK;
    const long long e1 = min(n, e0 + DOT_CHUNK);
    double acc[DOT_ROWS];
#pragma unroll
    for (int r = 0; r < DOT_ROWS; ++r) acc[r] = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += DOT_THREADS) {
        double we = w[e];
#pragma unroll
        for (int r = 0; r < DOT_ROWS; ++r)
            if (r < nr) acc[r] += (rows_mode == 0 ? V[(r0 + r) * ldv + e] : we) * we;
    }
    __shared__ double red[DOT_THREADS / 32][DOT_ROWS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < DOT_ROWS; ++r) {
        double v = warp_sum(acc[r]);
        if (lane == 0) red[wid][r] = v;
    }
    __syncthreads();
    if (threadIdx.x < nr) {
        double s = 0.0;
        for (int q = 0; q < DOT_THREADS / 32; ++q) s += red[q][threadIdx.x];
        partial[(long long)(r0 + threadIdx.x) * nchunk + blockIdx.x] = s;
    }
}

constexpr int PASS_THREADS = 256;
constexpr int PASS_EPT = 4;                       // vector elements per thread
constexpr int PASS_CHUNK = PASS_THREADS * PASS_EPT;

// One CGS2 pass: optional w -= V[0..j] hin (element-parallel, w held in
// registers), then the partial sums of V[0..j] . w (or of w . w) of this CTA's
// chunk, and the last CTA to finish reduces the partials in chunk order.
template <int MODE>
__global__ void __launch_bounds__(PASS_THREADS) k_pass(const double* __restrict__ V, long long ldv,
                                                       double* __restrict__ w, long long n, GmState* __restrict__ S,
                                                       const double* __restrict__ hin, double* __restrict__ hout,
                                                       double* __restrict__ partial, int nchunk, GmBatch B) {
    const int col = blockIdx.z;
    S += col;
    V += col * B.sV;
    w += col * B.sW;
    if (hin) hin += col * B.sSm;
    if (hout) hout += col * B.sSm;
    partial += col * B.sP;
    if (S->stop) return;
    const int nr = S->j + 1;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const long long e0 = (long long)blockIdx.x * PASS_CHUNK + t;
    __shared__ double red[PASS_THREADS / 32][8];
    __shared__ int last;
    double wv[PASS_EPT];
#pragma unroll
    for (int k = 0; k < PASS_EPT; ++k) {
        const long long e = e0 + (long long)k * PASS_THREADS;
        wv[k] = e < n ? w[e] : 0.0;
    }
    if (MODE != 0) {
        for (int i = 0; i < nr; ++i) {
            const double c = hin[i];
            const double* vi = V + (long long)i * ldv;
#pragma unroll
            for (int k = 0; k < PASS_EPT; ++k) {
                const long long e = e0 + (long long)k * PASS_THREADS;
                if (e < n) wv[k] -= c * vi[e];
            }
        }
#pragma unroll
        for (int k = 0; k < PASS_EPT; ++k) {
            const long long e = e0 + (long long)k * PASS_THREADS;
            if (e < n) w[e] = wv[k];
        }
    }
    const int nrows = MODE == 2 ? 1 : nr;
    for (int r0 = 0; r0 < nrows; r0 += 8) {
        double acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            acc[q] = 0.0;
            if (r0 + q < nrows) {
                const double* vi = MODE == 2 ? nullptr : V + (long long)(r0 + q) * ldv;
#pragma unroll
                for (int k = 0; k < PASS_EPT; ++k) {
                    const long long e = e0 + (long long)k * PASS_THREADS;
                    if (e < n) acc[q] += (MODE == 2 ? wv[k] : vi[e]) * wv[k];
                }
            }
            acc[q] = warp_sum(acc[q]);
        }
        if (lane < 8) {
            double v = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q == lane) v = acc[q];
            red[wid][lane] = v;
        }
        __syncthreads();
        if (t < 8 && r0 + t < nrows) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < PASS_THREADS / 32; ++q) s += red[q][t];
            partial[(long long)(r0 + t) * nchunk + blockIdx.x] = s;
        }
        __syncthreads();
    }
    // last CTA: reduce the partials of all chunks
    __threadfence();
    if (t == 0) last = atomicAdd(&S->cnt, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int row = wid; row < nrows; row += PASS_THREADS / 32) {
        double s = 0.0;
        for (int c = lane; c < nchunk; c += 32) s += partial[(long long)row * nchunk + c];
        s = warp_sum(s);
        if (lane == 0) {
            if (MODE == 2) S->nrm2 = s;
            else hout[row] = s;
        }
    }
    if (t == 0) {
        S->cnt = 0;
        if (MODE == 0) S->need_norm = 0;
    }
}

// h[row] (+)= sum_chunks partial; mode 0: h = sum, 1: h += sum, 2: store in S->nrm2
__global__ void k_dots_reduce(const double* __restrict__ partial, int nchunk, GmState* __restrict__ S,
                              double* __restrict__ h, int mode, int rows_mode, GmBatch B) {
    const int col = blockIdx.z;
    S += col;
    partial += col * B.sP;
    if (h) h += col * B.sSm;
    if (S->stop) return;
    const int nrows = rows_mode == 0 ? S->j + 1 : 1;
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (row >= nrows) return;
    double s = 0.0;
    for (int c = lane; c < nchunk; c += 32) s += partial[(long long)row * nchunk + c];
    s = warp_sum(s);
    if (lane == 0) {
        if (mode == 0) h[row] = s;
        else if (mode == 1) h[row] += s;
        else S->nrm2 = s;
    }
}

// w -= sum_{i<=j} c[i] V[i]
__global__ void k_orth_update(const double* __restrict__ V, long long ldv, double* __restrict__ w,
                              long long n, const GmState* __restrict__ S, const double* __restrict__ c, GmBatch B) {
    const int col = blockIdx.z;
    S += col;
    V += col * B.sV;
    w += col * B.sW;
    c += col * B.sSm;
    if (S->stop) return;
    const int nr = S->j + 1;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        double acc = w[e];
        for (int i = 0; i < nr; ++i) acc -= c[i] * V[i * ldv + e];
        w[e] = acc;
    }
}

// one Arnoldi step's scalar work: Hessenberg column, Givens, residual estimate
__global__ void k_givens(GmState* __restrict__ S, double* __restrict__ H, double* __restrict__ cs,
                         double* __restrict__ sn, double* __restrict__ gv, const double* __restrict__ h,
                         const double* __restrict__ h2, GmBatch B) {
    const int bc = blockIdx.z;
    S += bc;
    H += bc * B.sH;
    cs += bc * B.sSm;
    sn += bc * B.sSm;
    gv += bc * B.sSm;
    h += bc * B.sSm;
    h2 += bc * B.sSm;
    if (threadIdx.x != 0 || S->stop) return;
    const int j = S->j, m = S->m;
    double* col = H + (long long)j * (m + 1);          // column j, length m+1
    for (int i = 0; i <= j; ++i) col[i] = h[i] + h2[i];
    double hn = sqrt(fmax(S->nrm2, 0.0));
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    double a = col[j], b = col[j + 1];
    double den = hypot(a, b);
    double c = den > 0 ? a / den : 1.0, s = den > 0 ? b / den : 0.0;
    cs[j] = c;
    sn[j] = s;
    col[j] = den;
    col[j + 1] = 0.0;
    gv[j + 1] = -s * gv[j];
    gv[j] = c * gv[j];
    S->scale = hn > 0 ? 1.0 / hn : 0.0;
    S->j = j + 1;
    S->total += 1;
    S->res = fabs(gv[j + 1]);
    S->need_norm = 1;
    if (S->res <= S->tol || hn == 0.0) {
        S->converged = 1;
        S->stop = 1;
    } else if (S->j >= m || S->total >= S->max_iter) {
        S->stop = 1;
    }
}

// V[j] = w * scale  (j already advanced)
// V[j] = w * scale and the next preconditioner input vcur = V[j]
__global__ void k_normalize(double* __restrict__ V, long long ldv, const double* __restrict__ w,
                            long long n, GmState* __restrict__ S, double* __restrict__ vcur, GmBatch B) {
    const int col = blockIdx.z;
    S += col;
    V += col * B.sV;
    w += col * B.sW;
    vcur += col * B.sW;
    if (!S->need_norm) return;
    const int j = S->j;
    if (j > S->m) return;
    const double sc = S->scale;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const double v = w[e] * sc;
        V[j * ldv + e] = v;
        vcur[e] = v;
    }
}

__global__ void k_clear_norm(GmState* S) { S[blockIdx.z].need_norm = 0; }

// vcur = V[j]
__global__ void k_copy_row(const double* __restrict__ V, long long ldv, double* __restrict__ out,
                           long long n, const GmState* __restrict__ S, GmBatch B) {
    const int col = blockIdx.z;
    S += col;
    V += col * B.sV;
    out += col * B.sW;
    if (S->stop) return;
    const int j = S->j;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = V[j * ldv + e];
}

// y = H(1:k,1:k)^{-1} g(1:k), then t = V(:,1:k) y
__global__ void k_backsolve(const GmState* __restrict__ S, const double* __restrict__ H,
                            const double* __restrict__ gv, double* __restrict__ y, GmBatch B) {
    const int col = blockIdx.z;
    S += col;
    H += col * B.sH;
    gv += col * B.sSm;
    y += col * B.sSm;
    if (threadIdx.x != 0) return;
    const int k = S->j, m = S->m;
    for (int i = k - 1; i >= 0; --i) {
        double s = gv[i];
        for (int l = i + 1; l < k; ++l) s -= H[(long long)l * (m + 1) + i] * y[l];
        double d = H[(long long)i * (m + 1) + i];
        y[i] = d != 0.0 ? s / d : 0.0;
    }
}

// Condition estimate of the preconditioned operator from the cycle's
// Hessenberg: after the Givens rotations its leading k x k block is the
// triangular R, whose singular values are those of the (k+1) x k Hessenberg;
// sigma_max by power iteration on R^T R, sigma_min by inverse iteration
// (R^T z = x, R x' = z, column-oriented substitutions); kmax = max(kmax, ratio).
// R is staged in shared memory (cycles of up to GM_COND_MAX columns; longer
// cycles are not estimated) and two warps run the substitutions.
constexpr int GM_COND_MAX = 128;
constexpr int GM_COND_ITERS = 16;
constexpr int GM_COND_THREADS = 128;
// kappa_est = sigma_max(R) / sigma_min(R) of the triangular factor R of the
// Hessenberg: sigma_max(R) by power iteration on R^T R; then R is inverted in
// place (X = R^{-1}, column by column from X R = I: X(i, j) = -(sum_{i <= l < j}
// X(i, l) R(l, j)) / R(j, j), two barriers per column) and sigma_min(R) =
// 1 / sigma_max(X) by the same power iteration on X^T X.  A zero diagonal entry
// gives kappa_est = infinity.
__global__ void __launch_bounds__(GM_COND_THREADS) k_cond(const GmState* __restrict__ S,
                                                          const double* __restrict__ H,
                                                          double* __restrict__ kmax, GmBatch B) {
    extern __shared__ double Rs[];                  // k x k, row-major
    __shared__ double x[GM_COND_MAX], z[GM_COND_MAX], red[GM_COND_THREADS / 32];
    __shared__ int zero_s;
    S += blockIdx.z;
    H += blockIdx.z * B.sH;
    const int k = S->j, m = S->m, t = threadIdx.x;
    if (k <= 0 || k > GM_COND_MAX) return;
    for (int q = t; q < k * k; q += GM_COND_THREADS) {
        const int i = q / k, l = q - i * k;
        Rs[q] = l >= i ? H[(long long)l * (m + 1) + i] : 0.0;
    }
    if (t == 0) zero_s = 0;
    __syncthreads();
    auto norm = [&](const double* v) {
        double a = 0.0;
        for (int i = t; i < k; i += GM_COND_THREADS) a += v[i] * v[i];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if ((t & 31) == 0) red[t >> 5] = a;
        __syncthreads();
        double s2 = 0.0;
        for (int w = 0; w < GM_COND_THREADS / 32; ++w) s2 += red[w];
        __syncthreads();
        return sqrt(s2);
    };
    // largest singular value of the upper triangle in Rs: power iteration on Rs^T Rs
    auto sigma_max = [&](double x0, double dx) {
        for (int i = t; i < k; i += GM_COND_THREADS) x[i] = x0 + dx * i;
        __syncthreads();
        double sm = 0.0;
        for (int it = 0; it < GM_COND_ITERS; ++it) {
            const double nx = norm(x);
            for (int i = t; i < k; i += GM_COND_THREADS) x[i] /= nx;
            __syncthreads();
            for (int i = t; i < k; i += GM_COND_THREADS) {       // z = R x
                double a = 0.0;
                for (int l = i; l < k; ++l) a += Rs[i * k + l] * x[l];
                z[i] = a;
            }
            __syncthreads();
            sm = norm(z);
            for (int i = t; i < k; i += GM_COND_THREADS) {       // x = R^T z
                double a = 0.0;
                for (int l = 0; l <= i; ++l) a += Rs[l * k + i] * z[l];
                x[i] = a;
            }
            __syncthreads();
        }
        return sm;
    };
    const double smax = sigma_max(1.0, 1e-3);
    // X = R^{-1} in place: column j from the finished columns < j and R's column j
    for (int j = 0; j < k; ++j) {
        const double d = Rs[j * k + j];
        if (d == 0.0 && t == 0) zero_s = 1;
        double v[GM_COND_MAX / GM_COND_THREADS];
#pragma unroll
        for (int u = 0; u < GM_COND_MAX / GM_COND_THREADS; ++u) {
            const int i = t + u * GM_COND_THREADS;
            double a = 0.0;
            if (i < j)
                for (int l = i; l < j; ++l) a += Rs[i * k + l] * Rs[l * k + j];
            v[u] = d != 0.0 ? -a / d : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < GM_COND_MAX / GM_COND_THREADS; ++u) {
            const int i = t + u * GM_COND_THREADS;
            if (i < j) Rs[i * k + j] = v[u];
            if (i == j) Rs[j * k + j] = d != 0.0 ? 1.0 / d : 0.0;
        }
        __syncthreads();
    }
    const double sxmax = sigma_max(1.0, -1e-3);      // = 1 / sigma_min(R)
    if (t == 0) {
        // positive doubles order like their bit patterns: max over columns by atomicMax
        const double kap = (zero_s || !(sxmax > 0.0)) ? INFINITY : smax * sxmax;
        atomicMax(reinterpret_cast<unsigned long long*>(kmax), (unsigned long long)__double_as_longlong(kap));
    }
}

__global__ void k_combine(const double* __restrict__ V, long long ldv, const double* __restrict__ y,
                          const GmState* __restrict__ S, double* __restrict__ t, long long n, GmBatch B) {
    const int col = blockIdx.z;
    S += col;
    V += col * B.sV;
    y += col * B.sSm;
    t += col * B.sW;
    const int k = S->j;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < k; ++i) acc += y[i] * V[i * ldv + e];
        t[e] = acc;
    }
}

// start a cycle from r: beta = ||r||, V[0] = r / beta, g = beta e1
__global__ void k_cycle_start(GmState* __restrict__ S, double* __restrict__ gv, const double* __restrict__ partial,
                              int nchunk, GmBatch B) {
    const int col = blockIdx.z;
    S += col;
    gv += col * B.sSm;
    partial += col * B.sP;
    if (threadIdx.x != 0) return;
    if (S->done) {                      // a column that has finished stays stopped and adds nothing
        S->stop = 1;
        S->j = 0;
        return;
    }
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += partial[c];
    double beta = sqrt(fmax(s, 0.0));
    S->beta = beta;
    S->j = 0;
    S->stop = 0;
    S->need_norm = 0;
    gv[0] = beta;
    S->scale = beta > 0 ? 1.0 / beta : 0.0;
    S->res = beta;
    if (beta <= S->tol) {
        S->converged = 1;
        S->stop = 1;
    }
}

__global__ void k_scale_into(double* __restrict__ dst, long long sdst, const double* __restrict__ src, long long n,
                             const GmState* __restrict__ S, GmBatch B) {
    const int col = blockIdx.z;
    S += col;
    dst += col * sdst;
    src += col * B.sW;
    const double sc = S->scale;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = src[e] * sc;
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double a, double b,
                        long long n, GmBatch B) {
    y += blockIdx.z * B.sW;
    x += blockIdx.z * B.sW;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        y[e] = a * x[e] + b * y[e];
}

// flag = 1 when every column has stopped (the operators' skip flag of a batched solve)
__global__ void k_all_stopped(const GmState* __restrict__ S, int ncol, int* __restrict__ flag) {
    __shared__ int any_running;
    if (threadIdx.x == 0) any_running = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < ncol; c += blockDim.x)
        if (!S[c].stop) any_running = 1;
    __syncthreads();
    if (threadIdx.x == 0) *flag = any_running ? 0 : 1;
}

// y[:, c] = a x[:, c] + b y[:, c] with separate column strides
__global__ void k_axpby_cols(double* __restrict__ y, long long ldy, const double* __restrict__ x, long long ldx,
                             double a, double b, long long n) {
    y += blockIdx.z * ldy;
    x += blockIdx.z * ldx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        y[e] = a * x[e] + b * y[e];
}

inline int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)(g < 1184 ? (g < 1 ? 1 : g) : 1184);
}

}  // namespace

int gm_nchunk(long long n) { return (int)((n + DOT_CHUNK - 1) / DOT_CHUNK); }

// h (mode 0 set / 1 add) = V[0..j]^T w
int gm_dots(const double* V, long long ldv, const double* w, long long n, GmState* S, double* partial,
            double* h, int mode, int max_rows, cudaStream_t st, GmBatch B) {
    int nchunk = gm_nchunk(n);
    dim3 grid(nchunk, (max_rows + DOT_ROWS - 1) / DOT_ROWS, B.ncol);
    k_dots<<<grid, DOT_THREADS, 0, st>>>(V, ldv, w, n, S, 0, partial, nchunk, B);
    bddc_note_launches(1);
    k_dots_reduce<<<dim3((max_rows + 7) / 8, 1, B.ncol), 256, 0, st>>>(partial, nchunk, S, h, mode, 0, B);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

int gm_norm2(const double* w, long long n, GmState* S, double* partial, cudaStream_t st, GmBatch B) {
    int nchunk = gm_nchunk(n);
    k_dots<<<dim3(nchunk, 1, B.ncol), DOT_THREADS, 0, st>>>(nullptr, 0, w, n, S, 1, partial, nchunk, B);
    bddc_note_launches(1);
    k_dots_reduce<<<dim3(1, 1, B.ncol), 32, 0, st>>>(partial, nchunk, S, nullptr, 2, 1, B);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
int gm_orth_update(const double* V, long long ldv, double* w, long long n, const GmState* S,
                   const double* c, cudaStream_t st, GmBatch B) {
    k_orth_update<<<dim3(grid_for(n), 1, B.ncol), 256, 0, st>>>(V, ldv, w, n, S, c, B);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
int gm_givens(GmState* S, double* H, double* cs, double* sn, double* gv, const double* h,
              const double* h2, cudaStream_t st, GmBatch B) {
    k_givens<<<dim3(1, 1, B.ncol), 32, 0, st>>>(S, H, cs, sn, gv, h, h2, B);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
int gm_normalize(double* V, long long ldv, const double* w, long long n, GmState* S, double* vcur,
                 cudaStream_t st, GmBatch B) {
    // need_norm is cleared by the next iteration's first pass (k_pass<0>)
    k_normalize<<<dim3(grid_for(n), 1, B.ncol), 256, 0, st>>>(V, ldv, w, n, S, vcur, B);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
int gm_pass(int mode, const double* V, long long ldv, double* w, long long n, GmState* S, const double* hin,
            double* hout, double* partial, cudaStream_t st, GmBatch B) {
    const int nchunk = (int)((n + PASS_CHUNK - 1) / PASS_CHUNK);
    const dim3 grid(nchunk, 1, B.ncol);
    if (mode == 0) k_pass<0><<<grid, PASS_THREADS, 0, st>>>(V, ldv, w, n, S, hin, hout, partial, nchunk, B);
    else if (mode == 1) k_pass<1><<<grid, PASS_THREADS, 0, st>>>(V, ldv, w, n, S, hin, hout, partial, nchunk, B);
    else k_pass<2><<<grid, PASS_THREADS, 0, st>>>(V, ldv, w, n, S, hin, hout, partial, nchunk, B);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
int gm_copy_row(const double* V, long long ldv, double* out, long long n, const GmState* S,
                cudaStream_t st, GmBatch B) {
    k_copy_row<<<dim3(grid_for(n), 1, B.ncol), 256, 0, st>>>(V, ldv, out, n, S, B);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
int gm_cycle_start(const double* r, long long n, GmState* S, GmState* Sspare, double* gv, double* partial,
                   double* V0, double* vcur, cudaStream_t st, GmBatch B) {
    int nchunk = gm_nchunk(n);
    // plain norm pass that ignores the stop flag: private state copies
    k_dots<<<dim3(nchunk, 1, B.ncol), DOT_THREADS, 0, st>>>(nullptr, 0, r, n, Sspare, 1, partial, nchunk, B);
    bddc_note_launches(1);
    k_cycle_start<<<dim3(1, 1, B.ncol), 32, 0, st>>>(S, gv, partial, nchunk, B);
    bddc_note_launches(1);
    k_scale_into<<<dim3(grid_for(n), 1, B.ncol), 256, 0, st>>>(V0, B.sV, r, n, S, B);
    bddc_note_launches(1);
    k_scale_into<<<dim3(grid_for(n), 1, B.ncol), 256, 0, st>>>(vcur, B.sW, r, n, S, B);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
int gm_finish(const double* V, long long ldv, const GmState* S, const double* H, const double* gv,
              double* y, double* t, long long n, cudaStream_t st, GmBatch B) {
    k_backsolve<<<dim3(1, 1, B.ncol), 32, 0, st>>>(S, H, gv, y, B);
    bddc_note_launches(1);
    k_combine<<<dim3(grid_for(n), 1, B.ncol), 256, 0, st>>>(V, ldv, y, S, t, n, B);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
int vec_axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t st, GmBatch B) {
    k_axpby<<<dim3(grid_for(n), 1, B.ncol), 256, 0, st>>>(y, x, a, b, n, B);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
int gm_cond(const GmState* S, const double* H, int mmax, double* kmax, cudaStream_t st, GmBatch B) {
    const int kk = std::min(mmax, GM_COND_MAX);
    const size_t smem = sizeof(double) * kk * kk;
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_cond, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double) * GM_COND_MAX * GM_COND_MAX)));
    k_cond<<<dim3(1, 1, B.ncol), GM_COND_THREADS, smem, st>>>(S, H, kmax, B);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

int gm_all_stopped(const GmState* S, int ncol, int* flag, cudaStream_t st) {
    k_all_stopped<<<1, 256, 0, st>>>(S, ncol, flag);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
int vec_axpby_cols(double* y, long long ldy, const double* x, long long ldx, double a, double b, long long n,
                   int ncol, cudaStream_t st) {
    k_axpby_cols<<<dim3(grid_for(n), 1, ncol), 256, 0, st>>>(y, ldy, x, ldx, a, b, n);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
