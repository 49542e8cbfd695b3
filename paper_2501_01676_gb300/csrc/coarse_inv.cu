// Explicit inverse of a small coarse matrix S_Pi (n_Pi <= COARSE_GJ_MAX) for
// the preconditioner's coarse correction (Sect. 3, u_Pi = S_Pi^{-1} r_Pi).
//
//   X0  = FP32 Gauss-Jordan inverse of S_Pi (symmetrically scaled to unit
//         diagonal), one CTA, in shared memory, no pivoting (the symmetric part
//         of S_Pi is positive definite, as for the subdomain eliminations);
//   X_{k+1} = X_k (2I - S_Pi X_k)            (Newton-Schulz, FP64 products)
//
// Each Newton-Schulz step squares the relative error, so an FP32 start reaches
// FP64 accuracy in a few steps when kappa(S_Pi) * 2^-24 < 1.  The residual
// residual max |I - S_Pi X| of the last iterate and the norms of S_Pi and X are
// returned for the caller's check.
#include <cuda_runtime.h>

#include <utility>

#include "bddc_internal.h"

namespace {

constexpr int GJ_THREADS = 1024;
constexpr int GJ_MAX = 128;        // 32 x 32 threads x 4 x 4 patches
constexpr int GT64 = 8;           // FP64 product tile

// Thread (ty, tx) of a 32 x 32 grid holds the 4 x 4 patch rows 4ty.., columns
// 4tx.. of the (scaled) matrix in registers.  Per pivot k the owners publish
// column k and row k / pivot to shared memory (double-buffered by the parity of
// k, so one barrier per pivot), and every thread updates its patch.
__global__ void __launch_bounds__(GJ_THREADS) k_gj32(const double* __restrict__ S, int n, double* __restrict__ X,
                                                      int ldx, int* __restrict__ err) {
    __shared__ __align__(16) float fcol[2][GJ_MAX];
    __shared__ __align__(16) float rrow[2][GJ_MAX];
    __shared__ float pinv_s[2];
    __shared__ float ds[GJ_MAX];
    const int t = threadIdx.x;
    const int ty = t >> 5, tx = t & 31;
    const int i0 = 4 * ty, j0 = 4 * tx;
    // symmetric diagonal scaling D^{-1/2} S D^{-1/2} (S has a positive diagonal): the
    // FP32 start then sees the conditioning left after coefficient jumps are removed
    for (int i = t; i < n; i += GJ_THREADS) {
        const double sii = S[(long long)i * n + i];
        ds[i] = sii > 0.0 ? (float)(1.0 / sqrt(sii)) : 1.f;
    }
    __syncthreads();
    float a[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + u, j = j0 + v;
            a[u][v] = (i < n && j < n) ? (float)S[(long long)i * n + j] * ds[i] * ds[j] : (i == j ? 1.f : 0.f);
        }
    bool bad = false;
    for (int k = 0; k < n; ++k) {
        const int b = k & 1;
        const int ku = k - i0, kv = k - j0;           // position of row / column k in the patch
        // publish column k (raw) and row k (scaled by 1 / pivot)
        if (kv >= 0 && kv < 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (v == kv) fcol[b][i0 + u] = a[u][v];
        }
        __syncthreads();                               // column k (and the pivot) visible
        float p = fcol[b][k];
        if (!(fabsf(p) > 0.f) || !isfinite(p)) {
            bad = true;
            p = 1.f;
        }
        const float pi = 1.f / p;
        if (ku >= 0 && ku < 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (u == ku) rrow[b][j0 + v] = a[u][v] * pi;
        }
        __syncthreads();                               // row k visible
        float fr[4], rr[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) fr[u] = fcol[b][i0 + u];
#pragma unroll
        for (int v = 0; v < 4; ++v) rr[v] = rrow[b][j0 + v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int i = i0 + u, j = j0 + v;
                if (i == k) a[u][v] = (j == k) ? pi : rr[v];
                else if (j == k) a[u][v] = -fr[u] * pi;
                else a[u][v] -= fr[u] * rr[v];
            }
    }
    if (bad && t == 0) atomicOr(err, ERR_PIVOT);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + u, j = j0 + v;
            if (i < n && j < n) X[(long long)i * ldx + j] = (double)a[u][v] * ds[i] * ds[j];
        }
}

// C = alpha * A B + beta * C + gamma * I   (n x n, FP64, 16 x 16 tiles)
__global__ void __launch_bounds__(GT64 * GT64) k_gemm64(const double* __restrict__ A, int lda,
                                                        const double* __restrict__ B, int ldb, double* __restrict__ C,
                                                        int ldc, int n, double alpha, double beta, double gamma) {
    __shared__ double As[GT64][GT64 + 1], Bs[GT64][GT64 + 1];
    const int ty = threadIdx.x / GT64, tx = threadIdx.x % GT64;
    const int r = blockIdx.y * GT64 + ty, c = blockIdx.x * GT64 + tx;
    double acc = 0.0;
    for (int k0 = 0; k0 < n; k0 += GT64) {
        As[ty][tx] = (r < n && k0 + tx < n) ? A[(long long)r * lda + k0 + tx] : 0.0;
        Bs[ty][tx] = (k0 + ty < n && c < n) ? B[(long long)(k0 + ty) * ldb + c] : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GT64; ++k) acc += As[ty][k] * Bs[k][tx];
        __syncthreads();
    }
    if (r < n && c < n) {
        double v = alpha * acc + (r == c ? gamma : 0.0);
        if (beta != 0.0) v += beta * C[(long long)r * ldc + c];
        C[(long long)r * ldc + c] = v;
    }
}

// out[0] = max |R|, out[1] = ||S||_inf, out[2] = ||X||_inf: a warp per row (lanes
// across the row, so that the loads coalesce), combined with atomicMax on the
// bit patterns (non-negative doubles order like their integer images); out
// starts at zero.
__device__ __forceinline__ void atomic_max_nonneg(double* a, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

__global__ void k_resid_norms(const double* __restrict__ R, int ldr, const double* __restrict__ S, int lds,
                              const double* __restrict__ X, int ldx, int n, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    double m = 0.0, a = 0.0, b = 0.0;
    for (int j = lane; j < n; j += 32) {
        m = fmax(m, fabs(R[(long long)i * ldr + j]));
        a += fabs(S[(long long)i * lds + j]);
        b += fabs(X[(long long)i * ldx + j]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        atomic_max_nonneg(out, m);
        atomic_max_nonneg(out + 1, a);
        atomic_max_nonneg(out + 2, b);
    }
}

int gemm64(const double* A, int lda, const double* B, int ldb, double* C, int ldc, int n, double alpha,
           double beta, double gamma, cudaStream_t st) {
    const int g = (n + GT64 - 1) / GT64;
    k_gemm64<<<dim3(g, g), GT64 * GT64, 0, st>>>(A, lda, B, ldb, C, ldc, n, alpha, beta, gamma);
    bddc_note_launches(1);
    return BDDC_OK;
}

}  // namespace

// X (n x n, ld ldx) ~ S^{-1}; work: 2 * n * n doubles; resid: three doubles (device):
// max |I - S X|, ||S||_inf, ||X||_inf.
// Returns BDDC_EINVAL when n exceeds the single-CTA limit.
int coarse_inverse_small(const double* S, int n, double* X, int ldx, double* work, double* resid, int ns_steps,
                         int* err, cudaStream_t st) {
    if (n <= 0 || n > COARSE_GJ_MAX || n > GJ_MAX) return BDDC_EINVAL;
    k_gj32<<<1, GJ_THREADS, 0, st>>>(S, n, X, ldx, err);
    bddc_note_launches(1);
    double* R = work;              // n x n
    double* Y = work + (size_t)n * n;
    double* cur = X;
    int ldcur = ldx;
    double* nxt = Y;
    int ldnxt = n;
    for (int k = 0; k < ns_steps; ++k) {
        // R = 2I - S X ;  X <- X R
        BDDC_TRY(gemm64(S, n, cur, ldcur, R, n, n, -1.0, 0.0, 2.0, st));
        BDDC_TRY(gemm64(cur, ldcur, R, n, nxt, ldnxt, n, 1.0, 0.0, 0.0, st));
        std::swap(cur, nxt);
        std::swap(ldcur, ldnxt);
    }
    if (cur != X)
        BDDC_CUDA_TRY(cudaMemcpy2DAsync(X, sizeof(double) * ldx, cur, sizeof(double) * ldcur, sizeof(double) * n, n,
                                        cudaMemcpyDeviceToDevice, st));
    BDDC_TRY(gemm64(S, n, X, ldx, R, n, n, -1.0, 0.0, 1.0, st));
    BDDC_CUDA_TRY(cudaMemsetAsync(resid, 0, 3 * sizeof(double), st));
    k_resid_norms<<<(n + 7) / 8, 256, 0, st>>>(R, n, S, n, X, ldx, n, resid);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
