// Explicit inverse of a small coarse matrix S_Pi (n_Pi <= COARSE_GJ_MAX) for
// the preconditioner's coarse correction (Sect. 3, u_Pi = S_Pi^{-1} r_Pi).
//
//   X0  = FP32 Gauss-Jordan inverse of S_Pi, one CTA, in shared memory, no
//         pivoting (the symmetric part of S_Pi is positive definite, as for the
//         subdomain eliminations);
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
constexpr int GT64 = 16;          // FP64 product tile

// Warp w owns rows w, w+32, ...; lane l owns columns l, l+32, ...  Per pivot k:
// save column k and the scaled row k, then update every entry (2 barriers).
__global__ void __launch_bounds__(GJ_THREADS) k_gj32(const double* __restrict__ S, int n, double* __restrict__ X,
                                                      int ldx, int* __restrict__ err) {
    extern __shared__ float gj[];
    const int ld = n + 1;
    float* A = gj;                 // n x ld
    float* f = A + n * ld;         // column k
    float* r = f + n;              // row k scaled by 1 / pivot
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    constexpr int NW = GJ_THREADS / 32;
    for (int i = wid; i < n; i += NW)
        for (int j = lane; j < n; j += 32) A[i * ld + j] = (float)S[(long long)i * n + j];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        float p = A[k * ld + k];
        if (!(fabsf(p) > 0.f) || !isfinite(p)) {
            if (t == 0) atomicOr(err, ERR_PIVOT);
            p = 1.f;
        }
        const float pi = 1.f / p;
        if (wid == 0)
            for (int j = lane; j < n; j += 32) r[j] = A[k * ld + j] * pi;
        else if (wid == 1)
            for (int i = lane; i < n; i += 32) f[i] = A[i * ld + k];
        __syncthreads();
        for (int i = wid; i < n; i += NW) {
            const float fi = f[i];
            for (int j = lane; j < n; j += 32) {
                float v;
                if (i == k) v = (j == k) ? pi : r[j];
                else v = (j == k) ? -fi * pi : A[i * ld + j] - fi * r[j];
                A[i * ld + j] = v;
            }
        }
        __syncthreads();
    }
    for (int i = wid; i < n; i += NW)
        for (int j = lane; j < n; j += 32) X[(long long)i * ldx + j] = (double)A[i * ld + j];
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

// out[0] = max |R|, out[1] = ||S||_inf, out[2] = ||X||_inf  (one CTA; a warp per
// row, lanes across the row, so that the loads coalesce)
__global__ void k_resid_norms(const double* __restrict__ R, int ldr, const double* __restrict__ S, int lds,
                              const double* __restrict__ X, int ldx, int n, double* __restrict__ out) {
    __shared__ double red[3][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double m = 0.0, ns = 0.0, nx = 0.0;
    for (int i = wid; i < n; i += nw) {
        double a = 0.0, b = 0.0;
        for (int j = lane; j < n; j += 32) {
            m = fmax(m, fabs(R[(long long)i * ldr + j]));
            a += fabs(S[(long long)i * lds + j]);
            b += fabs(X[(long long)i * ldx + j]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        ns = fmax(ns, a);
        nx = fmax(nx, b);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
        red[0][wid] = m;
        red[1][wid] = ns;
        red[2][wid] = nx;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double r = 0.0;
        for (int w = 0; w < nw; ++w) r = fmax(r, red[threadIdx.x][w]);
        out[threadIdx.x] = r;
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
    if (n <= 0 || n > COARSE_GJ_MAX) return BDDC_EINVAL;
    const size_t smem = sizeof(float) * ((size_t)n * (n + 1) + 2 * (size_t)n);
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_gj32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_gj32<<<1, GJ_THREADS, smem, st>>>(S, n, X, ldx, err);
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
    k_resid_norms<<<1, 1024, 0, st>>>(R, n, S, n, X, ldx, n, resid);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
