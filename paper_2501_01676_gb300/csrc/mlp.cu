// Learned edge-GEP skip: edge features and a small FP32 MLP with hand-written
// forward, backward and Adam kernels (not in the paper; it predicts from
// local coefficients how many adaptive constraints the edge GEP of eq. equ-5-21
// will select, so that edges confidently predicted to select none can skip
// the GEP; the full GEP stays the fallback).
//
// Features of an edge (a line of n_E interior dofs along axis a, shared by
// the subdomains n(E)); touching elements are the 4 (n_E + 1) elements that
// contain the closed segment:
//   0-2 min / max / mean log10 nu over touching elements
//   3   max - min over n(E) of the per-subdomain mean log10 nu
//   4-6 mean |beta_a|, max |beta_a|, mean |beta| over the edge nodes
//   7   edge length (n_E + 1) h_a,  8  (H/h) / 10,  9  log10(h_a * f6 / (2 * 10^f2))
// Network: 10 -> 64 -> 64 -> 64 (ReLU) -> 8 logits, mean softmax cross-entropy;
// flat parameters W1[10][64], b1, W2[64][64], b2, W3[64][64], b3, W4[64][8], b4.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "bddc_internal.h"
#include "mlp.h"

namespace {

constexpr int NF = BDDC_MLP_FEATURES, NH = BDDC_MLP_HIDDEN, NC = BDDC_MLP_CLASSES;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NF * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NH, OFF_W4 = OFF_B3 + NH,
              OFF_B4 = OFF_W4 + NH * NC, NPARAM = OFF_B4 + NC;
static_assert(NPARAM == BDDC_MLP_PARAMS, "parameter layout");

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double wmin(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// one warp per edge
__global__ void k_edge_features(const EdgeDesc* __restrict__ ed, int nedges, const double* __restrict__ nu,
                                const double* __restrict__ beta, double3 bconst, const int* __restrict__ slab_x,
                                const int* __restrict__ slab_y, const int* __restrict__ slab_z, int nsx, int nsy,
                                int Ex, int Ey, double hx, double hy, double hz, float* __restrict__ F) {
    const int e = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= nedges) return;
    const EdgeDesc D = ed[e];
    const int a = D.axis;
    const int f0 = a == 0 ? 1 : 0, f1 = a == 2 ? 1 : 2;
    const int nel = 4 * (D.hi - D.lo + 2);
    double mn = 1e300, mx = -1e300, sm = 0.0;
    double ssum[4] = {0, 0, 0, 0}, scnt[4] = {0, 0, 0, 0};
    for (int q = lane; q < nel; q += 32) {
        int ea = D.lo - 1 + (q >> 2);
        int d1 = (q & 1) - 1, d2 = ((q >> 1) & 1) - 1;
        int idx[3];
        idx[a] = ea;
        idx[f0] = D.c0 + d1;
        idx[f1] = D.c1 + d2;
        long long el = idx[0] + (long long)Ex * (idx[1] + (long long)Ey * idx[2]);
        double ln = log10(nu[el]);
        mn = fmin(mn, ln);
        mx = fmax(mx, ln);
        sm += ln;
        int s = slab_x[idx[0]] + nsx * (slab_y[idx[1]] + nsy * slab_z[idx[2]]);
        for (int k = 0; k < 4; ++k)
            if (D.subs[k] == s) {
                ssum[k] += ln;
                scnt[k] += 1.0;
            }
    }
    mn = wmin(mn);
    mx = wmax(mx);
    sm = wsum(sm);
    for (int k = 0; k < 4; ++k) {
        ssum[k] = wsum(ssum[k]);
        scnt[k] = wsum(scnt[k]);
    }
    const int nE = D.hi - D.lo + 1;
    double bt = 0.0, btm = 0.0, bn = 0.0;
    for (int q = lane; q < nE; q += 32) {
        int idx[3];
        idx[a] = D.lo + q;
        idx[f0] = D.c0;
        idx[f1] = D.c1;
        long long nd = idx[0] + (long long)(Ex + 1) * (idx[1] + (long long)(Ey + 1) * idx[2]);
        double b0, b1, b2;
        if (beta) {
            b0 = beta[3 * nd];
            b1 = beta[3 * nd + 1];
            b2 = beta[3 * nd + 2];
        } else {
            b0 = bconst.x;
            b1 = bconst.y;
            b2 = bconst.z;
        }
        double ba = fabs(a == 0 ? b0 : (a == 1 ? b1 : b2));
        bt += ba;
        btm = fmax(btm, ba);
        bn += sqrt(b0 * b0 + b1 * b1 + b2 * b2);
    }
    bt = wsum(bt);
    btm = wmax(btm);
    bn = wsum(bn);
    if (lane == 0) {
        double mean = sm / nel;
        double lo = 1e300, hi = -1e300;
        for (int k = 0; k < 4; ++k)
            if (scnt[k] > 0) {
                double v = ssum[k] / scnt[k];
                lo = fmin(lo, v);
                hi = fmax(hi, v);
            }
        const double h = a == 0 ? hx : (a == 1 ? hy : hz);
        const double bnm = bn / nE;
        float* f = F + (long long)e * NF;
        f[0] = (float)mn;
        f[1] = (float)mx;
        f[2] = (float)mean;
        f[3] = (float)(hi - lo);
        f[4] = (float)(bt / nE);
        f[5] = (float)btm;
        f[6] = (float)bnm;
        f[7] = (float)((nE + 1) * h);
        f[8] = (float)(D.m / 10.0);
        f[9] = (float)log10(fmax(h * bnm / (2.0 * pow(10.0, mean)), 1e-30));
        f[10] = (float)log10(D.theta);
    }
}

// Z[r][j] = b[j] + sum_i A[r][i] W[i][j];  H = relu(Z) (relu != 0)
__global__ void k_layer(const float* __restrict__ A, int nin, const float* __restrict__ W, const float* __restrict__ b,
                        int nout, int rows, float* __restrict__ Z, float* __restrict__ H, int relu) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)rows * nout) return;
    const int r = (int)(q / nout), j = (int)(q - (long long)r * nout);
    float s = b[j];
    const float* ar = A + (long long)r * nin;
    for (int i = 0; i < nin; ++i) s += ar[i] * W[i * nout + j];
    Z[q] = s;
    if (H) H[q] = relu ? fmaxf(s, 0.f) : s;
}

// softmax cross-entropy: per-row loss, dL = (softmax - onehot) / rows
__global__ void k_softmax_ce(const float* __restrict__ L, const int* __restrict__ y, int rows, float* __restrict__ loss,
                             float* __restrict__ dL, float* __restrict__ P) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const float* l = L + (long long)r * NC;
    float m = l[0];
    for (int c = 1; c < NC; ++c) m = fmaxf(m, l[c]);
    float e[NC], s = 0.f;
    for (int c = 0; c < NC; ++c) {
        e[c] = expf(l[c] - m);
        s += e[c];
    }
    for (int c = 0; c < NC; ++c) {
        float p = e[c] / s;
        if (P) P[(long long)r * NC + c] = p;
        if (dL) dL[(long long)r * NC + c] = (p - (y && c == y[r] ? 1.f : 0.f)) / rows;
    }
    if (loss && y) loss[r] = -logf(fmaxf(e[y[r]] / s, 1e-30f));
}

// dA[r][i] = sum_j dZ[r][j] W[i][j], then (when Zp given) dZp = dA * (Zp > 0)
__global__ void k_back_act(const float* __restrict__ dZ, int nout, const float* __restrict__ W, int nin, int rows,
                           const float* __restrict__ Zp, float* __restrict__ dZp) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)rows * nin) return;
    const int r = (int)(q / nin), i = (int)(q - (long long)r * nin);
    const float* dz = dZ + (long long)r * nout;
    float s = 0.f;
    for (int j = 0; j < nout; ++j) s += dz[j] * W[i * nout + j];
    dZp[q] = (Zp == nullptr || Zp[q] > 0.f) ? s : 0.f;
}

// gW[i][j] = sum_r A[r][i] dZ[r][j], gb[j] = sum_r dZ[r][j]: one block per (i or bias) row,
// deterministic tree reduction over rows.
__global__ void k_wgrad(const float* __restrict__ A, int nin, const float* __restrict__ dZ, int nout, int rows,
                        float* __restrict__ gW, float* __restrict__ gb) {
    const int i = blockIdx.x;   // 0..nin-1 weights, nin: bias
    __shared__ float red[256];
    for (int j = 0; j < nout; ++j) {
        float s = 0.f;
        for (int r = threadIdx.x; r < rows; r += blockDim.x)
            s += (i < nin ? A[(long long)r * nin + i] : 1.f) * dZ[(long long)r * nout + j];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (i < nin) gW[i * nout + j] = red[0];
            else gb[j] = red[0];
        }
        __syncthreads();
    }
}

__global__ void k_sum(const float* __restrict__ v, int n, float* __restrict__ out) {
    __shared__ float red[256];
    float s = 0.f;
    for (int q = threadIdx.x; q < n; q += blockDim.x) s += v[q];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / n;
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1t, float b2t) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float b1 = 0.9f, b2 = 0.999f;
    float mk = b1 * m[k] + (1.f - b1) * g[k];
    float vk = b2 * v[k] + (1.f - b2) * g[k] * g[k];
    m[k] = mk;
    v[k] = vk;
    th[k] -= lr * (mk / (1.f - b1t)) / (sqrtf(vk / (1.f - b2t)) + 1e-8f);
}

inline int blocks(long long n, int th) { return (int)((n + th - 1) / th); }

struct Work {
    float *z1, *h1, *z2, *h2, *z3, *h3, *L, *dL, *d3, *d2, *d1, *loss, *g;
};

int alloc_work(Work& w, int rows, cudaStream_t st, std::vector<void*>& keep) {
    auto A = [&](float** p, size_t n) -> int {
        BDDC_CUDA_TRY(cudaMallocAsync((void**)p, std::max<size_t>(n, 1) * sizeof(float), st));
        keep.push_back(*p);
        return BDDC_OK;
    };
    BDDC_TRY(A(&w.z1, (size_t)rows * NH));
    BDDC_TRY(A(&w.h1, (size_t)rows * NH));
    BDDC_TRY(A(&w.z2, (size_t)rows * NH));
    BDDC_TRY(A(&w.h2, (size_t)rows * NH));
    BDDC_TRY(A(&w.z3, (size_t)rows * NH));
    BDDC_TRY(A(&w.h3, (size_t)rows * NH));
    BDDC_TRY(A(&w.L, (size_t)rows * NC));
    BDDC_TRY(A(&w.dL, (size_t)rows * NC));
    BDDC_TRY(A(&w.d3, (size_t)rows * NH));
    BDDC_TRY(A(&w.d2, (size_t)rows * NH));
    BDDC_TRY(A(&w.d1, (size_t)rows * NH));
    BDDC_TRY(A(&w.loss, (size_t)rows + 1));
    BDDC_TRY(A(&w.g, NPARAM));
    return BDDC_OK;
}

void free_work(std::vector<void*>& keep, cudaStream_t st) {
    for (void* p : keep) cudaFreeAsync(p, st);
    keep.clear();
}

int forward(const float* th, const float* X, int rows, Work& w, cudaStream_t st) {
    const int T = 256;
    k_layer<<<blocks((long long)rows * NH, T), T, 0, st>>>(X, NF, th + OFF_W1, th + OFF_B1, NH, rows, w.z1, w.h1, 1);
    bddc_note_launches(1);
    k_layer<<<blocks((long long)rows * NH, T), T, 0, st>>>(w.h1, NH, th + OFF_W2, th + OFF_B2, NH, rows, w.z2, w.h2, 1);
    bddc_note_launches(1);
    k_layer<<<blocks((long long)rows * NH, T), T, 0, st>>>(w.h2, NH, th + OFF_W3, th + OFF_B3, NH, rows, w.z3, w.h3, 1);
    bddc_note_launches(1);
    k_layer<<<blocks((long long)rows * NC, T), T, 0, st>>>(w.h3, NH, th + OFF_W4, th + OFF_B4, NC, rows, w.L, nullptr, 0);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

int backward(const float* th, const float* X, const int* y, int rows, Work& w, float* loss_dev, cudaStream_t st) {
    const int T = 256;
    k_softmax_ce<<<blocks(rows, T), T, 0, st>>>(w.L, y, rows, w.loss, w.dL, nullptr);
    bddc_note_launches(1);
    k_sum<<<1, 256, 0, st>>>(w.loss, rows, loss_dev);
    bddc_note_launches(1);
    float* g = w.g;
    k_wgrad<<<NH + 1, 256, 0, st>>>(w.h3, NH, w.dL, NC, rows, g + OFF_W4, g + OFF_B4);
    bddc_note_launches(1);
    k_back_act<<<blocks((long long)rows * NH, T), T, 0, st>>>(w.dL, NC, th + OFF_W4, NH, rows, w.z3, w.d3);
    bddc_note_launches(1);
    k_wgrad<<<NH + 1, 256, 0, st>>>(w.h2, NH, w.d3, NH, rows, g + OFF_W3, g + OFF_B3);
    bddc_note_launches(1);
    k_back_act<<<blocks((long long)rows * NH, T), T, 0, st>>>(w.d3, NH, th + OFF_W3, NH, rows, w.z2, w.d2);
    bddc_note_launches(1);
    k_wgrad<<<NH + 1, 256, 0, st>>>(w.h1, NH, w.d2, NH, rows, g + OFF_W2, g + OFF_B2);
    bddc_note_launches(1);
    k_back_act<<<blocks((long long)rows * NH, T), T, 0, st>>>(w.d2, NH, th + OFF_W2, NH, rows, w.z1, w.d1);
    bddc_note_launches(1);
    k_wgrad<<<NF + 1, 256, 0, st>>>(X, NF, w.d1, NH, rows, g + OFF_W1, g + OFF_B1);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

}  // namespace

int mlp_edge_features(const EdgeDesc* ed, int nedges, const double* nu, const double* beta, const double bconst[3],
                      const int* sx, const int* sy, const int* sz, int nsx, int nsy, int Ex, int Ey,
                      const double h[3], float* F, cudaStream_t st) {
    if (nedges <= 0) return BDDC_OK;
    k_edge_features<<<blocks(nedges, 8), 256, 0, st>>>(ed, nedges, nu, beta, make_double3(bconst[0], bconst[1], bconst[2]),
                                                       sx, sy, sz, nsx, nsy, Ex, Ey, h[0], h[1], h[2], F);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

int mlp_probs(const float* params_dev, const float* X, int rows, float* P, cudaStream_t st) {
    if (rows <= 0) return BDDC_OK;
    Work w;
    std::vector<void*> keep;
    BDDC_TRY(alloc_work(w, rows, st, keep));
    BDDC_TRY(forward(params_dev, X, rows, w, st));
    k_softmax_ce<<<blocks(rows, 256), 256, 0, st>>>(w.L, nullptr, rows, nullptr, nullptr, P);
    bddc_note_launches(1);
    free_work(keep, st);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

extern "C" {

int bddc_mlp_forward(const float* params_host, const float* X_dev, int rows, float* probs_dev, void* stream) {
    if (!params_host || !X_dev || !probs_dev || rows < 0) return BDDC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    float* th = nullptr;
    BDDC_CUDA_TRY(cudaMallocAsync((void**)&th, NPARAM * sizeof(float), st));
    BDDC_CUDA_TRY(cudaMemcpyAsync(th, params_host, NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    int rc = mlp_probs(th, X_dev, rows, probs_dev, st);
    cudaFreeAsync(th, st);
    BDDC_CUDA_TRY(cudaStreamSynchronize(st));
    return rc;
}

int bddc_mlp_loss_grad(const float* params_host, const float* X_dev, const int* y_dev, int rows, float* grad_host,
                       float* loss_host, void* stream) {
    if (!params_host || !X_dev || !y_dev || rows <= 0) return BDDC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    float* th = nullptr;
    float* ld = nullptr;
    BDDC_CUDA_TRY(cudaMallocAsync((void**)&th, NPARAM * sizeof(float), st));
    BDDC_CUDA_TRY(cudaMallocAsync((void**)&ld, sizeof(float), st));
    BDDC_CUDA_TRY(cudaMemcpyAsync(th, params_host, NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    Work w;
    std::vector<void*> keep;
    BDDC_TRY(alloc_work(w, rows, st, keep));
    BDDC_TRY(forward(th, X_dev, rows, w, st));
    BDDC_TRY(backward(th, X_dev, y_dev, rows, w, ld, st));
    if (grad_host) BDDC_CUDA_TRY(cudaMemcpyAsync(grad_host, w.g, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (loss_host) BDDC_CUDA_TRY(cudaMemcpyAsync(loss_host, ld, sizeof(float), cudaMemcpyDeviceToHost, st));
    free_work(keep, st);
    cudaFreeAsync(th, st);
    cudaFreeAsync(ld, st);
    BDDC_CUDA_TRY(cudaStreamSynchronize(st));
    return BDDC_OK;
}

int bddc_mlp_train(float* params_host, const float* X_dev, const int* y_dev, int rows, int epochs, float lr,
                   float* loss_host, void* stream) {
    if (!params_host || !X_dev || !y_dev || rows <= 0 || epochs < 0) return BDDC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    float *th = nullptr, *m = nullptr, *v = nullptr, *ld = nullptr;
    BDDC_CUDA_TRY(cudaMallocAsync((void**)&th, NPARAM * sizeof(float), st));
    BDDC_CUDA_TRY(cudaMallocAsync((void**)&m, NPARAM * sizeof(float), st));
    BDDC_CUDA_TRY(cudaMallocAsync((void**)&v, NPARAM * sizeof(float), st));
    BDDC_CUDA_TRY(cudaMallocAsync((void**)&ld, (epochs + 1) * sizeof(float), st));
    BDDC_CUDA_TRY(cudaMemcpyAsync(th, params_host, NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    BDDC_CUDA_TRY(cudaMemsetAsync(m, 0, NPARAM * sizeof(float), st));
    BDDC_CUDA_TRY(cudaMemsetAsync(v, 0, NPARAM * sizeof(float), st));
    Work w;
    std::vector<void*> keep;
    BDDC_TRY(alloc_work(w, rows, st, keep));
    double b1t = 1.0, b2t = 1.0;
    for (int ep = 0; ep < epochs; ++ep) {
        BDDC_TRY(forward(th, X_dev, rows, w, st));
        BDDC_TRY(backward(th, X_dev, y_dev, rows, w, ld + ep, st));
        b1t *= 0.9;
        b2t *= 0.999;
        k_adam<<<blocks(NPARAM, 256), 256, 0, st>>>(th, w.g, m, v, NPARAM, lr, (float)b1t, (float)b2t);
        bddc_note_launches(1);
    }
    BDDC_TRY(forward(th, X_dev, rows, w, st));
    BDDC_TRY(backward(th, X_dev, y_dev, rows, w, ld + epochs, st));
    BDDC_CUDA_TRY(cudaGetLastError());
    BDDC_CUDA_TRY(cudaMemcpyAsync(params_host, th, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (loss_host) BDDC_CUDA_TRY(cudaMemcpyAsync(loss_host, ld, (epochs + 1) * sizeof(float), cudaMemcpyDeviceToHost, st));
    free_work(keep, st);
    cudaFreeAsync(th, st);
    cudaFreeAsync(m, st);
    cudaFreeAsync(v, st);
    cudaFreeAsync(ld, st);
    BDDC_CUDA_TRY(cudaStreamSynchronize(st));
    return BDDC_OK;
}

}  // extern "C"
