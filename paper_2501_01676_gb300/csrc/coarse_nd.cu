// Assembly of the nested-dissection fronts of the coarse problem (the coarse
// matrix S_Pi of M^-1, Sect. 3).  The elimination of each front runs in the
// batched elimination engine; the solve sweeps run in the batched GEMV.
#include <cuda_runtime.h>

#include "bddc_internal.h"

namespace {

constexpr int ND_THREADS = 256;

// Extended front [[F11, F12, -I], [F21, F22, 0], [I, 0, 0]]: the blocks that
// touch an own unknown come from S_Pi; F22 starts at zero (the entries of two
// boundary unknowns belong to an ancestor's front) and collects the children's
// updates afterwards.
__global__ void __launch_bounds__(ND_THREADS) k_nd_fill(const NDFront* __restrict__ fr,
                                                        const NDRowJob* __restrict__ jobs,
                                                        const int* __restrict__ idx,
                                                        const double* __restrict__ S, int nPi,
                                                        double* __restrict__ F) {
    const NDRowJob j = jobs[blockIdx.x];
    const NDFront f = fr[j.front];
    const int n = f.n, m = f.n + f.b;
    const int* v = idx + f.vars_off;
    double* A = F + f.foff;
    for (int r = j.row0; r < j.row0 + j.nrows; ++r) {
        double* row = A + (long long)r * f.ld;
        const double* srow = r < m ? S + (long long)v[r] * nPi : nullptr;
        for (int c = threadIdx.x; c < f.ld; c += ND_THREADS) {
            double val = 0.0;
            if (c < m && r < m) {
                if (r < n || c < n) val = srow[v[c]];
            } else if (r < n && c >= m && c < f.N) {
                val = (c - m == r) ? -1.0 : 0.0;
            } else if (r >= m && c < n) {
                val = (r - m == c) ? 1.0 : 0.0;
            }
            row[c] = val;
        }
    }
}

// F_parent[map[r]][map[c]] += U_child[r][c], U = the child's b x b trailing block.
__global__ void __launch_bounds__(ND_THREADS) k_nd_add(const NDFront* __restrict__ fr,
                                                       const NDRowJob* __restrict__ jobs,
                                                       const int* __restrict__ idx, double* F) {
    const NDRowJob j = jobs[blockIdx.x];
    const NDFront fc = fr[j.front];
    const NDFront fp = fr[fc.parent];
    const int* map = idx + fc.map_off;
    const double* U = F + fc.foff + (long long)fc.n * fc.ld + fc.n;
    double* P = F + fp.foff;
    for (int r = j.row0; r < j.row0 + j.nrows; ++r) {
        double* prow = P + (long long)map[r] * fp.ld;
        const double* urow = U + (long long)r * fc.ld;
        for (int c = threadIdx.x; c < fc.b; c += ND_THREADS) atomicAdd(prow + map[c], urow[c]);
    }
}

}  // namespace

int nd_fill_run(const NDFront* fr_dev, const NDRowJob* jobs, int njobs, const int* idx, const double* S, int nPi,
                double* F, cudaStream_t st) {
    if (njobs <= 0) return BDDC_OK;
    k_nd_fill<<<njobs, ND_THREADS, 0, st>>>(fr_dev, jobs, idx, S, nPi, F);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

int nd_add_run(const NDFront* fr_dev, const NDRowJob* jobs, int njobs, const int* idx, double* F, cudaStream_t st) {
    if (njobs <= 0) return BDDC_OK;
    k_nd_add<<<njobs, ND_THREADS, 0, st>>>(fr_dev, jobs, idx, F);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
