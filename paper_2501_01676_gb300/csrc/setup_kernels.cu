// Data movement of the setup: gathers that build the engine's input matrices,
// the change of basis T_i^T S T_i onto primal / dual coordinates, and the
// extraction of the constrained-solver operators from the engine's output.
//
// Change of basis (Sect. 3, after eq. primal-constraints-F: "after performing
// a change of basis"): on every face / edge X of subdomain i the interface
// values are w_X = Q_X y_X with Q_X = [Q_X^Pi, Q_X^Delta] orthogonal; the
// first k_X coordinates are primal.  T_i is block diagonal over the entities.
#include <cuda_runtime.h>

#include "bddc_internal.h"
#include "setup_kernels.h"

namespace {

constexpr int TH = 256;

template <class TS, class TD>
__global__ void k_copy_blocks(const CopyJob* __restrict__ jobs) {
    const CopyJob J = jobs[blockIdx.x];
    const TS* src = (const TS*)J.src;
    TD* dst = (TD*)J.dst;
    for (int r = blockIdx.y; r < J.rows; r += gridDim.y) {
        const TS* sr = src + (long long)(J.r0 + r) * J.sld + J.c0;
        TD* dr = dst + (long long)r * J.dld;
        for (int c = threadIdx.x; c < J.cols; c += TH) dr[c] = (TD)(J.scale * (double)sr[c]);
    }
}

// dst[a][b] = S[p_a][p_b] (optionally symmetrised), p = perm list.  32 x 32
// tiles, 8 rows of 32 lanes: the lanes run along b for S[p_a][p_b] and along a
// for the transposed term S[p_b][p_a] (staged in shared memory), so both reads
// follow the contiguous runs of the permutation.
template <class TD>
__global__ void k_gather_perm(const GatherJob* __restrict__ jobs, const int* __restrict__ idx) {
    const GatherJob J = jobs[blockIdx.x];
    const int* p = idx + J.perm_off;
    TD* dst = (TD*)J.dst;
    const TD* sT = (const TD*)J.srcT;
    __shared__ double T2[32][33];
    const int nt = (J.n + 31) / 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    constexpr int RY = TH / 32;
    auto S = [&](long long i, long long j) -> double {
        return J.src ? J.src[i * J.sld + j] : (double)sT[i * J.sld + j];
    };
    for (int tile = blockIdx.y; tile < nt * nt; tile += gridDim.y) {
        const int a0 = (tile / nt) * 32, b0 = (tile % nt) * 32;
        if (J.sym) {
            for (int bb = ty; bb < 32; bb += RY) {
                const int b = b0 + bb, a = a0 + tx;
                T2[bb][tx] = (a < J.n && b < J.n) ? S(p[b], p[a]) : 0.0;
            }
            __syncthreads();
        }
        for (int aa = ty; aa < 32; aa += RY) {
            const int a = a0 + aa, b = b0 + tx;
            if (a < J.n && b < J.n) {
                double v = S(p[a], p[b]);
                if (J.sym) v = 0.5 * (v + T2[tx][aa]);
                dst[(long long)a * J.dld + b] = (TD)v;
            }
        }
        if (J.sym) __syncthreads();
    }
}

// Right multiplication Y[r][pos[l]] = sum_a B[r][pos[a]] Q[a][l] for one entity block
// (arithmetic and the scratch Y in precision TY).
template <class TY>
__global__ void k_transform_right(const TBlock* __restrict__ blocks, const int* __restrict__ idx, int qglob) {
    const TBlock B = blocks[blockIdx.x];
    extern __shared__ __align__(16) unsigned char qraw[];
    TY* Qs = reinterpret_cast<TY*>(qraw);
    const int n = B.n;
    const int* pos = idx + B.pos_off;
    TY* Y = (TY*)B.y;
    if (!B.identity && !qglob)
        for (int q = threadIdx.x; q < n * n; q += TH) Qs[q] = (TY)B.Q[q];
    __syncthreads();
    // Q from shared memory, or straight from global memory (qglob: too large to stage)
    auto Qv = [&](int a, int l) -> TY { return qglob ? (TY)B.Q[a * n + l] : Qs[a * n + l]; };
    const int rpi = n < TH ? TH / n : 1;                 // rows per CTA pass
    const int lr = (int)threadIdx.x / n, l0 = (int)threadIdx.x % n;
    if (lr >= rpi) return;
    for (int r = blockIdx.y * rpi + lr; r < B.nrows; r += gridDim.y * rpi)
    for (int l = l0; l < n; l += (n < TH ? n : TH)) {
        const double* row = B.src + (long long)r * B.sld;
        TY v;
        if (B.identity) {
            v = (TY)row[pos[l]];
            if (B.sym) v = (TY)0.5 * (v + (TY)B.src[(long long)pos[l] * B.sld + r]);
        } else {
            v = 0;
            for (int a = 0; a < n; ++a) {
                TY sv = (TY)row[pos[a]];
                if (B.sym) sv = (TY)0.5 * (sv + (TY)B.src[(long long)pos[a] * B.sld + r]);
                v += sv * Qv(a, l);
            }
        }
        Y[(long long)r * B.yld + pos[l]] = v;
    }
}

// Left multiplication Z[pos[l]][c] = sum_a Q[a][l] Y[pos[a]][c] and the
// permuted store X[perm[pos[l]]][perm[c]] = Z (entries with perm < 0 dropped).
template <class TY, class TD>
__global__ void k_transform_left(const TBlock* __restrict__ blocks, const int* __restrict__ idx, int qglob) {
    const TBlock B = blocks[blockIdx.x];
    extern __shared__ __align__(16) unsigned char qraw[];
    TY* Qs = reinterpret_cast<TY*>(qraw);
    const int n = B.n;
    const int* pos = idx + B.pos_off;
    const int* perm = idx + B.perm_off;
    const TY* Y = (const TY*)B.y;
    if (!B.identity && !qglob)
        for (int q = threadIdx.x; q < n * n; q += TH) Qs[q] = (TY)B.Q[q];
    __syncthreads();
    auto Qv = [&](int a, int l) -> TY { return qglob ? (TY)B.Q[a * n + l] : Qs[a * n + l]; };
    TD* X = (TD*)B.dst;
    for (int l = 0; l < n; ++l)
    for (int c = blockIdx.y * TH + threadIdx.x; c < B.nrows; c += gridDim.y * TH) {
        int pr = perm[pos[l]], pc = perm[c];
        if (pr < 0 || pc < 0) continue;
        TY v;
        if (B.identity) v = Y[(long long)pos[l] * B.yld + c];
        else {
            v = 0;
            for (int a = 0; a < n; ++a) v += Qv(a, l) * Y[(long long)pos[a] * B.yld + c];
        }
        X[(long long)pr * B.dld + pc] = (TD)v;
    }
}

// Change of basis by blocks, one CTA per (subdomain, row block X): for every
// column block Y gather B = S[pX, pY] (symmetric part if asked), W = B QY,
// Z = QX^T W, and store Z at the permuted positions (rows and columns of one
// entity are contiguous runs of the output).  Shared memory: QX, QY, B, W.
template <class TY, class TD>
__global__ void k_basis(const XRow* __restrict__ rows, const XSub* __restrict__ subs,
                        const XBlock* __restrict__ blks, int nmax) {
    const XRow R = rows[blockIdx.x];
    const XSub S = subs[R.sub];
    const XBlock BX = blks[S.blk_off + R.blk];
    extern __shared__ __align__(16) unsigned char braw[];
    TY* QX = reinterpret_cast<TY*>(braw);
    TY* QY = QX + nmax * nmax;
    TY* Bm = QY + nmax * nmax;
    TY* W = Bm + nmax * nmax;
    const int nx = BX.n;
    const int* px = BX.pos;
    const int* perm = S.perm;
    TD* dst = (TD*)S.dst;
    const int t = threadIdx.x;
    if (BX.Q)
        for (int q = t; q < nx * nx; q += TH) QX[q] = (TY)BX.Q[q];
    for (int yb = 0; yb < S.nblk; ++yb) {
        const XBlock BY = blks[S.blk_off + yb];
        const int ny = BY.n;
        const int* py = BY.pos;
        for (int q = t; q < nx * ny; q += TH) {
            const int a = q / ny, b = q - a * ny;
            const long long ia = px[a], ib = py[b];
            double v = S.src[ia * S.sld + ib];
            if (S.sym) v = 0.5 * (v + S.src[ib * S.sld + ia]);
            Bm[q] = (TY)v;
        }
        if (BY.Q)
            for (int q = t; q < ny * ny; q += TH) QY[q] = (TY)BY.Q[q];
        __syncthreads();
        const TY* Wp = Bm;
        if (BY.Q) {
            for (int q = t; q < nx * ny; q += TH) {
                const int a = q / ny, m = q - a * ny;
                const TY* br = Bm + a * ny;
                TY s = 0;
                for (int b = 0; b < ny; ++b) s += br[b] * QY[b * ny + m];
                W[q] = s;
            }
            __syncthreads();
            Wp = W;
        }
        for (int q = t; q < nx * ny; q += TH) {
            const int l = q / ny, m = q - l * ny;
            const int pr = perm[px[l]], pc = perm[py[m]];
            if (pr < 0 || pc < 0) continue;
            TY z;
            if (BX.Q) {
                z = 0;
                for (int a = 0; a < nx; ++a) z += QX[a * nx + l] * Wp[a * ny + m];
            } else {
                z = Wp[l * ny + m];
            }
            dst[(long long)pr * S.dld + pc] = (TD)z;
        }
        __syncthreads();
    }
}

// X[nB + pos[a]][perm[pos[l]]] = DQ[a][l];  X[perm[pos[l]]][nB + pos[a]] = -DQ[a][l]
template <class TD>
__global__ void k_fill_dt(const DTJob* __restrict__ jobs, const int* __restrict__ idx) {
    const DTJob J = jobs[blockIdx.x];
    const int* pos = idx + J.pos_off;
    const int* perm = idx + J.perm_off;
    TD* X = (TD*)J.dst;
    for (int q = threadIdx.x; q < J.n * J.n; q += TH) {
        int a = q / J.n, l = q % J.n;
        double v = J.DQ ? J.DQ[q] : (a == l ? J.scalar : 0.0);
        int pc = perm[pos[l]];
        X[(long long)(J.nB + pos[a]) * J.dld + pc] = (TD)v;
        X[(long long)pc * J.dld + J.nB + pos[a]] = (TD)(-v);
    }
}

// From the eliminated extended matrix of subdomain i
//   [S_Pi,i | -Psi^T D^T ; D Phi | P]  (rows/cols from nD on)
// write  S_Pi,i into the global coarse matrix (atomics), [P ; Psi^T D^T]
// into the first apply pool and D Phi into the second.
template <class TX, class TP>
__global__ void k_extract(const ExtractJob* __restrict__ jobs, const int* __restrict__ idx,
                          double* __restrict__ SPi, int nPi) {
    const ExtractJob J = jobs[blockIdx.x];
    const TX* X = (const TX*)J.X;
    const int nB = J.nB, np = J.np, nd = nB - np;
    const int* rpi = idx + J.rpi_off;
    TP* MA = (TP*)J.MA;
    TP* MC = (TP*)J.MC;
    for (int a = blockIdx.y; a < np; a += gridDim.y)
        for (int b = threadIdx.x; b < np; b += TH)
            atomicAdd(&SPi[(long long)rpi[a] * nPi + rpi[b]], (double)X[(long long)(nd + a) * J.xld + nd + b]);
    for (int a = blockIdx.y; a < nB; a += gridDim.y) {
        const TX* xr = X + (long long)(nB + a) * J.xld;
        for (int b = threadIdx.x; b < nB; b += TH) MA[(long long)a * J.ald + b] = (TP)xr[nB + b];
        for (int b = threadIdx.x; b < np; b += TH) MC[(long long)b * J.cld + a] = (TP)xr[nd + b];
    }
    for (int a = blockIdx.y; a < np; a += gridDim.y) {
        const TX* xr = X + (long long)(nd + a) * J.xld + nB;
        for (int b = threadIdx.x; b < nB; b += TH) MA[(long long)(nB + a) * J.ald + b] = (TP)(-xr[b]);
    }
}

__global__ void k_coarse_ext(const double* __restrict__ SPi, double* __restrict__ X, int n) {
    // X = [[S_Pi, -I], [I, 0]] (2n x 2n, ld 2n)
    const long long tot = 4LL * n * n;
    for (long long q = blockIdx.x * (long long)TH + threadIdx.x; q < tot; q += (long long)gridDim.x * TH) {
        int a = (int)(q / (2 * n)), b = (int)(q % (2 * n));
        double v;
        if (a < n && b < n) v = SPi[(long long)a * n + b];
        else if (a < n) v = (b - n == a) ? -1.0 : 0.0;
        else if (b < n) v = (a - n == b) ? 1.0 : 0.0;
        else v = 0.0;
        X[q] = v;
    }
}

}  // namespace

template <class TS, class TD>
int copy_blocks_run(const CopyJob* jobs, int count, int ychunks, cudaStream_t st) {
    if (count <= 0) return BDDC_OK;
    k_copy_blocks<TS, TD><<<dim3(count, ychunks), TH, 0, st>>>(jobs);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
template int copy_blocks_run<double, double>(const CopyJob*, int, int, cudaStream_t);
template int copy_blocks_run<float, double>(const CopyJob*, int, int, cudaStream_t);
template int copy_blocks_run<float, float>(const CopyJob*, int, int, cudaStream_t);
template int copy_blocks_run<double, float>(const CopyJob*, int, int, cudaStream_t);

namespace {
template <class T>
__global__ void k_extend_add(const ExtendJob* __restrict__ jobs) {
    const ExtendJob J = jobs[blockIdx.x];
    const T* S = (const T*)J.src;
    T* D = (T*)J.dst;
    const long long nn = (long long)J.n * J.n;
    for (long long q = (long long)blockIdx.y * TH + threadIdx.x; q < nn; q += (long long)gridDim.y * TH) {
        const int a = (int)(q / J.n), b = (int)(q - (long long)a * J.n);
        atomicAdd(&D[(long long)J.map[a] * J.dld + J.map[b]], S[(long long)a * J.sld + b]);
    }
}
}  // namespace

template <class T>
int extend_add_run(const ExtendJob* jobs, int count, int ychunks, cudaStream_t st) {
    if (count <= 0) return BDDC_OK;
    k_extend_add<T><<<dim3(count, ychunks), TH, 0, st>>>(jobs);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
template int extend_add_run<double>(const ExtendJob*, int, int, cudaStream_t);
template int extend_add_run<float>(const ExtendJob*, int, int, cudaStream_t);

template <class TD>
int gather_perm_run(const GatherJob* jobs, int count, const int* idx, int ychunks, cudaStream_t st) {
    if (count <= 0) return BDDC_OK;
    k_gather_perm<TD><<<dim3(count, ychunks), TH, 0, st>>>(jobs, idx);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
template int gather_perm_run<double>(const GatherJob*, int, const int*, int, cudaStream_t);
template int gather_perm_run<float>(const GatherJob*, int, const int*, int, cudaStream_t);

template <class TD>
int transform_run(const TBlock* blocks, int count, const int* idx, int maxn, int ychunks, cudaStream_t st) {
    if (count <= 0) return BDDC_OK;
    // Q staged in shared memory when it fits, else read from global memory (L1 / L2)
    const int qglob = (size_t)maxn * maxn * sizeof(TD) > 200 * 1024 ? 1 : 0;
    const size_t smem = qglob ? 0 : (size_t)maxn * maxn * sizeof(TD);
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_transform_right<TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_transform_left<TD, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_transform_right<TD><<<dim3(count, ychunks), TH, smem, st>>>(blocks, idx, qglob);
    bddc_note_launches(1);
    k_transform_left<TD, TD><<<dim3(count, ychunks), TH, smem, st>>>(blocks, idx, qglob);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
template int transform_run<double>(const TBlock*, int, const int*, int, int, cudaStream_t);
template int transform_run<float>(const TBlock*, int, const int*, int, int, cudaStream_t);

size_t basis_smem(int nmax, size_t elem) { return 4 * (size_t)nmax * nmax * elem; }

template <class TD>
int basis_run(const XRow* rows, int nrows, const XSub* subs, const XBlock* blks, int nmax, cudaStream_t st) {
    if (nrows <= 0) return BDDC_OK;
    const size_t smem = basis_smem(nmax, sizeof(TD));
    if (smem > 200 * 1024) {
        bddc_set_last_error("change-of-basis blocks larger than shared memory", __FILE__, __LINE__);
        return BDDC_EINVAL;
    }
    BDDC_CUDA_TRY(cudaFuncSetAttribute(k_basis<TD, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_basis<TD, TD><<<nrows, TH, smem, st>>>(rows, subs, blks, nmax);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
template int basis_run<double>(const XRow*, int, const XSub*, const XBlock*, int, cudaStream_t);
template int basis_run<float>(const XRow*, int, const XSub*, const XBlock*, int, cudaStream_t);

template <class TD>
int fill_dt_run(const DTJob* jobs, int count, const int* idx, cudaStream_t st) {
    if (count <= 0) return BDDC_OK;
    k_fill_dt<TD><<<count, TH, 0, st>>>(jobs, idx);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
template int fill_dt_run<double>(const DTJob*, int, const int*, cudaStream_t);
template int fill_dt_run<float>(const DTJob*, int, const int*, cudaStream_t);

template <class TX, class TP>
int extract_run(const ExtractJob* jobs, int count, const int* idx, double* SPi, int nPi, int ychunks,
                cudaStream_t st) {
    if (count <= 0) return BDDC_OK;
    k_extract<TX, TP><<<dim3(count, ychunks), TH, 0, st>>>(jobs, idx, SPi, nPi);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
template int extract_run<double, double>(const ExtractJob*, int, const int*, double*, int, int, cudaStream_t);
template int extract_run<float, float>(const ExtractJob*, int, const int*, double*, int, int, cudaStream_t);

int coarse_ext_run(const double* SPi, double* X, int n, cudaStream_t st) {
    if (n <= 0) return BDDC_OK;
    long long tot = 4LL * n * n;
    int g = (int)((tot + TH - 1) / TH);
    if (g > 4096) g = 4096;
    k_coarse_ext<<<g, TH, 0, st>>>(SPi, X, n);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
