// Element assembly of the stabilised Q1 system (Sect. 2).
//
// a(u,v) = b(u,v) + z(u,v),
//   b(u,v) = int nu grad u.grad v + C(x) Lu Lv + c~ u v,
//   z(u,v) = 1/2 int (beta.grad u v - beta.grad v u),
//   g(v)   = int f v + C(x) f Lv,
// with P_K = h_K |beta|_{K,inf} / (2 nu), C = tau h_K / (2 |beta|) when
// P_K >= 1 else tau h_K^2 / (4 nu), c~ = c - div(beta)/2.  For Q1 with
// elementwise-constant nu, L phi = beta.grad phi + c phi (the second-order
// term vanishes).  beta, f, div(beta) are nodal and interpolated trilinearly;
// |beta|_{K,inf} is the maximum over the 8 vertices and the 27 Gauss points.
// h_K = sqrt(hx^2 + hy^2 + hz^2).  Entry (i,j) = a(phi_j, phi_i).
//
// One block of 64 threads per element, one thread per matrix entry.  The
// element matrix is scattered (FP64 atomics) into
//   * the dense local matrix A^(s) of its subdomain (FP64 or FP32 copy),
//   * the global 27-point FP64 stencil of the free dofs (refinement residual),
//   * the global load vector.
#include <cuda_runtime.h>

#include "bddc_internal.h"

namespace {

struct AsmParams {
    int E[3];
    double h[3];
    double tau, c;
    double K0[64];        // reference stiffness int grad phi_j . grad phi_i on an h-box
    double M0[64];        // reference mass
    double N[27 * 8];     // shape values at the Gauss points
    double G[27 * 8 * 3]; // physical gradients
    double w[27];         // weights * |J|
    double wN[27 * 8];    // w_q N_a(x_q)
};

__constant__ AsmParams cP;

__device__ __forceinline__ int dof_of(int ix, int iy, int iz) {
    if (ix <= 0 || iy <= 0 || iz <= 0 || ix >= cP.E[0] || iy >= cP.E[1] || iz >= cP.E[2]) return -1;
    return (ix - 1) + (cP.E[0] - 1) * ((iy - 1) + (cP.E[1] - 1) * (iz - 1));
}

template <class TA>
__global__ void __launch_bounds__(64) k_assemble(
    const double* __restrict__ nu_elem, const double* __restrict__ beta_node,
    const double* __restrict__ f_node, const double* __restrict__ divb_node, double3 beta_const,
    const int* __restrict__ slab_of_x, const int* __restrict__ slab_of_y,
    const int* __restrict__ slab_of_z, int nsx, int nsy,
    const int* __restrict__ lut, const long long* __restrict__ lut_off,
    const int* __restrict__ box0, const int* __restrict__ boxn,
    TA* __restrict__ Aloc, const long long* __restrict__ a_off, const int* __restrict__ a_ld,
    double* __restrict__ stencil, double* __restrict__ F) {
    const int e = blockIdx.x;
    const int t = threadIdx.x;
    const int Ex = cP.E[0], Ey = cP.E[1];
    const int ex = e % Ex, ey = (e / Ex) % Ey, ez = e / (Ex * Ey);
    __shared__ double sb[8][3], sf[8], sdv[8];
    __shared__ double bg[27][8], Lp[27][8], wLp[27][8], wf[27], cq[27];
    __shared__ double P[8][9];
    __shared__ double bmax2[64];
    __shared__ double CK;
    if (t < 8) {
        int ix = ex + (t & 1), iy = ey + ((t >> 1) & 1), iz = ez + ((t >> 2) & 1);
        long long nd = ix + (long long)(Ex + 1) * (iy + (long long)(Ey + 1) * iz);
        if (beta_node) {
            sb[t][0] = beta_node[3 * nd];
            sb[t][1] = beta_node[3 * nd + 1];
            sb[t][2] = beta_node[3 * nd + 2];
        } else {
            sb[t][0] = beta_const.x;
            sb[t][1] = beta_const.y;
            sb[t][2] = beta_const.z;
        }
        sf[t] = f_node ? f_node[nd] : 0.0;
        sdv[t] = divb_node ? divb_node[nd] : 0.0;
    }
    __syncthreads();
    // per Gauss point q (thread q): beta, f, c~, beta.grad phi_a, L phi_a, w_q L phi_a
    double bm = 0.0;
    if (t < 27) {
        double b0 = 0, b1 = 0, b2 = 0, ff = 0, dd = 0;
        for (int a = 0; a < 8; ++a) {
            double n = cP.N[t * 8 + a];
            b0 += n * sb[a][0];
            b1 += n * sb[a][1];
            b2 += n * sb[a][2];
            ff += n * sf[a];
            dd += n * sdv[a];
        }
        const double w = cP.w[t];
        wf[t] = w * ff;
        cq[t] = w * (cP.c - 0.5 * dd);
        for (int a = 0; a < 8; ++a) {
            const double* g = &cP.G[(t * 8 + a) * 3];
            double v = b0 * g[0] + b1 * g[1] + b2 * g[2];
            double l = v + cP.c * cP.N[t * 8 + a];
            bg[t][a] = v;
            Lp[t][a] = l;
            wLp[t][a] = w * l;
        }
        bm = b0 * b0 + b1 * b1 + b2 * b2;
    } else if (t >= 32 && t < 40) {
        int a = t - 32;
        bm = sb[a][0] * sb[a][0] + sb[a][1] * sb[a][1] + sb[a][2] * sb[a][2];
    }
    bmax2[t] = bm;
    __syncthreads();
    if (t == 0) {
        double m2 = 0.0;
        for (int q = 0; q < 64; ++q) m2 = fmax(m2, bmax2[q]);
        double bmax = sqrt(m2);
        double hK = sqrt(cP.h[0] * cP.h[0] + cP.h[1] * cP.h[1] + cP.h[2] * cP.h[2]);
        double nu = nu_elem[e];
        double PK = hK * bmax / (2.0 * nu);
        CK = (PK >= 1.0) ? cP.tau * hK / (2.0 * bmax) : cP.tau * hK * hK / (4.0 * nu);
    }
    const int i = t >> 3, j = t & 7;      // test i, trial j
    // GLS part sum_q w L phi_j L phi_i and P_ij = sum_q w N_i beta.grad phi_j
    double gls = 0.0, pij = 0.0, reac = 0.0;
#pragma unroll 9
    for (int q = 0; q < 27; ++q) {
        gls += wLp[q][j] * Lp[q][i];
        pij += cP.wN[q * 8 + i] * bg[q][j];
    }
    if (divb_node) {
        for (int q = 0; q < 27; ++q) reac += cq[q] * cP.N[q * 8 + i] * cP.N[q * 8 + j];
    } else {
        reac = cP.c * cP.M0[i * 8 + j];
    }
    P[i][j] = pij;
    __syncthreads();
    const double acc = nu_elem[e] * cP.K0[i * 8 + j] + CK * gls + reac + 0.5 * (pij - P[j][i]);
    double fl = 0.0;
    if (j == 0)
        for (int q = 0; q < 27; ++q) fl += wf[q] * (cP.N[q * 8 + i] + CK * Lp[q][i]);
    // node indices of the entry
    const int ix = ex + (i & 1), iy = ey + ((i >> 1) & 1), iz = ez + ((i >> 2) & 1);
    const int jx = ex + (j & 1), jy = ey + ((j >> 1) & 1), jz = ez + ((j >> 2) & 1);
    const int di = dof_of(ix, iy, iz), dj = dof_of(jx, jy, jz);
    if (di >= 0 && dj >= 0) {
        int o = (jx - ix + 1) + 3 * (jy - iy + 1) + 9 * (jz - iz + 1);
        atomicAdd(&stencil[(long long)di * 27 + o], acc);
        // local matrix of the owning subdomain
        int s = slab_of_x[ex] + nsx * (slab_of_y[ey] + nsy * slab_of_z[ez]);
        const int* b0 = &box0[3 * s];
        const int* bn = &boxn[3 * s];
        int li = lut[lut_off[s] + (ix - b0[0]) + bn[0] * ((iy - b0[1]) + bn[1] * (iz - b0[2]))];
        int lj = lut[lut_off[s] + (jx - b0[0]) + bn[0] * ((jy - b0[1]) + bn[1] * (jz - b0[2]))];
        atomicAdd(&Aloc[a_off[s] + (long long)li * a_ld[s] + lj], (TA)acc);
    }
    if (j == 0 && di >= 0) atomicAdd(&F[di], fl);
}

double host_N(int a, double x, double y, double z) {
    double fx = (a & 1) ? x : 1 - x, fy = ((a >> 1) & 1) ? y : 1 - y, fz = ((a >> 2) & 1) ? z : 1 - z;
    return fx * fy * fz;
}

}  // namespace

// Fill the constant tables (Gauss rule, shape tables, reference stiffness).
int assemble_init(const HostMesh& hm, double tau, double c) {
    AsmParams P;
    for (int d = 0; d < 3; ++d) {
        P.E[d] = hm.E[d];
        P.h[d] = hm.h[d];
    }
    P.tau = tau;
    P.c = c;
    const double r = sqrt(3.0 / 5.0);
    const double xg[3] = {0.5 - 0.5 * r, 0.5, 0.5 + 0.5 * r};
    const double wg[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    const double det = hm.h[0] * hm.h[1] * hm.h[2];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i) {
                int q = i + 3 * j + 9 * k;
                double p[3] = {xg[i], xg[j], xg[k]};
                P.w[q] = wg[i] * wg[j] * wg[k] * det;
                for (int a = 0; a < 8; ++a) {
                    int bits[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
                    double f1[3], df[3];
                    for (int d = 0; d < 3; ++d) {
                        f1[d] = bits[d] ? p[d] : 1.0 - p[d];
                        df[d] = bits[d] ? 1.0 : -1.0;
                    }
                    P.N[q * 8 + a] = f1[0] * f1[1] * f1[2];
                    P.G[(q * 8 + a) * 3 + 0] = df[0] * f1[1] * f1[2] / hm.h[0];
                    P.G[(q * 8 + a) * 3 + 1] = f1[0] * df[1] * f1[2] / hm.h[1];
                    P.G[(q * 8 + a) * 3 + 2] = f1[0] * f1[1] * df[2] / hm.h[2];
                }
            }
    for (int q = 0; q < 27; ++q)
        for (int a = 0; a < 8; ++a) P.wN[q * 8 + a] = P.w[q] * P.N[q * 8 + a];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            double k0 = 0.0, m0 = 0.0;
            for (int q = 0; q < 27; ++q) {
                const double* gi = &P.G[(q * 8 + i) * 3];
                const double* gj = &P.G[(q * 8 + j) * 3];
                k0 += P.w[q] * (gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2]);
                m0 += P.w[q] * P.N[q * 8 + i] * P.N[q * 8 + j];
            }
            P.K0[i * 8 + j] = k0;
            P.M0[i * 8 + j] = m0;
        }
    (void)host_N;
    BDDC_CUDA_TRY(cudaMemcpyToSymbol(cP, &P, sizeof(P)));
    return BDDC_OK;
}

template <class TA>
int assemble_launch(const HostMesh& hm, const double* nu, const double* beta, const double* f,
                    const double* divb, const double bconst[3], const int* slab_x, const int* slab_y,
                    const int* slab_z, const int* lut, const long long* lut_off, const int* box0,
                    const int* boxn, TA* Aloc, const long long* a_off, const int* a_ld,
                    double* stencil, double* F, cudaStream_t st) {
    double3 bc = make_double3(bconst[0], bconst[1], bconst[2]);
    k_assemble<TA><<<hm.nelem, 64, 0, st>>>(nu, beta, f, divb, bc, slab_x, slab_y, slab_z, hm.nsub[0],
                                            hm.nsub[1], lut, lut_off, box0, boxn, Aloc, a_off, a_ld,
                                            stencil, F);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

template int assemble_launch<double>(const HostMesh&, const double*, const double*, const double*,
                                     const double*, const double*, const int*, const int*,
                                     const int*, const int*, const long long*, const int*,
                                     const int*, double*, const long long*, const int*, double*,
                                     double*, cudaStream_t);
template int assemble_launch<float>(const HostMesh&, const double*, const double*, const double*,
                                    const double*, const double*, const int*, const int*,
                                    const int*, const int*, const long long*, const int*,
                                    const int*, float*, const long long*, const int*, double*,
                                    double*, cudaStream_t);

// Global FP64 residual r = F - A u with the 27-point stencil (refinement).
__global__ void k_stencil_residual(const double* __restrict__ S, const double* __restrict__ u,
                                   const double* __restrict__ F, double* __restrict__ r, int fx,
                                   int fy, int fz, int nrhs, long long ld) {
    long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long n = (long long)fx * fy * fz;
    if (d >= n) return;
    int ix = (int)(d % fx), iy = (int)((d / fx) % fy), iz = (int)(d / ((long long)fx * fy));
    const double* row = S + d * 27;
    for (int c = 0; c < nrhs; ++c) {
        const double* uc = u + c * ld;
        double acc = F[c * ld + d];
        for (int o = 0; o < 27; ++o) {
            int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
            int jx = ix + ox, jy = iy + oy, jz = iz + oz;
            if (jx < 0 || jy < 0 || jz < 0 || jx >= fx || jy >= fy || jz >= fz) continue;
            acc -= row[o] * uc[jx + (long long)fx * (jy + (long long)fy * jz)];
        }
        r[c * ld + d] = acc;
    }
}

int stencil_residual(const HostMesh& hm, const double* S, const double* u, const double* F,
                     double* r, int nrhs, cudaStream_t st) {
    long long n = hm.ndof;
    int th = 256;
    k_stencil_residual<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(
        S, u, F, r, hm.E[0] - 1, hm.E[1] - 1, hm.E[2] - 1, nrhs, n);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
