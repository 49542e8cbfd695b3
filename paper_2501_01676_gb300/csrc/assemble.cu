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
// 64 threads per element (four elements per CTA), one thread per matrix
// entry.  The element matrix is scattered (FP64 atomics) into
//   * the dense local matrix A^(s) of its subdomain (FP64 or FP32 copy),
//   * the global 27-point FP64 stencil of the free dofs (refinement residual),
//   * the global load vector.
#include <cuda_runtime.h>

#include <algorithm>

#include "bddc_internal.h"

namespace {

// Reference tables of the uniform brick (one per context, in device memory).
struct AsmTables {
    double N[27 * 8];     // shape values at the Gauss points
    double G[27 * 8 * 3]; // physical gradients
    double w[27];         // weights * |J|
    double wN[27 * 8];    // w_q N_a(x_q)
    double K0[64];        // int grad phi_j . grad phi_i
    double M0[64];        // int phi_j phi_i
};
struct AsmScalars {
    int E[3];
    double h[3];
    double tau, c;
};

constexpr int ASM_EPB = 4;                 // elements per CTA (64 threads each)
constexpr int ASM_THREADS = 64 * ASM_EPB;

__device__ __forceinline__ int dof_of(const AsmScalars& P, int ix, int iy, int iz) {
    if (ix <= 0 || iy <= 0 || iz <= 0 || ix >= P.E[0] || iy >= P.E[1] || iz >= P.E[2]) return -1;
    return (ix - 1) + (P.E[0] - 1) * ((iy - 1) + (P.E[1] - 1) * (iz - 1));
}

// Persistent CTAs of four 64-thread element slots; the reference tables are
// read once per CTA into shared memory (divergent table reads then cost no
// serialisation).  Per element: nodal data (8 threads), Gauss-point data (27
// threads), the max |beta| by warp shuffles, then one thread per entry (i, j).
template <class TA>
__global__ void __launch_bounds__(ASM_THREADS) k_assemble(
    AsmScalars P, const AsmTables* __restrict__ tab, int nelem,
    const double* __restrict__ nu_elem, const double* __restrict__ beta_node,
    const double* __restrict__ f_node, const double* __restrict__ divb_node, double3 beta_const,
    const int* __restrict__ slab_of_x, const int* __restrict__ slab_of_y,
    const int* __restrict__ slab_of_z, int nsx, int nsy,
    const int* __restrict__ lut, const long long* __restrict__ lut_off,
    const int* __restrict__ box0, const int* __restrict__ boxn,
    TA* __restrict__ Aloc, const long long* __restrict__ a_off, const int* __restrict__ a_ld,
    double* __restrict__ stencil, double* __restrict__ F, const double* __restrict__ gnode) {
    __shared__ AsmTables tb;
    __shared__ double sb[ASM_EPB][8][3], sf[ASM_EPB][8], sdv[ASM_EPB][8];
    __shared__ double bg[ASM_EPB][27][8], Lp[ASM_EPB][27][8], wbg[ASM_EPB][27][8], cN[ASM_EPB][27][8];
    __shared__ double wf[ASM_EPB][27];
    __shared__ double Pm[ASM_EPB][8][9];
    __shared__ double Gs[ASM_EPB][36], Rs[ASM_EPB][36], Fs[ASM_EPB][8][2];
    __shared__ double bmx[ASM_EPB][2];
    {
        const double* src = reinterpret_cast<const double*>(tab);
        double* dst = reinterpret_cast<double*>(&tb);
        for (int q = threadIdx.x; q < (int)(sizeof(AsmTables) / sizeof(double)); q += ASM_THREADS) dst[q] = src[q];
    }
    __syncthreads();
    const int slot = threadIdx.x >> 6, t = threadIdx.x & 63, lane = threadIdx.x & 31;
    const int Ex = P.E[0], Ey = P.E[1];
    const double hK = sqrt(P.h[0] * P.h[0] + P.h[1] * P.h[1] + P.h[2] * P.h[2]);
    for (int e0 = blockIdx.x * ASM_EPB; e0 < nelem; e0 += gridDim.x * ASM_EPB) {
        const int e = e0 + slot;
        const bool act = e < nelem;
        const int ex = act ? e % Ex : 0, ey = act ? (e / Ex) % Ey : 0, ez = act ? e / (Ex * Ey) : 0;
        if (act && t < 8) {
            const int ix = ex + (t & 1), iy = ey + ((t >> 1) & 1), iz = ez + ((t >> 2) & 1);
            const long long nd = ix + (long long)(Ex + 1) * (iy + (long long)(Ey + 1) * iz);
            if (beta_node) {
                sb[slot][t][0] = beta_node[3 * nd];
                sb[slot][t][1] = beta_node[3 * nd + 1];
                sb[slot][t][2] = beta_node[3 * nd + 2];
            } else {
                sb[slot][t][0] = beta_const.x;
                sb[slot][t][1] = beta_const.y;
                sb[slot][t][2] = beta_const.z;
            }
            sf[slot][t] = f_node ? f_node[nd] : 0.0;
            sdv[slot][t] = divb_node ? divb_node[nd] : 0.0;
        }
        __syncthreads();
        // Gauss point q = t: beta, f, c~, beta.grad phi_a, L phi_a, w_q L phi_a
        double bm = 0.0;
        if (act && t < 27) {
            double b0 = 0, b1 = 0, b2 = 0, ff = 0, dd = 0;
            for (int a = 0; a < 8; ++a) {
                const double n = tb.N[t * 8 + a];
                b0 += n * sb[slot][a][0];
                b1 += n * sb[slot][a][1];
                b2 += n * sb[slot][a][2];
                ff += n * sf[slot][a];
                dd += n * sdv[slot][a];
            }
            const double w = tb.w[t];
            wf[slot][t] = w * ff;
            const double cqv = w * (P.c - 0.5 * dd);
            for (int a = 0; a < 8; ++a) {
                const double* g = &tb.G[(t * 8 + a) * 3];
                const double v = b0 * g[0] + b1 * g[1] + b2 * g[2];
                bg[slot][t][a] = v;
                Lp[slot][t][a] = v + P.c * tb.N[t * 8 + a];
                wbg[slot][t][a] = w * v;
                cN[slot][t][a] = cqv * tb.N[t * 8 + a];
            }
            bm = b0 * b0 + b1 * b1 + b2 * b2;
        } else if (act && t >= 32 && t < 40) {
            const int a = t - 32;
            bm = sb[slot][a][0] * sb[slot][a][0] + sb[slot][a][1] * sb[slot][a][1] + sb[slot][a][2] * sb[slot][a][2];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
        if (lane == 0) bmx[slot][t >> 5] = bm;
        __syncthreads();
        // The 27-point sums of the element matrix and load vector as work units of
        // one sum each, spread over all the CTA's threads (unit u: u < 160 G_ij,
        // 160 <= u < 320 the reaction R_ij, both on the upper triangle i <= j of the
        // symmetric parts; 320 <= u < 576 P_ij; 576 <= u < 640 the load sums):
        //   G_ij = sum_q w (beta.grad phi_i)(beta.grad phi_j),  R_ij = sum_q w c~ phi_i phi_j,
        //   P_ij = sum_q w phi_i beta.grad phi_j,  F1_i = sum_q w f phi_i,  F2_i = sum_q w f L phi_i.
        // With L phi = beta.grad phi + c phi the GLS sum is exactly
        //   sum_q w L phi_i L phi_j = G_ij + c (P_ij + P_ji) + c^2 M0_ij.
        for (int u = threadIdx.x; u < 640; u += ASM_THREADS) {
            double acc = 0.0;
            if (u < 320) {
                const bool gk = u < 160;
                const int v = gk ? u : u - 160;
                const int sl = v / 40, e36 = v - sl * 40;
                if (e36 >= 36 || e0 + sl >= nelem || (!gk && !divb_node)) continue;
                // packed upper triangle: e36 -> (i, j), i <= j
                int i = 0, r = e36;
                while (r >= 8 - i) { r -= 8 - i; ++i; }
                const int j = i + r;
                if (gk) {
#pragma unroll 9
                    for (int q = 0; q < 27; ++q) acc += wbg[sl][q][i] * bg[sl][q][j];
                    Gs[sl][e36] = acc;
                } else {
#pragma unroll 9
                    for (int q = 0; q < 27; ++q) acc += cN[sl][q][i] * tb.N[q * 8 + j];
                    Rs[sl][e36] = acc;
                }
            } else if (u < 576) {
                const int v = u - 320, sl = v >> 6, i = (v >> 3) & 7, j = v & 7;
                if (e0 + sl >= nelem) continue;
#pragma unroll 9
                for (int q = 0; q < 27; ++q) acc += tb.wN[q * 8 + i] * bg[sl][q][j];
                Pm[sl][i][j] = acc;
            } else {
                const int v = u - 576, sl = v >> 4, i = (v >> 1) & 7, part = v & 1;
                if (e0 + sl >= nelem) continue;
                if (part == 0) {
#pragma unroll 9
                    for (int q = 0; q < 27; ++q) acc += wf[sl][q] * tb.N[q * 8 + i];
                } else {
#pragma unroll 9
                    for (int q = 0; q < 27; ++q) acc += wf[sl][q] * Lp[sl][q][i];
                }
                Fs[sl][i][part] = acc;
            }
        }
        __syncthreads();
        const int i = t >> 3, j = t & 7;      // test i, trial j
        if (act) {
            const double bmax = sqrt(fmax(bmx[slot][0], bmx[slot][1]));
            const double nu = nu_elem[e];
            const double PK = hK * bmax / (2.0 * nu);
            const double CK = (PK >= 1.0) ? P.tau * hK / (2.0 * bmax) : P.tau * hK * hK / (4.0 * nu);
            const int lo = i < j ? i : j, hi = i < j ? j : i;
            const int e36 = lo * 8 - (lo * (lo - 1)) / 2 + (hi - lo);
            const double pij = Pm[slot][i][j], pji = Pm[slot][j][i];
            const double gls = Gs[slot][e36] + P.c * (pij + pji) + P.c * P.c * tb.M0[i * 8 + j];
            const double reac = divb_node ? Rs[slot][e36] : P.c * tb.M0[i * 8 + j];
            const double acc = nu * tb.K0[i * 8 + j] + CK * gls + reac + 0.5 * (pij - pji);
            const double fl = j == 0 ? Fs[slot][i][0] + CK * Fs[slot][i][1] : 0.0;
            // node indices of the entry
            const int ix = ex + (i & 1), iy = ey + ((i >> 1) & 1), iz = ez + ((i >> 2) & 1);
            const int jx = ex + (j & 1), jy = ey + ((j >> 1) & 1), jz = ez + ((j >> 2) & 1);
            const int di = dof_of(P, ix, iy, iz), dj = dof_of(P, jx, jy, jz);
            if (di >= 0 && dj >= 0) {
                const int o = (jx - ix + 1) + 3 * (jy - iy + 1) + 9 * (jz - iz + 1);
                atomicAdd(&stencil[(long long)di * 27 + o], acc);
                // local matrix of the owning subdomain
                const int s = slab_of_x[ex] + nsx * (slab_of_y[ey] + nsy * slab_of_z[ez]);
                const int* b0 = &box0[3 * s];
                const int* bn = &boxn[3 * s];
                const int li = lut[lut_off[s] + (ix - b0[0]) + bn[0] * ((iy - b0[1]) + bn[1] * (iz - b0[2]))];
                const int lj = lut[lut_off[s] + (jx - b0[0]) + bn[0] * ((jy - b0[1]) + bn[1] * (jz - b0[2]))];
                atomicAdd(&Aloc[a_off[s] + (long long)li * a_ld[s] + lj], (TA)acc);
            }
            // Dirichlet values on the boundary node j enter the load of node i
            if (gnode && di >= 0 && dj < 0)
                atomicAdd(&F[di], -acc * gnode[jx + (long long)(Ex + 1) * (jy + (long long)(Ey + 1) * jz)]);
            if (j == 0 && di >= 0) atomicAdd(&F[di], fl);
        }
        __syncthreads();       // the slot's shared data is rewritten by the next element
    }
}

// P1 on the six Kuhn tetrahedra of each brick (Sect. 4): tetrahedron k holds the
// local nodes vid[k] = {0, 1 << p0, 1 << p0 | 1 << p1, 7} for the k-th axis
// permutation p; G its barycentric gradients, pos[k][a] the position of brick node
// a in it (-1: not a vertex), the 4-point degree-2 rule lam[q][a] with weights
// vol / 4.
struct AsmTablesP1 {
    double G[6][4][3];
    double lam[4][4];
    double vol;
    int vid[6][4];
    int pos[6][8];
};

// Brick matrices of the P1 discretisation, four bricks per CTA (64 threads each):
// (1) nodal data; (2) per (tetrahedron, point) beta, f, c~ and beta.grad lambda_a by
// linear interpolation from the tetrahedron's vertices, and per tetrahedron the
// weight C(x) from its largest vertex |beta| and h_K = the brick's diagonal; (3)
// the 96 tetrahedron matrix entries and 24 loads, each a 4-point sum; (4) one
// thread per brick entry sums the tetrahedra holding both nodes and scatters as
// for Q1 (dense A^(s), stencil, loads, Dirichlet lifting).
template <class TA>
__global__ void __launch_bounds__(ASM_THREADS) k_assemble_p1(
    AsmScalars P, const AsmTablesP1* __restrict__ tab, int nelem,
    const double* __restrict__ nu_elem, const double* __restrict__ beta_node,
    const double* __restrict__ f_node, const double* __restrict__ divb_node, double3 beta_const,
    const int* __restrict__ slab_of_x, const int* __restrict__ slab_of_y,
    const int* __restrict__ slab_of_z, int nsx, int nsy,
    const int* __restrict__ lut, const long long* __restrict__ lut_off,
    const int* __restrict__ box0, const int* __restrict__ boxn,
    TA* __restrict__ Aloc, const long long* __restrict__ a_off, const int* __restrict__ a_ld,
    double* __restrict__ stencil, double* __restrict__ F, const double* __restrict__ gnode) {
    __shared__ AsmTablesP1 tb;
    __shared__ double sb[ASM_EPB][8][3], sf[ASM_EPB][8], sdv[ASM_EPB][8], sn2[ASM_EPB][8];
    __shared__ double bgq[ASM_EPB][6][4][4], Lq[ASM_EPB][6][4][4], fq[ASM_EPB][6][4], ctq[ASM_EPB][6][4];
    __shared__ double CKt[ASM_EPB][6], Mt[ASM_EPB][6][4][4], Ft[ASM_EPB][6][4];
    {
        const int* src = reinterpret_cast<const int*>(tab);
        int* dst = reinterpret_cast<int*>(&tb);
        for (int q = threadIdx.x; q < (int)(sizeof(AsmTablesP1) / sizeof(int)); q += ASM_THREADS) dst[q] = src[q];
    }
    __syncthreads();
    const int slot = threadIdx.x >> 6, t = threadIdx.x & 63;
    const int Ex = P.E[0], Ey = P.E[1];
    const double hK = sqrt(P.h[0] * P.h[0] + P.h[1] * P.h[1] + P.h[2] * P.h[2]);
    const double w = 0.25 * tb.vol;
    for (int e0 = blockIdx.x * ASM_EPB; e0 < nelem; e0 += gridDim.x * ASM_EPB) {
        const int e = e0 + slot;
        const bool act = e < nelem;
        const int ex = act ? e % Ex : 0, ey = act ? (e / Ex) % Ey : 0, ez = act ? e / (Ex * Ey) : 0;
        if (act && t < 8) {
            const int ix = ex + (t & 1), iy = ey + ((t >> 1) & 1), iz = ez + ((t >> 2) & 1);
            const long long nd = ix + (long long)(Ex + 1) * (iy + (long long)(Ey + 1) * iz);
            double b0 = beta_const.x, b1 = beta_const.y, b2 = beta_const.z;
            if (beta_node) {
                b0 = beta_node[3 * nd];
                b1 = beta_node[3 * nd + 1];
                b2 = beta_node[3 * nd + 2];
            }
            sb[slot][t][0] = b0;
            sb[slot][t][1] = b1;
            sb[slot][t][2] = b2;
            sn2[slot][t] = b0 * b0 + b1 * b1 + b2 * b2;
            sf[slot][t] = f_node ? f_node[nd] : 0.0;
            sdv[slot][t] = divb_node ? divb_node[nd] : 0.0;
        }
        __syncthreads();
        if (act && t < 24) {
            const int k = t >> 2, q = t & 3;
            double b0 = 0, b1 = 0, b2 = 0, ff = 0, dd = 0;
            for (int a = 0; a < 4; ++a) {
                const int v = tb.vid[k][a];
                const double l = tb.lam[q][a];
                b0 += l * sb[slot][v][0];
                b1 += l * sb[slot][v][1];
                b2 += l * sb[slot][v][2];
                ff += l * sf[slot][v];
                dd += l * sdv[slot][v];
            }
            for (int a = 0; a < 4; ++a) {
                const double g = b0 * tb.G[k][a][0] + b1 * tb.G[k][a][1] + b2 * tb.G[k][a][2];
                bgq[slot][k][q][a] = g;
                Lq[slot][k][q][a] = g + P.c * tb.lam[q][a];
            }
            fq[slot][k][q] = ff;
            ctq[slot][k][q] = P.c - 0.5 * dd;
        } else if (act && t >= 32 && t < 38) {
            const int k = t - 32;
            double m2 = 0.0;
            for (int a = 0; a < 4; ++a) m2 = fmax(m2, sn2[slot][tb.vid[k][a]]);
            const double bmax = sqrt(m2), nu = nu_elem[e];
            const double PK = hK * bmax / (2.0 * nu);
            CKt[slot][k] = (PK >= 1.0) ? P.tau * hK / (2.0 * bmax) : P.tau * hK * hK / (4.0 * nu);
        }
        __syncthreads();
        if (act) {
            const double nu = nu_elem[e];
            for (int u = t; u < 120; u += 64) {
                if (u < 96) {
                    const int k = u >> 4, a = (u >> 2) & 3, b = u & 3;      // test a, trial b
                    const double* Ga = tb.G[k][a];
                    const double* Gb = tb.G[k][b];
                    double st = 0.0, re = 0.0, sk = 0.0;
                    for (int q = 0; q < 4; ++q) {
                        st += Lq[slot][k][q][b] * Lq[slot][k][q][a];
                        re += ctq[slot][k][q] * tb.lam[q][a] * tb.lam[q][b];
                        sk += bgq[slot][k][q][b] * tb.lam[q][a] - bgq[slot][k][q][a] * tb.lam[q][b];
                    }
                    Mt[slot][k][a][b] = nu * tb.vol * (Ga[0] * Gb[0] + Ga[1] * Gb[1] + Ga[2] * Gb[2]) +
                                        w * (CKt[slot][k] * st + re + 0.5 * sk);
                } else {
                    const int v = u - 96, k = v >> 2, a = v & 3;
                    double s1 = 0.0, s2 = 0.0;
                    for (int q = 0; q < 4; ++q) {
                        s1 += fq[slot][k][q] * tb.lam[q][a];
                        s2 += fq[slot][k][q] * Lq[slot][k][q][a];
                    }
                    Ft[slot][k][a] = w * (s1 + CKt[slot][k] * s2);
                }
            }
        }
        __syncthreads();
        if (act) {
            const int i = t >> 3, j = t & 7;      // test i, trial j
            double acc = 0.0, fl = 0.0;
            for (int k = 0; k < 6; ++k) {
                const int pi = tb.pos[k][i], pj = tb.pos[k][j];
                if (pi >= 0 && pj >= 0) acc += Mt[slot][k][pi][pj];
                if (j == 0 && pi >= 0) fl += Ft[slot][k][pi];
            }
            const int ix = ex + (i & 1), iy = ey + ((i >> 1) & 1), iz = ez + ((i >> 2) & 1);
            const int jx = ex + (j & 1), jy = ey + ((j >> 1) & 1), jz = ez + ((j >> 2) & 1);
            const int di = dof_of(P, ix, iy, iz), dj = dof_of(P, jx, jy, jz);
            if (di >= 0 && dj >= 0) {
                const int o = (jx - ix + 1) + 3 * (jy - iy + 1) + 9 * (jz - iz + 1);
                atomicAdd(&stencil[(long long)di * 27 + o], acc);
                const int s = slab_of_x[ex] + nsx * (slab_of_y[ey] + nsy * slab_of_z[ez]);
                const int* b0 = &box0[3 * s];
                const int* bn = &boxn[3 * s];
                const int li = lut[lut_off[s] + (ix - b0[0]) + bn[0] * ((iy - b0[1]) + bn[1] * (iz - b0[2]))];
                const int lj = lut[lut_off[s] + (jx - b0[0]) + bn[0] * ((jy - b0[1]) + bn[1] * (jz - b0[2]))];
                atomicAdd(&Aloc[a_off[s] + (long long)li * a_ld[s] + lj], (TA)acc);
            }
            if (gnode && di >= 0 && dj < 0)
                atomicAdd(&F[di], -acc * gnode[jx + (long long)(Ex + 1) * (jy + (long long)(Ey + 1) * jz)]);
            if (j == 0 && di >= 0) atomicAdd(&F[di], fl);
        }
        __syncthreads();       // the slot's shared data is rewritten by the next brick
    }
}

}  // namespace

// The P1 tables of the brick h[0] x h[1] x h[2]: the six Kuhn tetrahedra (vertex
// coordinates from the node bits), their barycentric gradients (the rows of the
// inverse transpose of the edge matrix [x1 - x0; x2 - x0; x3 - x0], the first
// gradient minus their sum), one tetrahedron's volume, and the symmetric 4-point
// rule with barycentric coordinates (5 +- 3 sqrt 5) / 20 and (5 - sqrt 5) / 20.
static void assemble_tables_p1(const HostMesh& hm, AsmTablesP1& P) {
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    double xyz[8][3];
    for (int a = 0; a < 8; ++a)
        for (int d = 0; d < 3; ++d) xyz[a][d] = ((a >> d) & 1) * hm.h[d];
    for (int k = 0; k < 6; ++k) {
        const int v1 = 1 << perm[k][0], v2 = v1 | (1 << perm[k][1]);
        const int v[4] = {0, v1, v2, 7};
        for (int a = 0; a < 8; ++a) P.pos[k][a] = -1;
        for (int a = 0; a < 4; ++a) {
            P.vid[k][a] = v[a];
            P.pos[k][v[a]] = a;
        }
        double D[3][3];
        for (int r = 0; r < 3; ++r)
            for (int d = 0; d < 3; ++d) D[r][d] = xyz[v[r + 1]][d] - xyz[0][d];
        const double det = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
                           D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                           D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
        // inverse transpose by cofactors: (D^{-T})[r][d] = cof(D)[r][d] / det
        double cof[3][3];
        for (int r = 0; r < 3; ++r)
            for (int d = 0; d < 3; ++d) {
                const int r1 = (r + 1) % 3, r2 = (r + 2) % 3, d1 = (d + 1) % 3, d2 = (d + 2) % 3;
                cof[r][d] = D[r1][d1] * D[r2][d2] - D[r1][d2] * D[r2][d1];
            }
        for (int d = 0; d < 3; ++d) P.G[k][0][d] = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int d = 0; d < 3; ++d) {
                P.G[k][r + 1][d] = cof[r][d] / det;
                P.G[k][0][d] -= cof[r][d] / det;
            }
        P.vol = fabs(det) / 6.0;
    }
    const double qa = (5.0 + 3.0 * sqrt(5.0)) / 20.0, qb = (5.0 - sqrt(5.0)) / 20.0;
    for (int q = 0; q < 4; ++q)
        for (int a = 0; a < 4; ++a) P.lam[q][a] = q == a ? qa : qb;
}

// The reference tables of the brick h[0] x h[1] x h[2]: 3-point Gauss rule per
// direction, Q1 shape values and gradients, weights, stiffness and mass; or the P1
// tables (element 1).
int assemble_tables_bytes(int element) {
    return element == 1 ? (int)sizeof(AsmTablesP1) : (int)sizeof(AsmTables);
}
void assemble_tables(const HostMesh& hm, void* out, int element) {
    if (element == 1) {
        assemble_tables_p1(hm, *reinterpret_cast<AsmTablesP1*>(out));
        return;
    }
    AsmTables& P = *reinterpret_cast<AsmTables*>(out);
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
}

template <class TA>
int assemble_launch(const HostMesh& hm, double tau, double c, const void* tables, const double* nu,
                    const double* beta, const double* f, const double* divb, const double bconst[3],
                    const int* slab_x, const int* slab_y, const int* slab_z, const int* lut,
                    const long long* lut_off, const int* box0, const int* boxn, TA* Aloc,
                    const long long* a_off, const int* a_ld, double* stencil, double* F, const double* gnode,
                    int element, cudaStream_t st) {
    AsmScalars P;
    for (int d = 0; d < 3; ++d) {
        P.E[d] = hm.E[d];
        P.h[d] = hm.h[d];
    }
    P.tau = tau;
    P.c = c;
    double3 bc = make_double3(bconst[0], bconst[1], bconst[2]);
    int dev = 0, nsm = 0, occ = 0;
    BDDC_CUDA_TRY(cudaGetDevice(&dev));
    BDDC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (element == 1)
        BDDC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_assemble_p1<TA>, ASM_THREADS, 0));
    else
        BDDC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_assemble<TA>, ASM_THREADS, 0));
    const long long groups = ((long long)hm.nelem + ASM_EPB - 1) / ASM_EPB;
    const int grid = (int)std::max(1LL, std::min(groups, (long long)nsm * std::max(occ, 1)));
    if (element == 1)
        k_assemble_p1<TA><<<grid, ASM_THREADS, 0, st>>>(P, (const AsmTablesP1*)tables, hm.nelem, nu, beta, f, divb,
                                                        bc, slab_x, slab_y, slab_z, hm.nsub[0], hm.nsub[1], lut,
                                                        lut_off, box0, boxn, Aloc, a_off, a_ld, stencil, F, gnode);
    else
        k_assemble<TA><<<grid, ASM_THREADS, 0, st>>>(P, (const AsmTables*)tables, hm.nelem, nu, beta, f, divb, bc,
                                                     slab_x, slab_y, slab_z, hm.nsub[0], hm.nsub[1], lut, lut_off,
                                                     box0, boxn, Aloc, a_off, a_ld, stencil, F, gnode);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

template int assemble_launch<double>(const HostMesh&, double, double, const void*, const double*, const double*,
                                     const double*, const double*, const double*, const int*, const int*,
                                     const int*, const int*, const long long*, const int*, const int*, double*,
                                     const long long*, const int*, double*, double*, const double*, int,
                                     cudaStream_t);
template int assemble_launch<float>(const HostMesh&, double, double, const void*, const double*, const double*,
                                    const double*, const double*, const double*, const int*, const int*,
                                    const int*, const int*, const long long*, const int*, const int*, float*,
                                    const long long*, const int*, double*, double*, const double*, int,
                                     cudaStream_t);

// Local index of every node of each subdomain's box (x fastest): the interior
// dofs first, in box order, then the interface dofs in box order, -1 for nodes on
// the Dirichlet boundary: the order of the subdomain's dof list.  Interior ranks
// follow from the position in the interior sub-box; interface ranks from a
// block-wide prefix count over the box, in tiles of LUT_THREADS x LUT_PER nodes
// (thread t takes LUT_PER consecutive nodes).  One CTA per subdomain.
constexpr int LUT_THREADS = 256, LUT_PER = 4;
__global__ void __launch_bounds__(LUT_THREADS) k_build_lut(int Ex, int Ey, int Ez, const int* __restrict__ box0,
                                                           const int* __restrict__ boxn,
                                                           const long long* __restrict__ lut_off, int* __restrict__ lut) {
    const int s = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int b0x = box0[3 * s], b0y = box0[3 * s + 1], b0z = box0[3 * s + 2];
    const int nx = boxn[3 * s], ny = boxn[3 * s + 1], nz = boxn[3 * s + 2];
    const long long nn = (long long)nx * ny * nz;
    const int nI = max(nx - 2, 0) * max(ny - 2, 0) * max(nz - 2, 0);
    int* L = lut + lut_off[s];
    __shared__ int wsum[LUT_THREADS / 32];
    int carry = 0;
    for (long long base = 0; base < nn; base += (long long)LUT_THREADS * LUT_PER) {
        int kind[LUT_PER], cnt = 0;
        int ix[LUT_PER], iy[LUT_PER], iz[LUT_PER];
#pragma unroll
        for (int u = 0; u < LUT_PER; ++u) {
            const long long q = base + (long long)t * LUT_PER + u;
            kind[u] = 0;
            ix[u] = iy[u] = iz[u] = 0;
            if (q < nn) {
                ix[u] = (int)(q % nx);
                iy[u] = (int)((q / nx) % ny);
                iz[u] = (int)(q / ((long long)nx * ny));
                const int gx = b0x + ix[u], gy = b0y + iy[u], gz = b0z + iz[u];
                const bool dir = gx <= 0 || gy <= 0 || gz <= 0 || gx >= Ex || gy >= Ey || gz >= Ez;
                const bool in = ix[u] > 0 && ix[u] < nx - 1 && iy[u] > 0 && iy[u] < ny - 1 && iz[u] > 0 && iz[u] < nz - 1;
                kind[u] = dir ? 0 : (in ? 1 : 2);
                cnt += kind[u] == 2;
            }
        }
        // exclusive prefix of the interface counts over the block
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        int wpre = 0, tot = 0;
        for (int w = 0; w < LUT_THREADS / 32; ++w) {
            wpre += w < wid ? wsum[w] : 0;
            tot += wsum[w];
        }
        int r = carry + wpre + incl - cnt;
#pragma unroll
        for (int u = 0; u < LUT_PER; ++u) {
            const long long q = base + (long long)t * LUT_PER + u;
            if (q >= nn) continue;
            if (kind[u] == 1) L[q] = (ix[u] - 1) + (nx - 2) * ((iy[u] - 1) + (ny - 2) * (iz[u] - 1));
            else if (kind[u] == 2) L[q] = nI + r++;
            else L[q] = -1;
        }
        carry += tot;
        __syncthreads();      // wsum is rewritten by the next tile
    }
}

int build_lut_run(const HostMesh& hm, const int* box0, const int* boxn, const long long* lut_off, int* lut,
                  cudaStream_t st) {
    if (hm.nsd <= 0) return BDDC_OK;
    k_build_lut<<<hm.nsd, LUT_THREADS, 0, st>>>(hm.E[0], hm.E[1], hm.E[2], box0, boxn, lut_off, lut);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

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

// ---------------------------------------------------------------------------
// Input check of the coefficient arrays (Sect. 2 assumes nu > 0)
// ---------------------------------------------------------------------------
namespace {
__global__ void k_validate(const double* __restrict__ nu, long long nelem, const double* __restrict__ beta,
                           const double* __restrict__ f, const double* __restrict__ divb,
                           const double* __restrict__ g, long long nnodes, int* __restrict__ bad) {
    int b = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nelem; e += stride)
        if (!(nu[e] > 0.0) || !isfinite(nu[e])) b = 1;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnodes; q += stride) {
        if (beta && (!isfinite(beta[3 * q]) || !isfinite(beta[3 * q + 1]) || !isfinite(beta[3 * q + 2]))) b = 1;
        if (f && !isfinite(f[q])) b = 1;
        if (divb && !isfinite(divb[q])) b = 1;
        if (g && !isfinite(g[q])) b = 1;
    }
    if (b) atomicOr(bad, 1);
}
}  // namespace

int validate_coeffs_run(const double* nu, long long nelem, const double* beta, const double* f, const double* divb,
                        const double* g, long long nnodes, int* dflag, cudaStream_t st) {
    BDDC_CUDA_TRY(cudaMemsetAsync(dflag, 0, sizeof(int), st));
    const long long n = std::max(nelem, nnodes);
    const int blocks = (int)std::min<long long>((n + 255) / 256, 1184);
    k_validate<<<std::max(blocks, 1), 256, 0, st>>>(nu, nelem, beta, f, divb, g, nnodes, dflag);
    bddc_note_launches(1);
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}
