// Job descriptors of the setup data-movement kernels.
#pragma once
#include <cuda_runtime.h>

struct CopyJob {            // dst[r][c] = scale * src[r0 + r][c0 + c]
    const void* src;
    long long sld;
    int r0, c0, rows, cols;
    void* dst;
    long long dld;
    double scale;
};

struct GatherJob {          // dst[a][b] = S[p_a][p_b] (sym: symmetric part)
    const double* src;      // FP64 source, or NULL: srcT (the destination precision)
    long long sld;
    int n;
    int perm_off;
    int sym;
    void* dst;
    long long dld;
    const void* srcT;
};

struct TBlock {             // one entity block of one subdomain's change of basis
    const double* src;      // packed S^(i) (FP64)
    long long sld;
    int sym;                // use the symmetric part B^(i)
    void* y;                // n_B x n_B scratch of the subdomain (precision of the output)
    long long yld;
    int n;                  // entity size
    int pos_off;            // local interface positions of the entity
    int perm_off;           // transformed coordinate -> output index (n_B entries, -1 drop)
    const double* Q;        // n x n row-major, columns = new basis (NULL when identity)
    int identity;
    int nrows;              // n_B
    void* dst;
    long long dld;
};

struct DTJob {              // D_X^(i) Q_X blocks of the extended matrix
    int n, nB;
    int pos_off, perm_off;
    const double* DQ;       // n x n, or NULL for a vertex (scalar)
    double scalar;
    void* dst;
    long long dld;
};

struct ExtractJob {
    const void* X;
    long long xld;
    int nB, np;
    int rpi_off;            // global primal index of each local primal coordinate
    void* MA;               // [P ; Psi^T D^T]  ((nB + np) x nB)
    long long ald;
    void* MC;               // D Phi stored transposed (np x nB)
    long long cld;
};

// Change of basis by blocks: for one subdomain the output is
//   dst[perm[pX[l]]][perm[pY[m]]] = sum_{a,b} QX[a][l] S[pX[a]][pY[b]] QY[b][m]
// over all pairs of blocks (X, Y) of the subdomain (S or its symmetric part);
// a block without Q is the identity (several identity entities may share one).
struct XBlock {
    int n;
    const int* pos;         // n local interface positions (device)
    const double* Q;        // n x n row-major, columns = new basis; NULL = identity
};
struct XSub {
    const double* src;      // packed S^(i) (FP64)
    long long sld;
    int sym;
    int nblk, blk_off;      // the subdomain's blocks in the block table
    const int* perm;        // n_B entries: transformed coordinate -> output index (-1: drop)
    void* dst;
    long long dld;
};
struct XRow {               // one CTA: the rows of one block of one subdomain
    int sub, blk;
};

// Extend-add of one child box's Schur complement into its subdomain's matrix:
//   dst[map[a]][map[b]] += src[a][b]  (a, b < n; several children add into the
// same separator and interface entries, so the adds are atomic).
struct ExtendJob {
    const void* src;        // the child's S (kernel precision), row stride sld
    long long sld;
    int n;
    const int* map;         // n subdomain-local indices (device)
    void* dst;              // the subdomain's matrix (kernel precision)
    long long dld;
};
template <class T>
int extend_add_run(const ExtendJob* jobs, int count, int ychunks, cudaStream_t st);

template <class TD>
int basis_run(const XRow* rows, int nrows, const XSub* subs, const XBlock* blks, int nmax, cudaStream_t st);
size_t basis_smem(int nmax, size_t elem);

template <class TS, class TD>
int copy_blocks_run(const CopyJob* jobs, int count, int ychunks, cudaStream_t st);
template <class TD>
int gather_perm_run(const GatherJob* jobs, int count, const int* idx, int ychunks, cudaStream_t st);
template <class TD>
int transform_run(const TBlock* blocks, int count, const int* idx, int maxn, int ychunks, cudaStream_t st);
template <class TD>
int fill_dt_run(const DTJob* jobs, int count, const int* idx, cudaStream_t st);
template <class TX, class TP>
int extract_run(const ExtractJob* jobs, int count, const int* idx, double* SPi, int nPi, int ychunks,
                cudaStream_t st);
int coarse_ext_run(const double* SPi, double* X, int n, cudaStream_t st);
