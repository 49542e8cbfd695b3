// Job descriptors of the face and edge GEP kernels (one CTA per job).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#define EDGE_MAX_SUBS 4
#define FACE_NMAX 256          // largest face (dofs) of the face GEP kernel

struct FaceJob {
    int n;                    // face dofs n_F
    int mode;                 // 0 GEP, 1 all primal, 2 no face constraints
    double theta;             // Theta_F
    const double* Si;         // packed S^(i) (FP64), leading dim ldi
    const double* Sj;
    int ldi, ldj;
    const int* pi;            // local interface positions of the face in i / j
    const int* pj;
    const double* Bti;        // Schur complement of B^(i) onto F (ld ldbi)
    const double* Btj;
    int ldbi, ldbj;
    void* work;               // face_work_doubles(n) (+ face_eig_doubles(n)) elements of the kernel precision
    double* Q;                // out: n x n orthogonal, first k columns primal (row-major)
    double* DQi;              // out: D^(i) Q
    double* DQj;              // out: D^(j) Q
    double* lambda;           // out: n eigenvalues, largest first (NaN padded)
    int* neig;
    int* k;                   // out: primal count
};

struct EdgeJob {
    int n;                    // edge dofs n_E
    int m;                    // subdomains sharing the edge
    int nH;                   // prior primal unknowns (union, shared ones identified)
    int mode;                 // 0 GEP on prior-selected primal constraints, 1 all primal,
                              // 2 no edge constraints, 3 conventional edge GEP
    double theta;             // Theta_E
    const double* S[EDGE_MAX_SUBS];    // packed S^(k) in sorted n(E) order
    int ldS[EDGE_MAX_SUBS];
    const int* pos[EDGE_MAX_SUBS];     // local positions of the edge in S^(k)
    const void* Bt[EDGE_MAX_SUBS];     // Schur complement of B^(k) onto [E, H_k] (kernel precision)
    int ldBt[EDGE_MAX_SUBS];
    int h[EDGE_MAX_SUBS];              // |H_k|
    const int* hmap[EDGE_MAX_SUBS];    // H_k coordinate -> union index
    void* work;
    double* Q;                // out: n x n
    double* DQ[EDGE_MAX_SUBS];// out: D^(k) Q
    double* lambda;           // out: (m-1) n eigenvalues (mode 3: n), NaN padded
    double* BBout;            // out: B~~_E ((m-1) n square) for parity checks
    int* neig;
    int* k;
};

__host__ __device__ size_t face_work_doubles(int n);
// Elements of the two eigen-work matrices of a face of n dofs; face_eig_global<T>
// tells whether the kernel keeps them in global memory (then every job's
// workspace holds face_work_doubles(n) + face_eig_doubles(n) elements).
size_t face_eig_doubles(int n);
template <class T>
bool face_eig_global(int maxn);
size_t edge_work_doubles(int n, int m, int nH);
template <class T>
int face_run(const FaceJob* jobs_dev, int count, int maxn, int* err, cudaStream_t st);
template <class T>
int edge_run(const EdgeJob* jobs_dev, int count, int maxnw, int maxnz, size_t max_work, int* err, cudaStream_t st);
