// Internal declarations of libbddc (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bddc.h"

#define BDDC_CUDA_TRY(expr)                                                   \
    do {                                                                      \
        cudaError_t _e = (expr);                                              \
        if (_e != cudaSuccess) {                                              \
            bddc_set_last_error(cudaGetErrorString(_e), __FILE__, __LINE__);  \
            return BDDC_ECUDA;                                                \
        }                                                                     \
    } while (0)

#define BDDC_TRY(expr)                 \
    do {                               \
        int _r = (expr);               \
        if (_r < 0) return _r;         \
    } while (0)

void bddc_set_last_error(const char* msg, const char* file, int line);

// Host table -> device, asynchronous on st: the bytes are copied into a pinned
// staging arena of this host thread first (a copy from pageable memory would
// synchronise the stream before it starts).
int staged_upload(void* dev, const void* host, size_t bytes, cudaStream_t st);

// Process-wide count of kernels launched by the library (launches recorded
// while a stream is being captured are not counted; graph replays add their
// kernel nodes).
void bddc_note_launches(unsigned long long n);

// Optional CUDA-event timing of one kernel class (for roofline reporting).
enum { KT_NONE = 0, KT_ENGINE_UPDATE = 1, KT_ENGINE_PANEL = 2, KT_GEMV = 3, KT_FACE = 4, KT_EDGE = 5,
       KT_ASSEMBLE = 6, KT_TRANSFORM = 7, KT_TRI = 8, KT_COARSE = 9, KT_ENGINE_TASKS = 10, KT_APPLY_TASKS = 11,
       KT_LAST = 11 };
bool ktimer_on(int kind);
void ktimer_begin(int kind, cudaStream_t st);
void ktimer_end(int kind, cudaStream_t st, double flops, double bytes);

// Device-side error flags written by kernels (never trap).
enum {
    ERR_PIVOT = 1,        // zero / non-finite pivot in the batched LU
    ERR_JACOBI = 2,       // Jacobi eigen sweep cap reached
    ERR_SIZE = 4,         // a size exceeded a compiled limit
    ERR_TIMEOUT_TC = 8,   // a bounded wait for tensor-core work gave up
    ERR_TIMEOUT_ENGINE = 16,  // a bounded wait of the engine's task kernel gave up
    ERR_TIMEOUT_APPLY = 32,   // a bounded wait of the preconditioner's task kernel gave up
};

// ---------------------------------------------------------------------------
// Host description of the mesh, partition and interface classification.
// ---------------------------------------------------------------------------
struct Entity {
    int kind;                       // 0 vertex, 1 edge, 2 face
    std::vector<int> subs;          // sorted subdomain ids
    std::vector<int> dofs;          // ascending dof ids
    std::vector<std::vector<int>> pos;  // per subs[a]: local interface positions
    int k = 0;                      // primal count
    int prim_off = 0;               // first global primal index
    int slot = -1;                  // index within its kind
    double theta = 0.0;
};

struct SubInfo {
    int box0[3], box1[3];           // node-index box [box0, box1]
    int n, nI, nB;
    std::vector<int> dofs;          // local dof -> global dof (I then B)
    std::vector<int> gidx;          // local interface position -> Gamma index
    std::vector<int> ents;          // entity ids touching the subdomain
    std::vector<int> ent_slot;      // position of this subdomain in entity subs
    int max_slab;                   // largest slab element count (H/h)
};

struct HostMesh {
    int E[3], nsub[3], nsd;
    double lo[3], h[3];
    std::vector<int> off[3];
    int ndof, nelem, nnodes;
    std::vector<SubInfo> sub;
    std::vector<int> gamma;         // Gamma index -> dof
    std::vector<int> gamma_of_dof;  // dof -> Gamma index or -1
    std::vector<Entity> ent;        // vertices, edges, faces
    std::vector<int> by_kind[3];    // entity ids per kind in order
};

// The mesh in two parts: the partition, subdomain boxes and dof lists (all the
// assembly and the subdomain eliminations need), then the interface
// classification (entities, Gamma numbering, positions), which setup builds on
// the host while the GPU assembles; build_host_mesh does both.
int build_host_boxes(const bddc_mesh* mesh, const bddc_partition* part, HostMesh& hm);
int build_host_interface(HostMesh& hm);
int build_host_mesh(const bddc_mesh* mesh, const bddc_partition* part, HostMesh& hm);

// One level of nested dissection inside every subdomain: the child boxes (each
// slab of c >= 2 elements split into c/2 and c - c/2 elements) form a mesh of
// their own on the same grid (same dof numbering); every subdomain's numbering is
// rewritten to [separator dofs, interface dofs] (nI = the separators: the
// subdomain-interior nodes on a child box boundary); map[c] gives, for each
// interface dof of child c (in its own order), its index in the subdomain's new
// numbering.
struct LocalND {
    HostMesh child;
    std::vector<int> parent;                  // child -> subdomain
    std::vector<std::vector<int>> map;        // child -> subdomain-local indices of its interface dofs
};
int build_local_nd(HostMesh& hm, LocalND& nd);

// ---------------------------------------------------------------------------
// Device buffers
// ---------------------------------------------------------------------------
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
};

struct DevArena {                    // all device allocations of a context
    std::vector<void*> ptrs;
    size_t bytes = 0;
    int alloc(void** p, size_t bytes);
    void release();
};

// Largest interior (dofs strictly inside one subdomain) the condense / recover
// kernels hold in shared memory: 8192 (a 20^3 interior, H/h <= 21 per slab; the
// FP64 vector takes 64 KB).
constexpr int BDDC_MAX_INTERIOR = 8192;

// Coarse matrices up to this order are inverted by one CTA (FP32 Gauss-Jordan
// in shared memory) plus FP64 Newton-Schulz steps.
constexpr int COARSE_GJ_MAX = 128;
int coarse_inverse_small(const double* S, int n, double* X, int ldx, double* work, double* resid, int ns_steps,
                         int* err, cudaStream_t st);

// Batched partial LU (Schur complement engine) item descriptor.
template <class T>
struct EngItem {
    T* a;        // row-major matrix
    int n;       // order
    int k;       // leading rows/cols to eliminate
    int ld;      // leading dimension (elements)
};

// Trailing-update kind of the FP32 eliminations: CUDA cores, tensor cores with
// split-TF32 operands (about FP32 accuracy), tensor cores with BF16 operands.
enum { TC_NONE = 0, TC_SPLIT_TF32 = 1, TC_BF16 = 2 };

template <class T>
int engine_run(const EngItem<T>* items_dev, int count, int maxn, int maxk, T* diag_scratch,
               int* err, cudaStream_t st, const int* host_n = nullptr, const int* host_k = nullptr,
               int tensor_cores = TC_NONE);

// Scratch elements engine_run needs for `count` items eliminating up to maxk
// unknowns (FP64 if dbl).
long long engine_scratch_elems(int count, bool dbl, int maxk);

// Tensor-core (tcgen05, split TF32) trailing update of one FP32 engine panel of width <= nb.
int tc_update_run(const EngItem<float>* items_dev, int count, int maxn, int p, int nb, int* err, cudaStream_t st);
int tc_selftest_run(const float* A, const float* B, float* C, int nr, int nc, int K, int* err, cudaStream_t st);

// Generic batched gather -> GEMV -> scatter-add:  out[oidx[r]] += sum_c M[r][c] * in[iidx[c]]
struct GemvItem {
    long long moff;      // element offset of the matrix in the pool
    int rows, cols, ld;
    int iidx_off;        // offset of the gather index list (cols entries)
    int oidx_off;        // offset of the scatter index list (rows entries)
    int row0;            // first row handled by this work item
    int nrows;           // rows handled by this work item
    int col0;            // first column of this item's column slice
    int ncols;           // columns of the slice (<= the kernel's staging limit)
};

template <class T>
int gemv_run(const T* pool, const GemvItem* items_dev, int nitems, const int* idx,
             const double* in, double* out, int maxcols, int nrhs, int in_ld, int out_ld,
             cudaStream_t st, const int* skip_flag, double bytes = 0.0);

// Same product for tall, narrow operators stored transposed (ld = stride of a column).
template <class T>
int gemv_t_run(const T* pool, const GemvItem* items_dev, int nitems, const int* idx, const double* in,
               double* out, int nrhs, int in_ld, int out_ld, cudaStream_t st, const int* skip, double bytes);

// ---------------------------------------------------------------------------
// Coarse problem by nested dissection of the subdomain grid (coarse_plan.cpp,
// coarse_nd.cu).  Front a eliminates its n own primal unknowns; its boundary
// holds b unknowns of ancestor fronts.  The extended front
//   [[F11, F12, -I], [F21, F22, 0], [I, 0, 0]]     (order N = 2n + b)
// loses its n leading unknowns in the elimination engine, which leaves
//   [[F22 - F21 F11^-1 F12, F21 F11^-1], [-F11^-1 F12, F11^-1]]
// in its trailing block: the update added into the parent, the forward-sweep
// operator and the backward-sweep operator.
// ---------------------------------------------------------------------------
struct NDFront {
    int n, b;              // own / boundary unknowns
    int N, ld;             // extended order and its leading dimension
    long long foff;        // offset of the extended front in the front pool
    long long wf_off;      // forward operator -F21 F11^-1 (b x n, leading dim wf_ld), operator pool
    long long wb_off;      // backward operator [-F11^-1 F12 | F11^-1] (n x (b + n), leading dim wb_ld)
    int wf_ld, wb_ld;
    int vars_off;          // index pool: n + b global primal indices (own, then boundary)
    int map_off;           // index pool: b positions in the parent's front (-1: root)
    int parent;            // -1: root
    int height, depth;     // height: 0 at the leaves; depth: 0 at the roots
};

struct NDPlan {
    int nPi = 0;
    std::vector<NDFront> fr;                      // pre-order: parents before their subtrees
    std::vector<std::vector<int>> by_height;      // fronts per height (factorisation, forward sweep)
    std::vector<std::vector<int>> by_depth;       // fronts per depth (backward sweep)
    std::vector<int> idx;                         // index pool
    long long fpool = 0, opool = 0;               // elements of the front and operator pools
    std::vector<std::vector<GemvItem>> fwd, bwd;  // solve items per height / per depth
    double flops = 0.0;                           // factorisation flops (extended fronts)
    double bytes_solve = 0.0;                     // algorithmic bytes of one solve
};

// Host symbolic plan from the entities' primal counts and offsets (HostMesh).
int nd_plan(const HostMesh& hm, int nPi, NDPlan& P);
// Row and column extent of one sweep work item.
constexpr int ND_ITEM_ROWS = 16, ND_ITEM_COLS = 256;

// One CTA row-slice of a front: rows [row0, row0 + nrows) of front `front`.
struct NDRowJob {
    int front, row0, nrows;
};
// Fill the extended fronts of the jobs from the dense coarse matrix S (nPi x nPi, FP64).
int nd_fill_run(const NDFront* fr_dev, const NDRowJob* jobs, int njobs, const int* idx, const double* S, int nPi,
                double* F, cudaStream_t st);
// Add the trailing (update) blocks of the child fronts of the jobs (rows of the
// child's b x b update) into their parents' fronts.
int nd_add_run(const NDFront* fr_dev, const NDRowJob* jobs, int njobs, const int* idx, double* F, cudaStream_t st);

// ---------------------------------------------------------------------------
// M^-1 r as one persistent launch (apply_tasks.cu): work items in topological
// order with completion counters.
// ---------------------------------------------------------------------------
enum { AP_LOCAL = 0,    // rows of [P_i ; Psi_i^T D_i^T]: r -> zc (local part, coarse restriction)
       AP_SWEEP = 1,    // nested-dissection sweep operator (FP64): y2 -> y2, index pool B
       AP_DENSE = 2,    // explicit coarse inverse (FP64): y -> x inside y2
       AP_PROLONG = 3   // D_i Phi_i stored transposed: x -> zc
};
// counters: [0] next coarse-queue item, [1] abort, [2] restriction items done,
// [3] coarse-solve items done, [4] next local-queue item, [5] next restriction
// item, then per front: forward items of its children done, its backward items done
enum { AP_CTR_NEXT = 0, AP_CTR_ABORT = 1, AP_CTR_LOCAL = 2, AP_CTR_COARSE = 3, AP_CTR_NEXT_LOCAL = 4,
       AP_CTR_NEXT_RES = 5, AP_CTR_FRONTS = 6 };
struct ApTask {
    GemvItem it;
    int kind;
    int w0, t0, w1, t1;    // wait until ctr[w] >= t (w < 0: no wait)
    int s0, s1;            // ctr[s] += 1 when done (s < 0: none)
};
template <class T>
int apply_tasks_blocks();
// One CTA runs the one-launch apply's bounded wait on a counter nothing
// increments, with `limit` polls; *timed_out = 1 when it gave up as it must.
int wait_selftest_run(long long limit, int* timed_out);
// Device check of the coefficient arrays (nu > 0 and finite; beta, f, div beta
// finite; NULL arrays are skipped): *flag_dev (device int) = 1 when one fails.
// Asynchronous on st.
int validate_coeffs_run(const double* nu, long long nelem, const double* beta, const double* f, const double* divb,
                        const double* g,
                        long long nnodes, int* flag_dev, cudaStream_t st);
// tasks: the restriction queue (nres items), the coarse queue (ntasks items),
// then the local queue (nlocal items)
template <class T>
int apply_tasks_run(const ApTask* tasks, int nres, int ntasks, int nlocal, int nblocks, int* ctr, int nctr,
                    const T* MA, const double* CO, const T* MC, const int* idxA, const int* idxB, const double* r,
                    double* zc, int nG, int nPi, int* err, const int* skip, double bytes, cudaStream_t st);

// Small-matrix kernels for the GEPs live in gep.cu; launchers:
struct FaceJob;   // defined in gep.cu
struct EdgeJob;

struct bddc_ctx_impl;
