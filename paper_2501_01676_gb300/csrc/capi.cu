// C ABI of libbddc and the orchestration of setup and solve.
//
// Setup (all subdomains batched in every step):
//   1. element assembly -> dense A^(i), global FP64 stencil and load (Sect. 2)
//   2. batched partial LU of A^(i): factors of A_II and S^(i) (Sect. 3)
//   3. face Schur complements of B^(i) = sym(S^(i)) onto each face, face GEP
//      kernel (deluxe scaling, parallel sum, pencil, constraint basis)
//   4. per subdomain: change of basis on the faces, Schur complement of B^(i)
//      onto (edges, vertices, face primal coordinates); per (edge, subdomain):
//      Schur complement onto (E, H_k); edge GEP kernel (Sect. 3, new edge GEP)
//   5. per subdomain: extended matrix of T_i^T S^(i) T_i and D_i T_i, one
//      batched elimination of its dual block gives S_Pi,i, D_i Phi_i,
//      Psi_i^T D_i^T and P_i = D_i G_i D_i^T (block elimination of S~)
//   6. coarse matrix S_Pi (FP64) and its explicit inverse
// Solve: condensation, right-preconditioned GMRES (graph-replayed Arnoldi
// steps), interior recovery; MIXED precision wraps this in FP64 iterative
// refinement on the global system.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <memory>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <functional>
#include <tuple>
#include <string>
#include <unordered_map>
#include <vector>

#include "bddc_internal.h"
#include "gep.h"
#include "gmres.h"
#include "mlp.h"
#include "setup_kernels.h"

int assemble_tables_bytes(int element);
void assemble_tables(const HostMesh& hm, void* out, int element);
int build_lut_run(const HostMesh& hm, const int* box0, const int* boxn, const long long* lut_off, int* lut,
                  cudaStream_t st);
template <class TA>
int assemble_launch(const HostMesh& hm, double tau, double c, const void* tables, const double* nu,
                    const double* beta, const double* f, const double* divb, const double bconst[3],
                    const int* slab_x, const int* slab_y, const int* slab_z, const int* lut,
                    const long long* lut_off, const int* box0, const int* boxn, TA* Aloc,
                    const long long* a_off, const int* a_ld, double* stencil, double* F, const double* gnode, int element, cudaStream_t st);
int stencil_residual(const HostMesh& hm, const double* S, const double* u, const double* F, double* r,
                     int nrhs, cudaStream_t st);
// Condensation g += f_B - A_BI A_II^{-1} f_I and interior recovery, each as one
// triangular-solve kernel (CTA per subdomain) plus one batched GEMV over the
// rectangular factor blocks (ci: L_BI, ri: U_IB).
template <class T>
int condense_run(const T* pool, const void* items, int count, int maxnI, const int* lists, const double* F,
                 double* g, double* ystore, int nrhs, long long ldF, long long ldG, long long ldY,
                 const GemvItem* ci, int nci, double ci_bytes, cudaStream_t st);
template <class T>
int recover_run(const T* pool, const void* items, int count, int maxnI, const int* lists, const double* uG,
                double* ystore, double* u, int nrhs, long long ldG, long long ldU, long long ldY,
                const GemvItem* ri, int nri, double ri_bytes, cudaStream_t st);
size_t tri_item_size();
void tri_item_fill(void* dst, long long aoff, int n, int nI, int ld, int dof_off, int gidx_off,
                   long long yoff);
int gather_run(const double* src, const int* idx, double* dst, int n, cudaStream_t st);

// ---------------------------------------------------------------------------
#include <atomic>
static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};
static thread_local bool g_capturing = false;
void bddc_note_launches(unsigned long long n) {
    if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}

// ---- kernel timer: CUDA events around every launch of one kernel class ----
namespace {
struct KTimer {
    int kind = KT_NONE;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    cudaEvent_t open = nullptr;
    double flops = 0, bytes = 0;
    long long launches = 0;
};
std::mutex g_kt_mu;
KTimer g_kt;
}  // namespace

bool ktimer_on(int kind) { return !g_capturing && g_kt.kind == kind && kind != KT_NONE; }

void ktimer_begin(int kind, cudaStream_t st) {
    if (!ktimer_on(kind)) return;
    std::lock_guard<std::mutex> lk(g_kt_mu);
    cudaEventCreate(&g_kt.open);
    cudaEventRecord(g_kt.open, st);
}

void ktimer_end(int kind, cudaStream_t st, double flops, double bytes) {
    if (!ktimer_on(kind)) return;
    std::lock_guard<std::mutex> lk(g_kt_mu);
    if (!g_kt.open) return;
    cudaEvent_t e1;
    cudaEventCreate(&e1);
    cudaEventRecord(e1, st);
    g_kt.ev.push_back({g_kt.open, e1});
    g_kt.open = nullptr;
    g_kt.flops += flops;
    g_kt.bytes += bytes;
    g_kt.launches += 1;
}
void bddc_set_last_error(const char* msg, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s (%s:%d)", msg, file, line);
    g_last_error = buf;
}

namespace {
inline int r4(int n) { return (n + 3) & ~3; }
inline double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}
}  // namespace

// Pinned staging arena of the host tables uploaded during a setup, one per host
// thread.  Space is handed out in order; an event recorded after the last copy
// from the arena tells when all of it has been consumed: the arena restarts from
// the beginning only after that event (at the start of a setup, or when it is
// full), and grows when one table does not fit.
namespace {
struct PinnedArena {
    char* base = nullptr;
    size_t cap = 0, used = 0;
    cudaEvent_t last = nullptr;
    bool pending = false;
    ~PinnedArena() {
        if (last) cudaEventDestroy(last);
        if (base) cudaFreeHost(base);
    }
};
thread_local PinnedArena g_stage;

int stage_reset() {
    PinnedArena& A = g_stage;
    if (A.pending) BDDC_CUDA_TRY(cudaEventSynchronize(A.last));
    A.pending = false;
    A.used = 0;
    return BDDC_OK;
}

int stage_pinned(size_t bytes, cudaStream_t st, char** out) {
    (void)st;
    PinnedArena& A = g_stage;
    const size_t need = (bytes + 255) & ~size_t(255);
    if (A.used + need > A.cap) {
        BDDC_TRY(stage_reset());
        if (need > A.cap) {
            if (A.base) cudaFreeHost(A.base);
            A.base = nullptr;
            A.cap = std::max(need, std::max(2 * A.cap, size_t(32) << 20));
            if (cudaHostAlloc((void**)&A.base, A.cap, cudaHostAllocPortable) != cudaSuccess) {
                A.base = nullptr;
                A.cap = 0;
                bddc_set_last_error("pinned staging memory", __FILE__, __LINE__);
                return BDDC_ENOMEM;
            }
        }
    }
    *out = A.base + A.used;
    A.used += need;
    return BDDC_OK;
}

int stage_done(cudaStream_t st) {
    PinnedArena& A = g_stage;
    if (!A.last) BDDC_CUDA_TRY(cudaEventCreateWithFlags(&A.last, cudaEventDisableTiming));
    BDDC_CUDA_TRY(cudaEventRecord(A.last, st));
    A.pending = true;
    return BDDC_OK;
}
}  // namespace

int staged_upload(void* dev, const void* host, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return BDDC_OK;
    char* h = nullptr;
    BDDC_TRY(stage_pinned(bytes, st, &h));
    memcpy(h, host, bytes);
    BDDC_CUDA_TRY(cudaMemcpyAsync(dev, h, bytes, cudaMemcpyHostToDevice, st));
    return stage_done(st);
}

// Condensation / recovery data of one level of box eliminations (the subdomains,
// or with local nested dissection also the child boxes).
struct TriSet {
    void* tri = nullptr;                          // one TriItem per box
    int* lists = nullptr;
    GemvItem *itCI = nullptr, *itRI = nullptr;    // L_BI and U_IB blocks of the interior factors
    int count = 0, max_nI = 1, nitCI = 0, nitRI = 0;
    double bytesCI = 0, bytesRI = 0;
    long long ny = 1;                             // entries of the stored y_i of all boxes
};

struct bddc_ctx {
    HostMesh hm;
    bddc_opts o;
    cudaStream_t st = nullptr;
    cudaStream_t own = nullptr;   // created when the caller passes the legacy default stream
    int device = 0;               // the CUDA device current at setup (owns st and all buffers)
    bool mixed = false;
    std::vector<void*> allocs;
    size_t bytes = 0;
    bddc_stats stats;
    int nG = 0, nPi = 0;

    // Device memory lives as long as the context.  Requests under 1 MiB are
    // carved (256-byte aligned) out of 16 MiB chunks, so the ~10^3 small
    // per-entity buffers of a setup cost a handful of pool calls.
    static constexpr size_t kSmall = size_t(1) << 20, kChunk = size_t(16) << 20;
    char* chunk = nullptr;
    size_t chunk_used = 0;
    int raw_alloc(void** q, size_t b) {
        cudaError_t e = cudaMallocAsync(q, b, st);
        if (e != cudaSuccess) {
            bddc_set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
            return BDDC_ENOMEM;
        }
        allocs.push_back(*q);
        return BDDC_OK;
    }
    template <class T>
    int alloc(T** p, size_t n) {
        *p = nullptr;
        if (n == 0) n = 1;
        const size_t b = (n * sizeof(T) + 255) & ~size_t(255);
        void* q = nullptr;
        if (b >= kSmall) {
            BDDC_TRY(raw_alloc(&q, b));
        } else {
            if (!chunk || chunk_used + b > kChunk) {
                void* c = nullptr;
                BDDC_TRY(raw_alloc(&c, kChunk));
                chunk = (char*)c;
                chunk_used = 0;
            }
            q = chunk + chunk_used;
            chunk_used += b;
        }
        bytes += n * sizeof(T);
        *p = (T*)q;
        return BDDC_OK;
    }
    // Host tables go to the device through a pinned staging arena: a copy from
    // pageable memory would synchronise the stream first (the host would wait for
    // all queued GPU work before every table), a copy from pinned memory does not.
    template <class T>
    int upload(T** p, const std::vector<T>& v) {
        BDDC_TRY(alloc(p, v.size()));
        if (v.empty()) return BDDC_OK;
        const size_t b = v.size() * sizeof(T);
        char* h = nullptr;
        BDDC_TRY(stage_pinned(b, st, &h));
        memcpy(h, v.data(), b);
        BDDC_CUDA_TRY(cudaMemcpyAsync(*p, h, b, cudaMemcpyHostToDevice, st));
        return stage_done(st);
    }

    // coefficients
    double *nu = nullptr, *beta = nullptr, *f = nullptr, *divb = nullptr;
    double* gdir = nullptr;     // Dirichlet values at the nodes (NULL: zero)
    double bconst[3] = {0, 0, 0};
    double c = 0.0;
    // assembly / factors
    double *stencil = nullptr, *F = nullptr;
    void* A = nullptr;
    std::vector<long long> aoff;
    std::vector<int> ald;
    // packed S
    void* ST = nullptr;
    double* S64 = nullptr;
    std::vector<long long> soff;
    std::vector<int> sld;
    // entities
    std::vector<double*> Q, lam;      // per entity (faces/edges), device
    std::vector<std::vector<double*>> DQ;  // per entity, per side
    std::vector<int> kk, neig;         // host copies
    int* d_k = nullptr;
    int* d_neig = nullptr;
    std::vector<double*> BB;           // edge B~~_E (tests)
    float* d_feat = nullptr;           // edge features (n_edges x BDDC_MLP_FEATURES)
    float* mlp_params = nullptr;       // device copy of the network, when the learned skip is on
    std::vector<char> edge_skipped;    // per edge (edge order)
    // apply operators
    void *MA = nullptr, *MC = nullptr;
    std::vector<long long> maoff, mcoff;
    std::vector<int> mald, mcld, np_s;
    double* SPiInv = nullptr;
    // coarse problem by nested dissection (coarse_path 2): FP64 fronts and sweep operators
    bool coarse_nd = false;
    double* ndOps = nullptr;
    int* ndIdx = nullptr;
    GemvItem *ndFwd = nullptr, *ndBwd = nullptr;
    std::vector<int> ndFwdOff, ndBwdOff;     // per group: first item (last entry: total)
    std::vector<double> ndFwdBytes, ndBwdBytes;
    // M^-1 r as one persistent launch (apply_tasks.cu)
    ApTask* apTasks = nullptr;
    int nApRes = 0, nApTasks = 0, nApLocal = 0, nApCtr = 0, apBlocks = 0;
    int* apCtr = nullptr;
    double apBytes = 0.0;
    int* gidx_pool = nullptr;
    GemvItem *itS = nullptr, *itM1 = nullptr, *itC = nullptr, *itM3 = nullptr;
    int nitS = 0, nitM1 = 0, nitC = 0, nitM3 = 0, maxcols = 0;
    // algorithmic bytes of one product: matrix stream + gathered inputs + scattered outputs
    double bytesS = 0, bytesM1 = 0, bytesC = 0, bytesM3 = 0;
    // condense / recover
    TriSet tp;                  // the subdomains (interior = separators with local_nd)
    double* ystore = nullptr;
    // local nested dissection (opts.local_nd): child boxes, their matrices and
    // substitution data, and the load with their corrections
    std::unique_ptr<LocalND> lnd;
    void* Ac = nullptr;
    std::vector<long long> aoffc;
    std::vector<int> aldc;
    TriSet tc;
    double *Fc = nullptr, *yc = nullptr;
    // work vectors
    double *zc = nullptr, *uPi = nullptr, *g = nullptr, *xG = nullptr, *r = nullptr, *w = nullptr,
           *vcur = nullptr, *t = nullptr;
    double *uglob = nullptr, *res = nullptr, *corr = nullptr, *Fin = nullptr;
    int* gamma_dofs = nullptr;
    // GMRES
    int gm_m = 0;
    double *V = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *gv = nullptr, *hh = nullptr,
           *hh2 = nullptr, *yy = nullptr, *partial = nullptr;
    GmState* gst = nullptr;
    GmState* hst = nullptr;     // pinned host copy
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    unsigned long long graph_kernels = 0;
    int* err = nullptr;
    struct BatchWS* bw = nullptr;   // workspace of the batched multi-RHS solver (first use)
    double* kmax = nullptr;     // largest condition estimate of the solve's GMRES cycles
    double* scal = nullptr;     // pinned host scratch
    // setup phase boundaries on the stream (GPU timeline; read once at the end)
    cudaEvent_t phase_ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    void phase_mark(int k) {
        if (!phase_ev[k]) cudaEventCreate(&phase_ev[k]);
        cudaEventRecord(phase_ev[k], st);
    }
    double phase_ms(int a, int b) {
        float ms = 0.f;
        if (phase_ev[a] && phase_ev[b] && cudaEventElapsedTime(&ms, phase_ev[a], phase_ev[b]) == cudaSuccess)
            return ms;
        return 0.0;
    }
};

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
template <class T>
static int run_engine(bddc_ctx* C, const std::vector<EngItem<T>>& items) {
    if (items.empty()) return BDDC_OK;
    int maxn = 0, maxk = 0;
    for (auto& it : items) {
        maxn = std::max(maxn, it.n);
        maxk = std::max(maxk, it.k);
    }
    EngItem<T>* d = nullptr;
    BDDC_TRY(C->upload(&d, items));
    T* scr = nullptr;
    BDDC_TRY(C->alloc(&scr, (size_t)engine_scratch_elems((int)items.size(), sizeof(T) == 8, maxk)));
    std::vector<int> hn(items.size()), hk(items.size());
    for (size_t i = 0; i < items.size(); ++i) {
        hn[i] = items[i].n;
        hk[i] = items[i].k;
    }
    int kind = C->o.precision == BDDC_PREC_BF16 ? TC_BF16 : (C->o.tensor_cores ? TC_SPLIT_TF32 : TC_NONE);
    // the tensor-core tasks stage rows by 16-byte copies: 16-byte aligned matrices and rows
    for (auto& it : items)
        if ((it.ld & 3) != 0 || (reinterpret_cast<uintptr_t>(it.a) & 15) != 0) kind = TC_NONE;
    return engine_run<T>(d, (int)items.size(), maxn, maxk, scr, C->err, C->st, hn.data(), hk.data(), kind);
}

// Change of basis of a list of entity blocks (TBlock, grouped by output
// matrix): the block kernel when its shared-memory tiles fit, else the
// row/column kernel pair.  Identity entities of a subdomain are merged into
// blocks of at most 64 positions.
template <class T>
static int change_basis(bddc_ctx* C, const std::vector<TBlock>& tb, const int* d_idx, const std::vector<int>& idxv,
                        int maxn_q, cudaStream_t st) {
    if (tb.empty()) return BDDC_OK;
    constexpr int IDCHUNK = 64;
    std::vector<int> extra;
    struct HB { int n; long long pos; bool ext; const double* Q; };
    std::vector<std::vector<HB>> groups;
    std::vector<const TBlock*> head;
    std::vector<int> gid(tb.size());
    std::unordered_map<const void*, int> group_of;
    std::vector<std::vector<int>> members;
    for (size_t i = 0; i < tb.size(); ++i) {
        int g = -1;
        if (!head.empty() && head.back()->dst == tb[i].dst) {
            g = (int)head.size() - 1;
        } else {
            auto f = group_of.find(tb[i].dst);
            if (f != group_of.end()) g = f->second;
        }
        if (g < 0) {
            g = (int)head.size();
            head.push_back(&tb[i]);
            groups.emplace_back();
            members.emplace_back();
            group_of[tb[i].dst] = g;
        }
        gid[i] = g;
        members[g].push_back((int)i);
    }
    int nmax = 1;
    for (size_t g = 0; g < groups.size(); ++g) {
        std::vector<int> ids;
        for (int i : members[g]) {
            const TBlock& B = tb[i];
            if (B.identity) {
                for (int l = 0; l < B.n; ++l) ids.push_back(idxv[B.pos_off + l]);
            } else {
                groups[g].push_back(HB{B.n, (long long)B.pos_off, false, B.Q});
                nmax = std::max(nmax, B.n);
            }
        }
        for (size_t c0 = 0; c0 < ids.size(); c0 += IDCHUNK) {
            const int n = (int)std::min<size_t>(IDCHUNK, ids.size() - c0);
            groups[g].push_back(HB{n, (long long)extra.size(), true, nullptr});
            extra.insert(extra.end(), ids.begin() + c0, ids.begin() + c0 + n);
            nmax = std::max(nmax, n);
        }
    }
    (void)maxn_q;
    if (basis_smem(nmax, sizeof(T)) > 200 * 1024) {
        // large entities: two passes through an n_B x n_B scratch per output
        size_t ytot = 0;
        std::vector<TBlock> tb2 = tb;
        std::vector<long long> yo(groups.size());
        for (size_t g = 0; g < groups.size(); ++g) {
            yo[g] = (long long)ytot;
            ytot += (size_t)head[g]->nrows * head[g]->nrows;
        }
        T* Y = nullptr;
        BDDC_TRY(C->alloc(&Y, ytot));
        int mq = 1;
        for (size_t i = 0; i < tb2.size(); ++i) {
            tb2[i].y = Y + yo[gid[i]];
            tb2[i].yld = tb2[i].nrows;
            if (!tb2[i].identity) mq = std::max(mq, tb2[i].n);
        }
        TBlock* d_tb;
        BDDC_TRY(C->upload(&d_tb, tb2));
        return transform_run<T>(d_tb, (int)tb2.size(), d_idx, mq, 4, st);
    }
    int* d_extra = nullptr;
    BDDC_TRY(C->upload(&d_extra, extra));
    std::vector<XBlock> xb;
    std::vector<XSub> xs;
    std::vector<XRow> xr;
    for (size_t g = 0; g < groups.size(); ++g) {
        const TBlock& H = *head[g];
        XSub S;
        S.src = H.src;
        S.sld = H.sld;
        S.sym = H.sym;
        S.nblk = (int)groups[g].size();
        S.blk_off = (int)xb.size();
        S.perm = d_idx + H.perm_off;
        S.dst = H.dst;
        S.dld = H.dld;
        for (size_t b = 0; b < groups[g].size(); ++b) {
            const HB& h = groups[g][b];
            xb.push_back(XBlock{h.n, h.ext ? d_extra + h.pos : d_idx + h.pos, h.Q});
            xr.push_back(XRow{(int)xs.size(), (int)b});
        }
        xs.push_back(S);
    }
    XBlock* d_xb;
    XSub* d_xs;
    XRow* d_xr;
    BDDC_TRY(C->upload(&d_xb, xb));
    BDDC_TRY(C->upload(&d_xs, xs));
    BDDC_TRY(C->upload(&d_xr, xr));
    return basis_run<T>(d_xr, (int)xr.size(), d_xs, d_xb, nmax, st);
}

// Coarse problem by nested dissection of the subdomain grid: symbolic plan on
// the host, then per height of the tree (leaves first) the fronts are filled
// from S_Pi, the children's updates are added, the engine eliminates the own
// unknowns of every front of that height in one launch (FP64), and the sweep
// operators are copied out of the trailing blocks.
static int coarse_nd_setup(bddc_ctx* C, const double* SPi, NDPlan& P) {
    cudaStream_t st = C->st;
    const int nPi = C->nPi;
    BDDC_TRY(nd_plan(C->hm, nPi, P));
    double* Fp = nullptr;
    BDDC_TRY(C->alloc(&Fp, (size_t)P.fpool));
    BDDC_TRY(C->alloc(&C->ndOps, (size_t)P.opool));
    BDDC_TRY(C->upload(&C->ndIdx, P.idx));
    NDFront* d_fr = nullptr;
    BDDC_TRY(C->upload(&d_fr, P.fr));
    const int H = (int)P.by_height.size();
    // row jobs of every height, uploaded once
    const int RJ = 8;
    std::vector<NDRowJob> fill, add;
    std::vector<int> fill_off(H + 1, 0), add_off(H + 1, 0);
    std::vector<CopyJob> cj;
    std::vector<int> cj_off(H + 1, 0);
    for (int h = 0; h < H; ++h) {
        fill_off[h] = (int)fill.size();
        add_off[h] = (int)add.size();
        cj_off[h] = (int)cj.size();
        for (int a : P.by_height[h]) {
            const NDFront& f = P.fr[a];
            for (int r0 = 0; r0 < f.N; r0 += RJ) fill.push_back(NDRowJob{a, r0, std::min(RJ, f.N - r0)});
            if (f.b > 0 && f.n > 0)
                cj.push_back(CopyJob{Fp + f.foff, f.ld, f.n, f.n + f.b, f.b, f.n, C->ndOps + f.wf_off, f.wf_ld, -1.0});
            if (f.n > 0)
                cj.push_back(CopyJob{Fp + f.foff, f.ld, f.n + f.b, f.n, f.n, f.b + f.n, C->ndOps + f.wb_off, f.wb_ld,
                                     1.0});
        }
        // children (at lower heights) of this height's fronts
        for (int a = 0; a < (int)P.fr.size(); ++a) {
            const NDFront& f = P.fr[a];
            if (f.parent < 0 || f.b == 0 || P.fr[f.parent].height != h) continue;
            for (int r0 = 0; r0 < f.b; r0 += RJ) add.push_back(NDRowJob{a, r0, std::min(RJ, f.b - r0)});
        }
    }
    fill_off[H] = (int)fill.size();
    add_off[H] = (int)add.size();
    cj_off[H] = (int)cj.size();
    NDRowJob *d_fill = nullptr, *d_add = nullptr;
    CopyJob* d_cj = nullptr;
    BDDC_TRY(C->upload(&d_fill, fill));
    BDDC_TRY(C->upload(&d_add, add));
    BDDC_TRY(C->upload(&d_cj, cj));
    for (int h = 0; h < H; ++h) {
        BDDC_TRY(nd_fill_run(d_fr, d_fill + fill_off[h], fill_off[h + 1] - fill_off[h], C->ndIdx, SPi, nPi, Fp, st));
        BDDC_TRY(nd_add_run(d_fr, d_add + add_off[h], add_off[h + 1] - add_off[h], C->ndIdx, Fp, st));
        std::vector<EngItem<double>> items;
        for (int a : P.by_height[h])
            if (P.fr[a].n > 0) items.push_back(EngItem<double>{Fp + P.fr[a].foff, P.fr[a].N, P.fr[a].n, P.fr[a].ld});
        BDDC_TRY(run_engine<double>(C, items));
        if (cj_off[h + 1] > cj_off[h])
            BDDC_TRY((copy_blocks_run<double, double>(d_cj + cj_off[h], cj_off[h + 1] - cj_off[h], 8, st)));
    }
    // sweep items, concatenated per group
    std::vector<GemvItem> fw, bw;
    C->ndFwdOff.assign(1, 0);
    C->ndBwdOff.assign(1, 0);
    C->ndFwdBytes.clear();
    C->ndBwdBytes.clear();
    for (int h = 0; h < H; ++h) {
        fw.insert(fw.end(), P.fwd[h].begin(), P.fwd[h].end());
        C->ndFwdOff.push_back((int)fw.size());
        double by = 0.0;
        for (int a : P.by_height[h]) by += 8.0 * P.fr[a].b * P.fr[a].n + 12.0 * (P.fr[a].n + P.fr[a].b);
        C->ndFwdBytes.push_back(by);
    }
    for (int d = 0; d < (int)P.by_depth.size(); ++d) {
        bw.insert(bw.end(), P.bwd[d].begin(), P.bwd[d].end());
        C->ndBwdOff.push_back((int)bw.size());
        double by = 0.0;
        for (int a : P.by_depth[d])
            by += 8.0 * P.fr[a].n * (P.fr[a].b + P.fr[a].n) + 12.0 * (P.fr[a].b + 2.0 * P.fr[a].n);
        C->ndBwdBytes.push_back(by);
    }
    BDDC_TRY(C->upload(&C->ndFwd, fw));
    BDDC_TRY(C->upload(&C->ndBwd, bw));
    C->coarse_nd = true;
    C->stats.coarse_fronts = (int)P.fr.size();
    C->stats.coarse_levels = H;
    C->stats.coarse_factor_gflop = P.flops * 1e-9;
    return BDDC_OK;
}

// Work items of M^-1 r in topological order for the one-launch apply: the local
// part with the coarse restriction, the coarse solve (forward sweep by height,
// backward sweep by depth, or the explicit inverse), the prolongation.
template <class T>
static int build_apply_tasks(bddc_ctx* C, const std::vector<GemvItem>& iM1, const std::vector<GemvItem>& iLoc,
                             const std::vector<GemvItem>& iCt, const std::vector<GemvItem>& iM3, const NDPlan* P) {
    std::vector<ApTask> t;
    auto add = [&](const GemvItem& it, int kind, int w0, int t0, int w1, int t1, int s0, int s1) {
        ApTask a;
        a.it = it;
        a.kind = kind;
        a.w0 = w0;
        a.t0 = t0;
        a.w1 = w1;
        a.t1 = t1;
        a.s0 = s0;
        a.s1 = s1;
        t.push_back(a);
    };
    const int nA = (int)iM1.size();
    for (const GemvItem& it : iM1) add(it, AP_LOCAL, -1, 0, -1, 0, AP_CTR_LOCAL, -1);
    C->nApRes = nA;
    int ncoarse = 0;
    int nfr = 0;
    if (C->nPi > 0 && P) {
        nfr = (int)P->fr.size();
        auto fctr = [&](int a) { return AP_CTR_FRONTS + a; };           // forward items of a's children done
        auto bctr = [&](int a) { return AP_CTR_FRONTS + nfr + a; };     // backward items of a done
        std::vector<int> nfw(nfr, 0), nbw(nfr, 0), nchild_fw(nfr, 0);
        // items per front, recounted from the plan's sizes
        auto nitems = [](int rows, int cols) {
            return ((rows + ND_ITEM_ROWS - 1) / ND_ITEM_ROWS) * ((cols + ND_ITEM_COLS - 1) / ND_ITEM_COLS);
        };
        for (int a = 0; a < nfr; ++a) {
            const NDFront& f = P->fr[a];
            nfw[a] = (f.b > 0 && f.n > 0) ? nitems(f.b, f.n) : 0;
            nbw[a] = f.n > 0 ? nitems(f.n, f.b + f.n) : 0;
            if (f.parent >= 0) nchild_fw[f.parent] += nfw[a];
        }
        // forward items by height, front by front, in the plan's item order
        for (size_t h = 0; h < P->by_height.size(); ++h) {
            size_t k = 0;
            for (int a : P->by_height[h]) {
                const NDFront& f = P->fr[a];
                for (int q = 0; q < nfw[a]; ++q, ++k)
                    add(P->fwd[h][k], AP_SWEEP, AP_CTR_LOCAL, nA, nchild_fw[a] > 0 ? fctr(a) : -1, nchild_fw[a],
                        f.parent >= 0 ? fctr(f.parent) : -1, -1);
            }
            if (k != P->fwd[h].size()) return BDDC_EINVAL;
        }
        for (size_t d = 0; d < P->by_depth.size(); ++d) {
            size_t k = 0;
            for (int a : P->by_depth[d]) {
                const NDFront& f = P->fr[a];
                for (int q = 0; q < nbw[a]; ++q, ++k) {
                    if (f.parent < 0)
                        add(P->bwd[d][k], AP_SWEEP, AP_CTR_LOCAL, nA, nchild_fw[a] > 0 ? fctr(a) : -1, nchild_fw[a],
                            bctr(a), AP_CTR_COARSE);
                    else
                        add(P->bwd[d][k], AP_SWEEP, bctr(f.parent), nbw[f.parent], -1, 0, bctr(a), AP_CTR_COARSE);
                    ++ncoarse;
                }
            }
            if (k != P->bwd[d].size()) return BDDC_EINVAL;
        }
        C->apBytes = C->bytesM1 + P->bytes_solve + C->bytesM3;
    } else if (C->nPi > 0) {
        for (const GemvItem& it : iCt) add(it, AP_DENSE, AP_CTR_LOCAL, nA, -1, 0, AP_CTR_COARSE, -1);
        ncoarse = (int)iCt.size();
        C->apBytes = C->bytesM1 + C->bytesC + C->bytesM3;
    } else {
        C->apBytes = C->bytesM1;
    }
    if (C->nPi > 0)
        for (const GemvItem& it : iM3) add(it, AP_PROLONG, AP_CTR_COARSE, ncoarse, -1, 0, -1, -1);
    C->nApTasks = (int)t.size() - nA;
    for (const GemvItem& it : iLoc) add(it, AP_LOCAL, -1, 0, -1, 0, -1, -1);
    C->nApLocal = (int)t.size() - nA - C->nApTasks;
    C->nApCtr = AP_CTR_FRONTS + 2 * nfr;
    BDDC_TRY(C->upload(&C->apTasks, t));
    BDDC_TRY(C->alloc(&C->apCtr, (size_t)C->nApCtr));
    C->apBlocks = apply_tasks_blocks<T>();
    return BDDC_OK;
}

// y2 = [y (nPi) | x (nPi)]: y holds the coarse right-hand side on entry (it is
// transformed in place by the forward sweep), x receives S_Pi^-1 y.
static int coarse_nd_solve(bddc_ctx* C, double* y2, const int* skip) {
    const int nPi = C->nPi;
    BDDC_CUDA_TRY(cudaMemsetAsync(y2 + nPi, 0, sizeof(double) * nPi, C->st));
    for (size_t h = 0; h + 1 < C->ndFwdOff.size(); ++h) {
        const int a = C->ndFwdOff[h], b = C->ndFwdOff[h + 1];
        if (b > a)
            BDDC_TRY(gemv_run<double>(C->ndOps, C->ndFwd + a, b - a, C->ndIdx, y2, y2, 0, 1, 0, 0, C->st, skip,
                                      C->ndFwdBytes[h]));
    }
    for (size_t d = 0; d + 1 < C->ndBwdOff.size(); ++d) {
        const int a = C->ndBwdOff[d], b = C->ndBwdOff[d + 1];
        if (b > a)
            BDDC_TRY(gemv_run<double>(C->ndOps, C->ndBwd + a, b - a, C->ndIdx, y2, y2, 0, 1, 0, 0, C->st, skip,
                                      C->ndBwdBytes[d]));
    }
    return BDDC_OK;
}

// Rows per S x work item, chosen by measurement: every candidate's item list is
// timed on the context's own operators (CUDA events on the setup stream, one
// warm-up launch, the mean of three), the first time a shape class (subdomains,
// interface rows, precision) is seen in the process; later setups of the class
// reuse the choice.  The measurement waits for the setup work queued before it.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, long long, int>, int> g_tune_rows;

template <class T>
static int tune_gemv_rows(bddc_ctx* C, const std::vector<GemvItem>& iS0, int rb0,
                          const std::function<void(std::vector<GemvItem>&, int)>& build, int* rb_out,
                          double* us_out) {
    *rb_out = rb0;
    *us_out = 0.0;
    double *x = nullptr, *y = nullptr;
    BDDC_TRY(C->alloc(&x, (size_t)C->nG));
    BDDC_TRY(C->alloc(&y, (size_t)C->nG));
    BDDC_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * C->nG, C->st));
    BDDC_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * C->nG, C->st));
    cudaEvent_t e0, e1;
    BDDC_CUDA_TRY(cudaEventCreate(&e0));
    BDDC_CUDA_TRY(cudaEventCreate(&e1));
    double best = 1e300;
    int rc = BDDC_OK;
    for (int rb : {32, 64, 128, 256}) {
        std::vector<GemvItem> v;
        if (rb == rb0) v = iS0;
        else build(v, rb);
        GemvItem* d = nullptr;
        if ((rc = C->upload(&d, v)) != BDDC_OK) break;
        const int nit = (int)v.size();
        if ((rc = gemv_run<T>((const T*)C->ST, d, nit, C->gidx_pool, x, y, C->maxcols, 1, 0, 0, C->st, nullptr)) !=
            BDDC_OK)
            break;
        if (cudaEventRecord(e0, C->st) != cudaSuccess) { rc = BDDC_ECUDA; break; }
        for (int r = 0; r < 3 && rc == BDDC_OK; ++r)
            rc = gemv_run<T>((const T*)C->ST, d, nit, C->gidx_pool, x, y, C->maxcols, 1, 0, 0, C->st, nullptr);
        if (rc != BDDC_OK) break;
        float ms = 0.f;
        if (cudaEventRecord(e1, C->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = BDDC_ECUDA;
            break;
        }
        const double us = 1000.0 * ms / 3.0;
        if (us < best) {
            best = us;
            *rb_out = rb;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == BDDC_OK) *us_out = best;
    return rc;
}

// Element assembly into the dense matrices of a list of boxes (the subdomains, or
// the child boxes of local nested dissection) stored at (aoff, ald) in pool, in
// each box's own numbering (interior, then interface, box order); the global
// stencil and load (C->stencil, C->F, zeroed by the caller) are assembled with it.
template <class T>
static int assemble_boxes(bddc_ctx* C, const HostMesh& mesh, T* pool, const std::vector<long long>& aoff,
                          const std::vector<int>& ald) {
    cudaStream_t st = C->st;
    const int nbox = mesh.nsd;
    // node -> local index table of every box, built on the GPU (k_build_lut)
    std::vector<int> box0(3 * nbox), boxn(3 * nbox);
    std::vector<long long> lut_off(nbox);
    long long lut_n = 0;
    for (int s = 0; s < nbox; ++s) {
        const SubInfo& S = mesh.sub[s];
        lut_off[s] = lut_n;
        long long nb = 1;
        for (int d = 0; d < 3; ++d) {
            box0[3 * s + d] = S.box0[d];
            boxn[3 * s + d] = S.box1[d] - S.box0[d] + 1;
            nb *= boxn[3 * s + d];
        }
        lut_n += nb;
    }
    std::vector<int> slab[3];
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < mesh.nsub[d]; ++s)
            for (int e = mesh.off[d][s]; e < mesh.off[d][s + 1]; ++e) slab[d].push_back(s);
    int *d_lut, *d_box0, *d_boxn, *d_sx, *d_sy, *d_sz, *d_ald;
    long long *d_lutoff, *d_aoff;
    BDDC_TRY(C->upload(&d_lutoff, lut_off));
    BDDC_TRY(C->upload(&d_box0, box0));
    BDDC_TRY(C->upload(&d_boxn, boxn));
    BDDC_TRY(C->alloc(&d_lut, (size_t)std::max(lut_n, 1LL)));
    BDDC_TRY(build_lut_run(mesh, d_box0, d_boxn, d_lutoff, d_lut, st));
    BDDC_TRY(C->upload(&d_sx, slab[0]));
    BDDC_TRY(C->upload(&d_sy, slab[1]));
    BDDC_TRY(C->upload(&d_sz, slab[2]));
    BDDC_TRY(C->upload(&d_aoff, aoff));
    BDDC_TRY(C->upload(&d_ald, ald));
    std::vector<char> tabs((size_t)assemble_tables_bytes(C->o.element));
    assemble_tables(mesh, tabs.data(), C->o.element);
    char* d_tabs = nullptr;
    BDDC_TRY(C->upload(&d_tabs, tabs));
    ktimer_begin(KT_ASSEMBLE, st);
    BDDC_TRY(assemble_launch<T>(mesh, C->o.tau, C->c, d_tabs, C->nu, C->beta, C->f, C->divb, C->bconst, d_sx, d_sy,
                                d_sz, d_lut, d_lutoff, d_box0, d_boxn, pool, d_aoff, d_ald, C->stencil, C->F, C->gdir,
                                C->o.element, st));
    ktimer_end(KT_ASSEMBLE, st, 0.0, 0.0);
    return BDDC_OK;
}

// Condensation / recovery data of a list of boxes whose factors sit in one pool
// (aoff, ald): per box its dof list (interior, then interface), the map of its
// interface to the output vector (the Gamma numbering, or with global_out the
// global dofs: the child boxes of local nested dissection condense into a copy of
// the load and recover from the global solution), and the GEMV items of L_BI and
// U_IB in column slices of the kernel's staging width.
template <class T>
static int build_tri(bddc_ctx* C, const std::vector<SubInfo>& subs, const std::vector<long long>& aoff,
                     const std::vector<int>& ald, bool global_out, TriSet& ts) {
    const int nbox = (int)subs.size();
    std::vector<int> lists;
    std::vector<char> items(tri_item_size() * std::max(nbox, 1));
    long long yo = 0;
    std::vector<GemvItem> ci, ri;
    const double tsz = sizeof(T), iv = 8.0 + 4.0;
    ts = TriSet();
    for (int s = 0; s < nbox; ++s) {
        const SubInfo& S = subs[s];
        const int nI = S.nI, nB = S.nB, ld = ald[s];
        const int dof_off = (int)lists.size();
        lists.insert(lists.end(), S.dofs.begin(), S.dofs.end());
        const int go = (int)lists.size();
        const std::vector<int> omap = global_out ? std::vector<int>(S.dofs.begin() + nI, S.dofs.end()) : S.gidx;
        if ((int)omap.size() != nB) return BDDC_EINVAL;
        lists.insert(lists.end(), omap.begin(), omap.end());
        tri_item_fill(items.data() + tri_item_size() * s, aoff[s], S.n, nI, ld, dof_off, go, yo);
        // y positions of the box, and the interface map behind nI unused slots
        // (the U_IB items read columns nI .. n-1 of A through input slots nI .. n-1)
        const int yi = (int)lists.size();
        for (int q = 0; q < nI; ++q) lists.push_back((int)(yo + q));
        const int gp = (int)lists.size();
        lists.insert(lists.end(), (size_t)nI, 0);
        lists.insert(lists.end(), omap.begin(), omap.end());
        if (nI > 0 && nB > 0) {
            for (int c0 = 0; c0 < nI; c0 += 2048)
                for (int r0 = 0; r0 < nB; r0 += 32)
                    ci.push_back(GemvItem{aoff[s] + (long long)nI * ld, nB, nI, ld, yi, go, r0, std::min(32, nB - r0),
                                          c0, std::min(2048, nI - c0)});
            for (int c0 = 0; c0 < nB; c0 += 2048)
                for (int r0 = 0; r0 < nI; r0 += 32)
                    ri.push_back(GemvItem{aoff[s], nI, S.n, ld, gp, yi, r0, std::min(32, nI - r0), nI + c0,
                                          std::min(2048, nB - c0)});
            ts.bytesCI += tsz * nB * nI + iv * (nI + nB);
            ts.bytesRI += tsz * nI * nB + iv * (nB + nI);
        }
        yo += nI;
        ts.max_nI = std::max(ts.max_nI, nI);
    }
    if ((long long)lists.size() + yo > INT_MAX) return BDDC_EINVAL;
    ts.count = nbox;
    ts.ny = std::max(yo, 1LL);
    BDDC_TRY(C->upload(&ts.lists, lists));
    BDDC_TRY(C->upload((char**)&ts.tri, items));
    BDDC_TRY(C->upload(&ts.itCI, ci));
    BDDC_TRY(C->upload(&ts.itRI, ri));
    ts.nitCI = (int)ci.size();
    ts.nitRI = (int)ri.size();
    return BDDC_OK;
}

// g = F_Gamma - A_Gamma,I A_II^{-1} F_I for nrhs columns (F, Fw: ndof x nrhs; g: nG
// x nrhs; y of the boxes stored for the recovery).  With local nested dissection the
// children's interiors are condensed first, into Fw (a copy of F that receives
// their corrections on the separators and the interface), then the separators.
template <class T>
static int condense_all(bddc_ctx* C, const double* F, double* g, double* ystore, double* Fw, double* yc, int nrhs,
                        cudaStream_t st) {
    const long long nG = C->nG, ndof = C->hm.ndof;
    const double* Fp = F;
    if (C->lnd) {
        const TriSet& c = C->tc;
        BDDC_CUDA_TRY(cudaMemcpyAsync(Fw, F, sizeof(double) * ndof * nrhs, cudaMemcpyDeviceToDevice, st));
        BDDC_TRY(condense_run<T>((const T*)C->Ac, c.tri, c.count, c.max_nI, c.lists, F, Fw, yc, nrhs, ndof, ndof, c.ny,
                                 c.itCI, c.nitCI, c.bytesCI, st));
        Fp = Fw;
    }
    for (int c = 0; c < nrhs; ++c) BDDC_TRY(gather_run(Fp + c * ndof, C->gamma_dofs, g + c * nG, (int)nG, st));
    const TriSet& t = C->tp;
    return condense_run<T>((const T*)C->A, t.tri, t.count, t.max_nI, t.lists, Fp, g, ystore, nrhs, ndof, nG, t.ny,
                           t.itCI, t.nitCI, t.bytesCI, st);
}

// u = [A_II^{-1}(F_I - A_I,Gamma x_Gamma); x_Gamma] from the stored y (nrhs columns);
// with local nested dissection the separators first, then the children's
// interiors from the solution just written on their boundaries.
template <class T>
static int recover_all(bddc_ctx* C, const double* xG, double* ystore, double* u, double* yc, int nrhs,
                       cudaStream_t st) {
    const long long nG = C->nG, ndof = C->hm.ndof;
    const TriSet& t = C->tp;
    BDDC_TRY(recover_run<T>((const T*)C->A, t.tri, t.count, t.max_nI, t.lists, xG, ystore, u, nrhs, nG, ndof, t.ny,
                            t.itRI, t.nitRI, t.bytesRI, st));
    if (C->lnd) {
        const TriSet& c = C->tc;
        BDDC_TRY(recover_run<T>((const T*)C->Ac, c.tri, c.count, c.max_nI, c.lists, u, yc, u, nrhs, ndof, ndof, c.ny,
                                c.itRI, c.nitRI, c.bytesRI, st));
    }
    return BDDC_OK;
}

template <class T>
static int setup_impl(bddc_ctx* C) {
    HostMesh& hm = C->hm;
    cudaStream_t st = C->st;
    const int nsd = hm.nsd;
    C->phase_mark(0);
    // ---- 0. local nested dissection: child boxes, subdomains renumbered to
    //         [separators, interface] ---------------------------------------
    if (C->o.local_nd) {
        C->lnd.reset(new LocalND);
        BDDC_TRY(build_local_nd(hm, *C->lnd));
        for (const SubInfo& K : C->lnd->child.sub)
            if (K.nI > BDDC_MAX_INTERIOR) {
                bddc_set_last_error("child box interior larger than the interior-solve limit", __FILE__, __LINE__);
                return BDDC_EINVAL;
            }
    }
    for (const SubInfo& S : hm.sub)
        if (S.nI > BDDC_MAX_INTERIOR) {
            bddc_set_last_error("subdomain interior (separators with local_nd) larger than the interior-solve limit",
                                __FILE__, __LINE__);
            return BDDC_EINVAL;
        }
    // element -> subdomain slab maps (edge features of the learned skip)
    int *d_sx = nullptr, *d_sy = nullptr, *d_sz = nullptr;
    {
        std::vector<int> slab[3];
        for (int d = 0; d < 3; ++d)
            for (int s = 0; s < hm.nsub[d]; ++s)
                for (int e = hm.off[d][s]; e < hm.off[d][s + 1]; ++e) slab[d].push_back(s);
        BDDC_TRY(C->upload(&d_sx, slab[0]));
        BDDC_TRY(C->upload(&d_sy, slab[1]));
        BDDC_TRY(C->upload(&d_sz, slab[2]));
    }
    // ---- 1. assembly --------------------------------------------------------
    C->aoff.resize(nsd);
    C->ald.resize(nsd);
    long long atot = 0;
    for (int s = 0; s < nsd; ++s) {
        C->ald[s] = r4(hm.sub[s].n);
        C->aoff[s] = atot;
        atot += (long long)hm.sub[s].n * C->ald[s];
    }
    T* A = nullptr;
    BDDC_TRY(C->alloc(&A, atot));
    C->A = A;
    BDDC_CUDA_TRY(cudaMemsetAsync(A, 0, atot * sizeof(T), st));
    BDDC_TRY(C->alloc(&C->stencil, (size_t)27 * hm.ndof));
    BDDC_TRY(C->alloc(&C->F, hm.ndof));
    BDDC_CUDA_TRY(cudaMemsetAsync(C->stencil, 0, sizeof(double) * 27 * (size_t)hm.ndof, st));
    BDDC_CUDA_TRY(cudaMemsetAsync(C->F, 0, sizeof(double) * hm.ndof, st));
    double fl = 0.0;           // flops of the box eliminations
    auto elim_flops = [](double n, double k) {
        const double m = n - k;
        return 2.0 / 3.0 * k * k * k + 2.0 * k * k * m + 2.0 * k * m * m;
    };
    if (!C->lnd) {
        BDDC_TRY(assemble_boxes<T>(C, hm, A, C->aoff, C->ald));
    } else {
        // children: assembly, interior eliminations, then their Schur complements
        // added into the subdomains' matrices over [separators, interface]
        const HostMesh& ch = C->lnd->child;
        const int nch = ch.nsd;
        C->aoffc.resize(nch);
        C->aldc.resize(nch);
        long long ctot = 0;
        for (int c = 0; c < nch; ++c) {
            C->aldc[c] = r4(ch.sub[c].n);
            C->aoffc[c] = ctot;
            ctot += (long long)ch.sub[c].n * C->aldc[c];
        }
        T* Ac = nullptr;
        BDDC_TRY(C->alloc(&Ac, std::max(ctot, 1LL)));
        C->Ac = Ac;
        BDDC_CUDA_TRY(cudaMemsetAsync(Ac, 0, ctot * sizeof(T), st));
        BDDC_TRY(assemble_boxes<T>(C, ch, Ac, C->aoffc, C->aldc));
        std::vector<EngItem<T>> items;
        for (int c = 0; c < nch; ++c)
            if (ch.sub[c].nI > 0) {
                items.push_back(EngItem<T>{Ac + C->aoffc[c], ch.sub[c].n, ch.sub[c].nI, C->aldc[c]});
                fl += elim_flops(ch.sub[c].n, ch.sub[c].nI);
            }
        if (!items.empty()) BDDC_TRY(run_engine<T>(C, items));
        std::vector<int> mapv;
        std::vector<long long> moff(nch);
        for (int c = 0; c < nch; ++c) {
            moff[c] = (long long)mapv.size();
            mapv.insert(mapv.end(), C->lnd->map[c].begin(), C->lnd->map[c].end());
        }
        int* d_map = nullptr;
        BDDC_TRY(C->upload(&d_map, mapv));
        std::vector<ExtendJob> xj;
        for (int c = 0; c < nch; ++c) {
            const SubInfo& K = ch.sub[c];
            if (K.nB == 0) continue;
            const int p = C->lnd->parent[c];
            xj.push_back(ExtendJob{Ac + C->aoffc[c] + (long long)K.nI * C->aldc[c] + K.nI, C->aldc[c], K.nB,
                                   d_map + moff[c], A + C->aoff[p], C->ald[p]});
        }
        ExtendJob* d_xj = nullptr;
        BDDC_TRY(C->upload(&d_xj, xj));
        BDDC_TRY(extend_add_run<T>(d_xj, (int)xj.size(), 16, st));
        C->stats.nd_children = nch;
    }
    C->phase_mark(1);
    // ---- 2. partial LU: S^(i) (with local_nd: the separators) ---------------
    {
        std::vector<EngItem<T>> items;
        for (int s = 0; s < nsd; ++s)
            if (!C->lnd || hm.sub[s].nI > 0) {
                items.push_back(EngItem<T>{A + C->aoff[s], hm.sub[s].n, hm.sub[s].nI, C->ald[s]});
                fl += elim_flops(hm.sub[s].n, hm.sub[s].nI);
            }
        if (!items.empty()) BDDC_TRY(run_engine<T>(C, items));
        C->stats.factor_gflop = fl * 1e-9;
    }
    C->soff.resize(nsd);
    C->sld.resize(nsd);
    long long stot = 0;
    for (int s = 0; s < nsd; ++s) {
        C->sld[s] = r4(hm.sub[s].nB);
        C->soff[s] = stot;
        stot += (long long)hm.sub[s].nB * C->sld[s];
    }
    T* ST = nullptr;
    BDDC_TRY(C->alloc(&ST, stot));
    C->ST = ST;
    {
        std::vector<CopyJob> jobs(nsd);
        for (int s = 0; s < nsd; ++s) {
            SubInfo& S = hm.sub[s];
            jobs[s] = CopyJob{A + C->aoff[s], C->ald[s], S.nI, S.nI, S.nB, S.nB, ST + C->soff[s], C->sld[s], 1.0};
        }
        CopyJob* d;
        BDDC_TRY(C->upload(&d, jobs));
        BDDC_TRY((copy_blocks_run<T, T>(d, nsd, 32, st)));
        if (C->mixed) {
            BDDC_TRY(C->alloc(&C->S64, stot));
            for (int s = 0; s < nsd; ++s) jobs[s] = CopyJob{ST + C->soff[s], C->sld[s], 0, 0, hm.sub[s].nB, hm.sub[s].nB, C->S64 + C->soff[s], C->sld[s], 1.0};
            CopyJob* d2;
            BDDC_TRY(C->upload(&d2, jobs));
            BDDC_TRY((copy_blocks_run<T, double>(d2, nsd, 32, st)));
        } else {
            C->S64 = (double*)ST;
        }
    }
    {
        // the interface classification on the host while the GPU assembles and
        // eliminates the interiors (nothing above needs it)
        const auto t0 = std::chrono::steady_clock::now();
        BDDC_TRY(build_host_interface(hm));
        C->nG = (int)hm.gamma.size();
        C->stats.t_mesh_ms += ms_since(t0);
    }
    C->phase_mark(2);
    // interface maps
    std::vector<int> gl;
    std::vector<int> gl_off(nsd);
    for (int s = 0; s < nsd; ++s) {
        gl_off[s] = (int)gl.size();
        gl.insert(gl.end(), hm.sub[s].gidx.begin(), hm.sub[s].gidx.end());
    }
    // entity position lists on the device
    const int nent = (int)hm.ent.size();
    std::vector<int> posl;
    std::vector<std::vector<int>> pos_off(nent);
    for (int e = 0; e < nent; ++e)
        for (size_t a = 0; a < hm.ent[e].subs.size(); ++a) {
            pos_off[e].push_back((int)posl.size());
            posl.insert(posl.end(), hm.ent[e].pos[a].begin(), hm.ent[e].pos[a].end());
        }
    int* d_pos = nullptr;
    BDDC_TRY(C->upload(&d_pos, posl));
    C->Q.assign(nent, nullptr);
    C->lam.assign(nent, nullptr);
    C->DQ.assign(nent, {});
    C->BB.assign(nent, nullptr);
    C->kk.assign(nent, 0);
    C->neig.assign(nent, 0);
    BDDC_TRY(C->alloc(&C->d_k, nent));
    BDDC_TRY(C->alloc(&C->d_neig, nent));
    BDDC_CUDA_TRY(cudaMemsetAsync(C->d_k, 0, sizeof(int) * nent, st));
    BDDC_CUDA_TRY(cudaMemsetAsync(C->d_neig, 0, sizeof(int) * nent, st));
    for (int e = 0; e < nent; ++e) {
        Entity& E = hm.ent[e];
        int n = (int)E.dofs.size();
        BDDC_TRY(C->alloc(&C->Q[e], (size_t)n * n));
        BDDC_TRY(C->alloc(&C->lam[e], (size_t)3 * n + 1));
        C->DQ[e].resize(E.subs.size());
        if (E.kind == 0) {
            E.k = 1;
            continue;
        }
        for (size_t a = 0; a < E.subs.size(); ++a) BDDC_TRY(C->alloc(&C->DQ[e][a], (size_t)n * n));
        E.theta = E.kind == 1 ? C->o.theta_E : C->o.theta_F;
        if (E.kind == 2 && !(C->o.theta_F > 0)) {
            int m = 0;
            for (int s : E.subs) m = std::max(m, hm.sub[s].max_slab);
            E.theta = 1.0 + std::log((double)m);
        }
    }
    // ---- 3. faces ------------------------------------------------------------
    const int face_mode = C->o.all_primal ? 1 : (C->o.face_gep ? 0 : 2);
    std::vector<int>& faces = hm.by_kind[2];
    if (!faces.empty()) {
        std::vector<int> permv;
        std::vector<GatherJob> gj;
        std::vector<EngItem<T>> items;
        // Face Schur complements of B^(i) (the symmetric part of S^(i)) in two levels,
        // both exact by the quotient property of Schur complements: (1) per
        // subdomain eliminate the edge and vertex positions, leaving the Schur
        // complement on its face positions; (2) per (face, side) eliminate the other
        // faces' positions from it.  Level 1 is shared by the subdomain's faces.
        double* Bt64 = nullptr;
        std::vector<long long> bo;
        long long btot = 0;
        for (int e : faces) {
            int nF = (int)hm.ent[e].dofs.size();
            bo.push_back(btot);
            btot += 2LL * nF * nF;
        }
        BDDC_TRY(C->alloc(&Bt64, btot));
        int* d_perm = nullptr;
        if (face_mode == 0) {
            std::vector<int> nFP(nsd), nEV(nsd);
            std::vector<std::vector<int>> fpos(nsd);              // face positions, in entity order
            std::vector<std::unordered_map<int, int>> foff(nsd);  // face entity -> offset in fpos
            std::vector<long long> w1o(nsd);
            long long w1tot = 0;
            for (int s = 0; s < nsd; ++s) {
                SubInfo& S = hm.sub[s];
                std::vector<int> ev;
                for (size_t q = 0; q < S.ents.size(); ++q) {
                    Entity& E = hm.ent[S.ents[q]];
                    const std::vector<int>& ps = E.pos[S.ent_slot[q]];
                    if (E.kind == 2) {
                        foff[s][S.ents[q]] = (int)fpos[s].size();
                        fpos[s].insert(fpos[s].end(), ps.begin(), ps.end());
                    } else {
                        ev.insert(ev.end(), ps.begin(), ps.end());
                    }
                }
                nEV[s] = (int)ev.size();
                nFP[s] = (int)fpos[s].size();
                w1o[s] = w1tot;
                w1tot += (long long)S.nB * r4(S.nB);
                const int off = (int)permv.size();
                permv.insert(permv.end(), ev.begin(), ev.end());
                permv.insert(permv.end(), fpos[s].begin(), fpos[s].end());
                // from S^(i) in the working precision (in the mixed solver S64 is its FP64 copy:
                // the same values, twice the bytes)
                gj.push_back(GatherJob{nullptr, C->sld[s], S.nB, off, 1, nullptr, r4(S.nB), ST + C->soff[s]});
                items.push_back(EngItem<T>{nullptr, S.nB, nEV[s], r4(S.nB)});
            }
            T* W1 = nullptr;
            BDDC_TRY(C->alloc(&W1, (size_t)std::max(w1tot, 1LL)));
            for (int s = 0; s < nsd; ++s) {
                gj[s].dst = W1 + w1o[s];
                items[s].a = W1 + w1o[s];
            }
            // level 2: per (face, side), from the trailing face block of level 1
            std::vector<long long> f2o;
            long long f2tot = 0;
            for (int e : faces)
                for (int a = 0; a < 2; ++a) {
                    const int s = hm.ent[e].subs[a];
                    f2o.push_back(f2tot);
                    f2tot += (long long)nFP[s] * r4(nFP[s]);
                }
            T* FB = nullptr;
            BDDC_TRY(C->alloc(&FB, (size_t)std::max(f2tot, 1LL)));
            std::vector<GatherJob> gj2;
            std::vector<EngItem<T>> items2;
            std::vector<CopyJob> cj;
            int q = 0;
            for (size_t fi = 0; fi < faces.size(); ++fi) {
                const int e = faces[fi];
                Entity& E = hm.ent[e];
                const int nF = (int)E.dofs.size();
                for (int a = 0; a < 2; ++a, ++q) {
                    const int s = E.subs[a];
                    const int n2 = nFP[s], f0 = foff[s][e];
                    const int off = (int)permv.size();
                    for (int b = 0; b < n2; ++b)
                        if (b < f0 || b >= f0 + nF) permv.push_back(b);
                    for (int b = 0; b < nF; ++b) permv.push_back(f0 + b);
                    const int l1 = r4(hm.sub[s].nB);
                    // (no symmetrisation here: the face GEP reads the symmetric part of its result)
                    gj2.push_back(GatherJob{nullptr, l1, n2, off, 0, FB + f2o[q], r4(n2),
                                            W1 + w1o[s] + (long long)nEV[s] * l1 + nEV[s]});
                    items2.push_back(EngItem<T>{FB + f2o[q], n2, n2 - nF, r4(n2)});
                    cj.push_back(CopyJob{FB + f2o[q], r4(n2), n2 - nF, n2 - nF, nF, nF,
                                         Bt64 + bo[fi] + (long long)a * nF * nF, nF, 1.0});
                }
            }
            BDDC_TRY(C->upload(&d_perm, permv));
            GatherJob* d_gj;
            BDDC_TRY(C->upload(&d_gj, gj));
            BDDC_TRY(gather_perm_run<T>(d_gj, (int)gj.size(), d_perm, 64, st));
            BDDC_TRY(run_engine<T>(C, items));
            GatherJob* d_gj2;
            BDDC_TRY(C->upload(&d_gj2, gj2));
            BDDC_TRY(gather_perm_run<T>(d_gj2, (int)gj2.size(), d_perm, 64, st));
            BDDC_TRY(run_engine<T>(C, items2));
            CopyJob* d_cj;
            BDDC_TRY(C->upload(&d_cj, cj));
            BDDC_TRY((copy_blocks_run<T, double>(d_cj, (int)cj.size(), 8, st)));
        }
        std::vector<FaceJob> fj;
        int maxn = 0;
        for (int e : faces) maxn = std::max(maxn, (int)hm.ent[e].dofs.size());
        const bool eig_global = face_eig_global<T>(maxn);
        for (size_t fi = 0; fi < faces.size(); ++fi) {
            int e = faces[fi];
            Entity& E = hm.ent[e];
            int n = (int)E.dofs.size();
            FaceJob J;
            memset(&J, 0, sizeof(J));
            J.n = n;
            J.mode = face_mode;
            J.theta = E.theta;
            int i = E.subs[0], j = E.subs[1];
            J.Si = C->S64 + C->soff[i];
            J.Sj = C->S64 + C->soff[j];
            J.ldi = C->sld[i];
            J.ldj = C->sld[j];
            J.pi = d_pos + pos_off[e][0];
            J.pj = d_pos + pos_off[e][1];
            J.Bti = Bt64 + bo[fi];
            J.Btj = Bt64 + bo[fi] + (long long)n * n;
            J.ldbi = J.ldbj = n;
            T* fw = nullptr;
            BDDC_TRY(C->alloc(&fw, face_work_doubles(n) + (eig_global ? face_eig_doubles(n) : 0)));
            J.work = fw;
            J.Q = C->Q[e];
            J.DQi = C->DQ[e][0];
            J.DQj = C->DQ[e][1];
            J.lambda = C->lam[e];
            J.neig = C->d_neig + e;
            J.k = C->d_k + e;
            fj.push_back(J);
        }
        FaceJob* d_fj;
        BDDC_TRY(C->upload(&d_fj, fj));
        ktimer_begin(KT_FACE, st);
        BDDC_TRY(face_run<T>(d_fj, (int)fj.size(), maxn, C->err, st));
        ktimer_end(KT_FACE, st, 0.0, 0.0);
    }
    BDDC_CUDA_TRY(cudaMemcpyAsync(C->kk.data(), C->d_k, sizeof(int) * nent, cudaMemcpyDeviceToHost, st));
    BDDC_CUDA_TRY(cudaStreamSynchronize(st));
    for (int e : faces) hm.ent[e].k = C->kk[e];
    C->phase_mark(3);
    // ---- 4. edges --------------------------------------------------------------
    // edge kernel modes: 0 edge GEP on prior-selected primal constraints, 1 all
    // primal, 2 no edge constraints, 3 conventional edge GEP
    const int edge_mode = C->o.all_primal ? 1
                          : C->o.edge_gep == BDDC_EDGE_NEW ? 0
                          : C->o.edge_gep == BDDC_EDGE_OLD ? 3 : 2;
    const bool edge_schur = edge_mode == 0 || edge_mode == 3;   // per-(edge, subdomain) Schur complements
    std::vector<int>& edges = hm.by_kind[1];
    // edge features (always) and the learned skip decision
    C->edge_skipped.assign(edges.size(), 0);
    std::vector<char> active(nsd, 0);
    if (!edges.empty()) {
        std::vector<EdgeDesc> ed(edges.size());
        for (size_t ei = 0; ei < edges.size(); ++ei) {
            Entity& E = hm.ent[edges[ei]];
            EdgeDesc& D = ed[ei];
            auto coords = [&](int d, int* c) {
                c[0] = d % (hm.E[0] - 1) + 1;
                c[1] = (d / (hm.E[0] - 1)) % (hm.E[1] - 1) + 1;
                c[2] = d / ((hm.E[0] - 1) * (hm.E[1] - 1)) + 1;
            };
            int a0[3], a1[3];
            coords(E.dofs.front(), a0);
            coords(E.dofs.back(), a1);
            int axis = -1;
            for (int d = 0; d < 3; ++d)
                if (a0[d] != a1[d]) axis = d;
            if (axis < 0) {   // one-dof edge: the direction in which all owners share a slab
                for (int d = 0; d < 3 && axis < 0; ++d) {
                    bool same = true;
                    int c0 = -1;
                    for (int sd : E.subs) {
                        int sc = d == 0 ? sd % hm.nsub[0] : (d == 1 ? (sd / hm.nsub[0]) % hm.nsub[1] : sd / (hm.nsub[0] * hm.nsub[1]));
                        if (c0 < 0) c0 = sc;
                        else if (sc != c0) same = false;
                    }
                    if (same) axis = d;
                }
            }
            if (axis < 0) return BDDC_EINVAL;
            D.axis = axis;
            D.lo = a0[axis];
            D.hi = a1[axis];
            const int f0 = axis == 0 ? 1 : 0, f1 = axis == 2 ? 1 : 2;
            D.c0 = a0[f0];
            D.c1 = a0[f1];
            D.m = 0;
            D.theta = E.theta;
            for (int q = 0; q < 4; ++q) {
                D.subs[q] = q < (int)E.subs.size() ? E.subs[q] : -1;
                if (q < (int)E.subs.size()) D.m = std::max(D.m, hm.sub[E.subs[q]].max_slab);
            }
        }
        EdgeDesc* d_ed;
        BDDC_TRY(C->upload(&d_ed, ed));
        BDDC_TRY(C->alloc(&C->d_feat, edges.size() * BDDC_MLP_FEATURES));
        BDDC_TRY(mlp_edge_features(d_ed, (int)edges.size(), C->nu, C->beta, C->bconst, d_sx, d_sy, d_sz, hm.nsub[0],
                                   hm.nsub[1], hm.E[0], hm.E[1], hm.h, C->d_feat, st));
        if (edge_mode == 0 && C->o.learned_skip_p >= 0.0 && C->mlp_params) {
            float* probs = nullptr;
            BDDC_TRY(C->alloc(&probs, edges.size() * BDDC_MLP_CLASSES));
            BDDC_TRY(mlp_probs(C->mlp_params, C->d_feat, (int)edges.size(), probs, st));
            std::vector<float> hp(edges.size() * BDDC_MLP_CLASSES);
            BDDC_CUDA_TRY(cudaMemcpyAsync(hp.data(), probs, sizeof(float) * hp.size(), cudaMemcpyDeviceToHost, st));
            BDDC_CUDA_TRY(cudaStreamSynchronize(st));
            for (size_t ei = 0; ei < edges.size(); ++ei)
                C->edge_skipped[ei] = hp[ei * BDDC_MLP_CLASSES] >= (float)C->o.learned_skip_p;
        }
        for (size_t ei = 0; ei < edges.size(); ++ei)
            if (!C->edge_skipped[ei])
                for (int sd : hm.ent[edges[ei]].subs) active[sd] = 1;
        int nsk = 0;
        for (char c : C->edge_skipped) nsk += c;
        C->stats.edges_skipped = nsk;
    }
    if (!edges.empty()) {
        // per subdomain: transformed B onto [face duals | edges, vertices, face primals]
        std::vector<int> idxv;
        std::vector<int> nelim(nsd, 0), nkeep(nsd, 0);
        std::vector<std::map<long long, int>> keypos(nsd);   // H / edge-dof key -> index in W
        std::vector<int> ew_off(nsd, -1);
        auto key_of = [](int kind, int e, int l) -> long long { return ((long long)kind << 40) | ((long long)e << 16) | l; };
        std::vector<TBlock> tb;
        T* W = nullptr;
        double* W64 = nullptr;
        std::vector<long long> woff(nsd, 0), w64off(nsd, 0);
        if (edge_schur) {
            long long wtot = 0, w64tot = 0;
            for (int s = 0; s < nsd; ++s) {
                int nB = hm.sub[s].nB;
                woff[s] = wtot;
                wtot += (long long)nB * r4(nB);
            }
            BDDC_TRY(C->alloc(&W, wtot));
            std::vector<int> perm_off(nsd);
            std::vector<EngItem<T>> items;
            for (int s = 0; s < nsd; ++s) {
                if (!active[s]) continue;
                SubInfo& S = hm.sub[s];
                int nB = S.nB;
                std::vector<int> perm(nB, -1);
                int ne = 0;
                // eliminated: face duals
                for (size_t q = 0; q < S.ents.size(); ++q) {
                    Entity& E = hm.ent[S.ents[q]];
                    if (E.kind != 2) continue;
                    const std::vector<int>& p = E.pos[S.ent_slot[q]];
                    for (int l = E.k; l < (int)p.size(); ++l) perm[p[l]] = ne++;
                }
                int kp = ne;
                for (int kind : {1, 0, 2})
                    for (size_t q = 0; q < S.ents.size(); ++q) {
                        Entity& E = hm.ent[S.ents[q]];
                        if (E.kind != kind) continue;
                        const std::vector<int>& p = E.pos[S.ent_slot[q]];
                        int cnt = kind == 2 ? E.k : (int)p.size();
                        for (int l = 0; l < cnt; ++l) {
                            perm[p[l]] = kp;
                            keypos[s][key_of(kind, S.ents[q], l)] = kp - ne;
                            ++kp;
                        }
                    }
                nelim[s] = ne;
                nkeep[s] = nB - ne;
                perm_off[s] = (int)idxv.size();
                idxv.insert(idxv.end(), perm.begin(), perm.end());
                items.push_back(EngItem<T>{W + woff[s], nB, ne, r4(nB)});
            }
            int posbase = (int)idxv.size();
            idxv.insert(idxv.end(), posl.begin(), posl.end());
            int maxn = 1;
            for (int s = 0; s < nsd; ++s) {
                if (!active[s]) continue;
                SubInfo& S = hm.sub[s];
                for (size_t q = 0; q < S.ents.size(); ++q) {
                    int e = S.ents[q];
                    Entity& E = hm.ent[e];
                    int n = (int)E.dofs.size();
                    TBlock B;
                    memset(&B, 0, sizeof(B));
                    B.src = C->S64 + C->soff[s];
                    B.sld = C->sld[s];
                    B.sym = 1;
                    B.y = nullptr;           // scratch of the two-pass fallback: set by change_basis
                    B.yld = 0;
                    B.n = n;
                    B.pos_off = posbase + pos_off[e][S.ent_slot[q]];
                    B.perm_off = perm_off[s];
                    B.identity = E.kind != 2;
                    B.Q = E.kind == 2 ? C->Q[e] : nullptr;
                    B.nrows = S.nB;
                    B.dst = W + woff[s];
                    B.dld = r4(S.nB);
                    if (E.kind == 2) maxn = std::max(maxn, n);
                    tb.push_back(B);
                }
            }
            int* d_idx;
            BDDC_TRY(C->upload(&d_idx, idxv));
            ktimer_begin(KT_TRANSFORM, st);
            BDDC_TRY(change_basis<T>(C, tb, d_idx, idxv, maxn, st));
            ktimer_end(KT_TRANSFORM, st, 0.0, 0.0);
            BDDC_TRY(run_engine<T>(C, items));
            // trailing blocks to FP64
            std::vector<CopyJob> cj;
            for (int s = 0; s < nsd; ++s) {
                w64off[s] = w64tot;
                w64tot += (long long)nkeep[s] * nkeep[s];
            }
            BDDC_TRY(C->alloc(&W64, w64tot));
            for (int s = 0; s < nsd; ++s)
                if (active[s])
                    cj.push_back(CopyJob{W + woff[s], r4(hm.sub[s].nB), nelim[s], nelim[s], nkeep[s], nkeep[s],
                                         W64 + w64off[s], nkeep[s], 1.0});
            CopyJob* d_cj;
            BDDC_TRY(C->upload(&d_cj, cj));
            BDDC_TRY((copy_blocks_run<T, double>(d_cj, (int)cj.size(), 8, st)));
        }
        // per (edge, subdomain): Schur complement onto [E, H_k]
        std::vector<int> gidxv, hmv;
        std::vector<GatherJob> gj;
        std::vector<EngItem<T>> items;
        std::vector<std::vector<int>> hsz(edges.size()), hoff(edges.size()), itn(edges.size());
        std::vector<std::vector<long long>> ito(edges.size());
        std::vector<int> nH(edges.size(), 0);
        T* EB = nullptr;
        if (edge_schur) {
            long long etot = 0;
            for (size_t ei = 0; ei < edges.size(); ++ei)
                if (!C->edge_skipped[ei])
                    for (int s : hm.ent[edges[ei]].subs) etot += (long long)nkeep[s] * r4(nkeep[s]);
            BDDC_TRY(C->alloc(&EB, etot));
            etot = 0;
            for (size_t ei = 0; ei < edges.size(); ++ei) {
                if (C->edge_skipped[ei]) continue;
                int e = edges[ei];
                Entity& E = hm.ent[e];
                int nE = (int)E.dofs.size();
                // union of H over n(E)
                std::map<long long, int> hu;
                for (int s : E.subs) {
                    SubInfo& S = hm.sub[s];
                    for (size_t q = 0; q < S.ents.size(); ++q) {
                        Entity& X = hm.ent[S.ents[q]];
                        if (X.kind == 0) hu[key_of(0, S.ents[q], 0)] = 0;
                        if (X.kind == 2)
                            for (int l = 0; l < X.k; ++l) hu[key_of(2, S.ents[q], l)] = 0;
                    }
                }
                int cnt = 0;
                for (auto& kv : hu) kv.second = cnt++;
                nH[ei] = cnt;
                for (size_t a = 0; a < E.subs.size(); ++a) {
                    int s = E.subs[a];
                    SubInfo& S = hm.sub[s];
                    std::vector<int> perm, hk;
                    // other edges' dofs first
                    for (size_t q = 0; q < S.ents.size(); ++q) {
                        int x = S.ents[q];
                        Entity& X = hm.ent[x];
                        if (X.kind != 1 || x == e) continue;
                        for (int l = 0; l < (int)X.dofs.size(); ++l) perm.push_back(keypos[s][key_of(1, x, l)]);
                    }
                    int nel = (int)perm.size();
                    for (int l = 0; l < nE; ++l) perm.push_back(keypos[s][key_of(1, e, l)]);
                    for (size_t q = 0; q < S.ents.size(); ++q) {
                        int x = S.ents[q];
                        Entity& X = hm.ent[x];
                        if (X.kind == 0) {
                            perm.push_back(keypos[s][key_of(0, x, 0)]);
                            hk.push_back(hu[key_of(0, x, 0)]);
                        }
                    }
                    for (size_t q = 0; q < S.ents.size(); ++q) {
                        int x = S.ents[q];
                        Entity& X = hm.ent[x];
                        if (X.kind == 2)
                            for (int l = 0; l < X.k; ++l) {
                                perm.push_back(keypos[s][key_of(2, x, l)]);
                                hk.push_back(hu[key_of(2, x, l)]);
                            }
                    }
                    int n = (int)perm.size();
                    int off = (int)gidxv.size();
                    gidxv.insert(gidxv.end(), perm.begin(), perm.end());
                    // rows padded to a multiple of 4 elements (16-byte aligned rows for the engine)
                    const int ldn = r4(n);
                    gj.push_back(GatherJob{W64 + w64off[s], nkeep[s], n, off, 0, EB + etot, ldn, nullptr});
                    items.push_back(EngItem<T>{EB + etot, n, nel, ldn});
                    ito[ei].push_back(etot + (long long)nel * ldn + nel);
                    itn[ei].push_back(ldn);
                    hsz[ei].push_back((int)hk.size());
                    hoff[ei].push_back((int)hmv.size());
                    hmv.insert(hmv.end(), hk.begin(), hk.end());
                    etot += (long long)n * ldn;
                }
            }
            int* d_gi;
            BDDC_TRY(C->upload(&d_gi, gidxv));
            GatherJob* d_gj;
            BDDC_TRY(C->upload(&d_gj, gj));
            BDDC_TRY(gather_perm_run<T>(d_gj, (int)gj.size(), d_gi, 8, st));
            BDDC_TRY(run_engine<T>(C, items));
        }
        int* d_hm = nullptr;
        BDDC_TRY(C->upload(&d_hm, hmv));
        std::vector<EdgeJob> ej;
        int maxnw = 1, maxnz = 1;
        size_t maxwork = 0;
        for (size_t ei = 0; ei < edges.size(); ++ei) {
            int e = edges[ei];
            Entity& E = hm.ent[e];
            int n = (int)E.dofs.size(), m = (int)E.subs.size();
            if (m > EDGE_MAX_SUBS) {
                bddc_set_last_error("an edge shared by more than 4 subdomains", __FILE__, __LINE__);
                return BDDC_EINVAL;
            }
            EdgeJob J;
            memset(&J, 0, sizeof(J));
            J.n = n;
            J.m = m;
            J.nH = nH[ei];
            J.mode = C->edge_skipped[ei] ? 2 : edge_mode;
            J.theta = E.theta;
            for (int a = 0; a < m; ++a) {
                int s = E.subs[a];
                J.S[a] = C->S64 + C->soff[s];
                J.ldS[a] = C->sld[s];
                J.pos[a] = d_pos + pos_off[e][a];
                J.DQ[a] = C->DQ[e][a];
                if (J.mode == 0 || J.mode == 3) {
                    J.Bt[a] = EB + ito[ei][a];
                    J.ldBt[a] = itn[ei][a];
                    J.h[a] = hsz[ei][a];
                    J.hmap[a] = d_hm + hoff[ei][a];
                }
            }
            maxnw = std::max(maxnw, (m - 1) * n);
            maxnz = std::max(maxnz, m * n + J.nH);
            T* ew = nullptr;
            maxwork = std::max(maxwork, edge_work_doubles(n, m, J.nH));
            BDDC_TRY(C->alloc(&ew, edge_work_doubles(n, m, J.nH)));
            J.work = ew;
            BDDC_TRY(C->alloc(&C->BB[e], (size_t)(m - 1) * n * (m - 1) * n));
            J.BBout = C->BB[e];
            J.Q = C->Q[e];
            J.lambda = C->lam[e];
            J.neig = C->d_neig + e;
            J.k = C->d_k + e;
            ej.push_back(J);
        }
        EdgeJob* d_ej;
        BDDC_TRY(C->upload(&d_ej, ej));
        ktimer_begin(KT_EDGE, st);
        BDDC_TRY(edge_run<T>(d_ej, (int)ej.size(), maxnw, maxnz, maxwork, C->err, st));
        ktimer_end(KT_EDGE, st, 0.0, 0.0);
    }
    BDDC_CUDA_TRY(cudaMemcpyAsync(C->kk.data(), C->d_k, sizeof(int) * nent, cudaMemcpyDeviceToHost, st));
    BDDC_CUDA_TRY(cudaMemcpyAsync(C->neig.data(), C->d_neig, sizeof(int) * nent, cudaMemcpyDeviceToHost, st));
    BDDC_CUDA_TRY(cudaStreamSynchronize(st));
    for (int e : edges) hm.ent[e].k = C->kk[e];
    C->phase_mark(4);
    // ---- 5. primal numbering, extended matrices, coarse operators --------------
    int np = 0;
    C->stats.pnumF = C->stats.pnumE = 0;
    for (int kind : {0, 2, 1})
        for (int e : hm.by_kind[kind]) {
            hm.ent[e].prim_off = np;
            np += hm.ent[e].k;
            if (kind == 2) C->stats.pnumF += hm.ent[e].k;
            if (kind == 1) C->stats.pnumE += hm.ent[e].k;
        }
    C->nPi = np;
    const int nPi = np;
    std::vector<int> idxv, rpi_off(nsd), perm_off(nsd);
    C->np_s.assign(nsd, 0);
    std::vector<long long> xoff(nsd);
    std::vector<int> xld(nsd);
    long long xtot = 0;
    for (int s = 0; s < nsd; ++s) {
        SubInfo& S = hm.sub[s];
        std::vector<int> rp;
        for (size_t q = 0; q < S.ents.size(); ++q) {
            Entity& E = hm.ent[S.ents[q]];
            for (int l = 0; l < E.k; ++l) rp.push_back(E.prim_off + l);
        }
        C->np_s[s] = (int)rp.size();
        rpi_off[s] = (int)idxv.size();
        idxv.insert(idxv.end(), rp.begin(), rp.end());
        int nd = S.nB - (int)rp.size();
        std::vector<int> perm(S.nB, -1);
        int cd = 0, cp = nd;
        for (size_t q = 0; q < S.ents.size(); ++q) {
            Entity& E = hm.ent[S.ents[q]];
            const std::vector<int>& p = E.pos[S.ent_slot[q]];
            for (int l = 0; l < (int)p.size(); ++l) perm[p[l]] = l < E.k ? cp++ : cd++;
        }
        perm_off[s] = (int)idxv.size();
        idxv.insert(idxv.end(), perm.begin(), perm.end());
        xld[s] = r4(2 * S.nB);
        xoff[s] = xtot;
        xtot += (long long)2 * S.nB * xld[s];
    }
    int posbase = (int)idxv.size();
    idxv.insert(idxv.end(), posl.begin(), posl.end());
    int* d_idx;
    BDDC_TRY(C->upload(&d_idx, idxv));
    T* X = nullptr;
    BDDC_TRY(C->alloc(&X, xtot));
    BDDC_CUDA_TRY(cudaMemsetAsync(X, 0, xtot * sizeof(T), st));
    {
        std::vector<TBlock> tb;
        std::vector<DTJob> dj;
        int maxn = 1;
        for (int s = 0; s < nsd; ++s) {
            SubInfo& S = hm.sub[s];
            for (size_t q = 0; q < S.ents.size(); ++q) {
                int e = S.ents[q];
                Entity& E = hm.ent[e];
                int n = (int)E.dofs.size();
                TBlock B;
                memset(&B, 0, sizeof(B));
                B.src = C->S64 + C->soff[s];
                B.sld = C->sld[s];
                B.sym = 0;
                B.y = nullptr;
                B.yld = 0;
                B.n = n;
                B.pos_off = posbase + pos_off[e][S.ent_slot[q]];
                B.perm_off = perm_off[s];
                B.identity = E.kind == 0;
                B.Q = E.kind == 0 ? nullptr : C->Q[e];
                B.nrows = S.nB;
                B.dst = X + xoff[s];
                B.dld = xld[s];
                if (E.kind != 0) maxn = std::max(maxn, n);
                tb.push_back(B);
                DTJob D;
                D.n = n;
                D.nB = S.nB;
                D.pos_off = B.pos_off;
                D.perm_off = perm_off[s];
                D.DQ = E.kind == 0 ? nullptr : C->DQ[e][S.ent_slot[q]];
                D.scalar = 1.0 / (double)E.subs.size();
                D.dst = X + xoff[s];
                D.dld = xld[s];
                dj.push_back(D);
            }
        }
        DTJob* d_dj;
        BDDC_TRY(C->upload(&d_dj, dj));
        ktimer_begin(KT_TRANSFORM, st);
        BDDC_TRY(change_basis<T>(C, tb, d_idx, idxv, maxn, st));
        ktimer_end(KT_TRANSFORM, st, 0.0, 0.0);
        BDDC_TRY(fill_dt_run<T>(d_dj, (int)dj.size(), d_idx, st));
        std::vector<EngItem<T>> items;
        for (int s = 0; s < nsd; ++s)
            items.push_back(EngItem<T>{X + xoff[s], 2 * hm.sub[s].nB, hm.sub[s].nB - C->np_s[s], xld[s]});
        BDDC_TRY(run_engine<T>(C, items));
    }
    C->phase_mark(5);
    // operators of the apply
    C->maoff.resize(nsd);
    C->mcoff.resize(nsd);
    C->mald.resize(nsd);
    C->mcld.resize(nsd);
    long long matot = 0, mctot = 0;
    for (int s = 0; s < nsd; ++s) {
        int nB = hm.sub[s].nB;
        C->mald[s] = r4(nB);
        C->maoff[s] = matot;
        matot += (long long)(nB + C->np_s[s]) * C->mald[s];
        C->mcld[s] = r4(nB);                       // D_i Phi_i stored transposed: np x nB
        C->mcoff[s] = mctot;
        mctot += (long long)std::max(C->np_s[s], 1) * C->mcld[s];
    }
    T *MA = nullptr, *MC = nullptr;
    BDDC_TRY(C->alloc(&MA, matot));
    BDDC_TRY(C->alloc(&MC, mctot));
    BDDC_CUDA_TRY(cudaMemsetAsync(MC, 0, mctot * sizeof(T), st));
    C->MA = MA;
    C->MC = MC;
    double* SPi = nullptr;
    BDDC_TRY(C->alloc(&SPi, (size_t)std::max(nPi, 1) * std::max(nPi, 1)));
    BDDC_CUDA_TRY(cudaMemsetAsync(SPi, 0, sizeof(double) * std::max(nPi, 1) * std::max(nPi, 1), st));
    {
        std::vector<ExtractJob> xj(nsd);
        for (int s = 0; s < nsd; ++s)
            xj[s] = ExtractJob{X + xoff[s], xld[s], hm.sub[s].nB, C->np_s[s], rpi_off[s], MA + C->maoff[s],
                               C->mald[s], MC + C->mcoff[s], C->mcld[s]};
        ExtractJob* d_xj;
        BDDC_TRY(C->upload(&d_xj, xj));
        BDDC_TRY((extract_run<T, T>(d_xj, nsd, d_idx, SPi, nPi, 32, st)));
    }
    // coarse inverse (FP64).  Small coarse problems: FP32 Gauss-Jordan + FP64
    // Newton-Schulz, accepted when max |I - S_Pi X| is at the precision's level
    // (read back after the host has built the apply's work items); otherwise, or
    // when rejected, [[S_Pi, -I], [I, 0]] -> S_Pi^{-1} by the elimination engine.
    const int ldc = r4(std::max(nPi, 1));
    bool coarse_done = false;
    const bool coarse_small = nPi > 0 && nPi <= COARSE_GJ_MAX && !C->o.coarse_elim;
    double* hres = reinterpret_cast<double*>(C->hst + 3);    // pinned: max|I - S X|, ||S||, ||X||
    ktimer_begin(KT_COARSE, st);
    if (coarse_small) {
        BDDC_TRY(C->alloc(&C->SPiInv, (size_t)std::max(nPi, 1) * ldc));
        double* work = nullptr;
        double* resid = nullptr;
        BDDC_TRY(C->alloc(&work, 2LL * nPi * nPi));
        BDDC_TRY(C->alloc(&resid, 3));
        const int steps = C->mixed ? 3 : 4;
        int* gjflag = nullptr;                    // a failed FP32 pivot only shows in the residual
        BDDC_TRY(C->alloc(&gjflag, 1));
        BDDC_TRY(coarse_inverse_small(SPi, nPi, C->SPiInv, ldc, work, resid, steps, gjflag, st));
        BDDC_CUDA_TRY(cudaMemcpyAsync(hres, resid, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    // gemv work items
    std::vector<int> gi;
    std::vector<GemvItem> iS, iM1, iC, iM3, iCt, iM1loc, iM1res;
    const int nG = C->nG;
    auto split = [](std::vector<GemvItem>& v, long long moff, int rows, int cols, int ld, int io, int oo,
                    int RB = 32, int CB = 2048) {
        // CB: column-slice width, <= the GEMV kernel's staging width and a multiple of its vector width
        for (int c0 = 0; c0 < cols; c0 += CB)
            for (int r0 = 0; r0 < rows; r0 += RB) {
                GemvItem it;
                it.moff = moff;
                it.rows = rows;
                it.cols = cols;
                it.ld = ld;
                it.iidx_off = io;
                it.oidx_off = oo;
                it.row0 = r0;
                it.nrows = std::min(RB, rows - r0);
                it.col0 = c0;
                it.ncols = std::min(CB, cols - c0);
                v.push_back(it);
            }
    };
    C->maxcols = std::max(nPi, 1);
    // rows per work item: large enough that the gather of a subdomain's input is
    // amortised over many streamed rows, small enough for ~4 items per SM
    long long rows_tot = 0;
    for (int s = 0; s < nsd; ++s) rows_tot += hm.sub[s].nB;
    const int RBs = (int)std::max(32LL, std::min(128LL, (rows_tot / (4 * 152) + 31) / 32 * 32));
    std::vector<int> og_s(nsd);
    for (int s = 0; s < nsd; ++s) {
        SubInfo& S = hm.sub[s];
        int nB = S.nB, nps = C->np_s[s];
        C->maxcols = std::max(C->maxcols, nB);
        int og = (int)gi.size();
        og_s[s] = og;
        gi.insert(gi.end(), S.gidx.begin(), S.gidx.end());
        int orp = (int)gi.size();
        for (int q = 0; q < nps; ++q) gi.push_back(idxv[rpi_off[s] + q]);
        int om1 = (int)gi.size();
        gi.insert(gi.end(), S.gidx.begin(), S.gidx.end());
        for (int q = 0; q < nps; ++q) gi.push_back(nG + idxv[rpi_off[s] + q]);
        split(iS, C->soff[s], nB, nB, C->sld[s], og, og, RBs);
        split(iM1, C->maoff[s], nB + nps, nB, C->mald[s], og, om1, RBs);
        // the one-launch apply: local rows and coarse-restriction rows as separate items
        for (int c0 = 0; c0 < nB; c0 += 2048) {
            const int nc = std::min(2048, nB - c0);
            for (int r0 = 0; r0 < nB; r0 += RBs)
                iM1loc.push_back(GemvItem{C->maoff[s], nB + nps, nB, C->mald[s], og, om1, r0,
                                          std::min(RBs, nB - r0), c0, nc});
            for (int r0 = nB; r0 < nB + nps; r0 += 32)
                iM1res.push_back(GemvItem{C->maoff[s], nB + nps, nB, C->mald[s], og, om1, r0,
                                          std::min(32, nB + nps - r0), c0, nc});
        }
        if (nps > 0) split(iM3, C->mcoff[s], nB, nps, C->mcld[s], orp, og, 256);
        const double ts = sizeof(T), iv = 8.0 + 4.0;   // FP64 value + int32 index per gather/scatter
        C->bytesS += ts * nB * nB + iv * 2.0 * nB;
        C->bytesM1 += ts * (nB + nps) * nB + iv * (nB + nB + nps);
        C->bytesM3 += ts * nB * nps + iv * (nps + nB);
    }
    {
        int oc = (int)gi.size();
        for (int q = 0; q < nPi; ++q) gi.push_back(nG + q);
        int oi = (int)gi.size();
        for (int q = 0; q < nPi; ++q) gi.push_back(q);
        if (nPi > 0) split(iC, 0, nPi, nPi, ldc, oc, oi, 32, 512);
        // the same product inside the one-launch apply: y -> x within [y | x]
        int ty = (int)gi.size();
        for (int q = 0; q < nPi; ++q) gi.push_back(q);
        int tx = (int)gi.size();
        for (int q = 0; q < nPi; ++q) gi.push_back(nPi + q);
        if (nPi > 0) split(iCt, 0, nPi, nPi, ldc, ty, tx, 32, 512);
        C->bytesC = 8.0 * nPi * nPi + 24.0 * nPi;
    }
    BDDC_TRY(C->upload(&C->gidx_pool, gi));
    {
        // rows per S x work item: measured once per shape class and process
        auto build = [&](std::vector<GemvItem>& v, int rb) {
            for (int s = 0; s < nsd; ++s) split(v, C->soff[s], hm.sub[s].nB, hm.sub[s].nB, C->sld[s], og_s[s], og_s[s], rb);
        };
        const auto key = std::make_tuple(nsd, rows_tot, (int)sizeof(T));
        int rb = RBs;
        double us = 0.0;
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto f = g_tune_rows.find(key);
            if (f != g_tune_rows.end()) {
                rb = f->second;
                have = true;
            }
        }
        if (!have) {
            BDDC_TRY(tune_gemv_rows<T>(C, iS, RBs, build, &rb, &us));
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_rows[key] = rb;
        }
        if (rb != RBs) {
            iS.clear();
            build(iS, rb);
        }
        C->stats.gemv_rows = rb;
        C->stats.gemv_tune_us = us;
    }
    BDDC_TRY(C->upload(&C->itS, iS));
    BDDC_TRY(C->upload(&C->itM1, iM1));
    BDDC_TRY(C->upload(&C->itC, iC));
    BDDC_TRY(C->upload(&C->itM3, iM3));
    C->nitS = (int)iS.size();
    C->nitM1 = (int)iM1.size();
    C->nitC = (int)iC.size();
    C->nitM3 = (int)iM3.size();
    // condense / recover items
    BDDC_TRY(build_tri<T>(C, hm.sub, C->aoff, C->ald, false, C->tp));
    if (C->lnd) BDDC_TRY(build_tri<T>(C, C->lnd->child.sub, C->aoffc, C->aldc, true, C->tc));
    if (coarse_small) {
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        // FP64 rounding floor of I - S X: a few n eps ||S|| ||X||; the mixed apply
        // needs the inverse to FP32 accuracy only
        const double floor64 = 8.0 * nPi * 1.11e-16 * hres[1] * hres[2];
        const double target = C->mixed ? std::max(1e-9, floor64) : std::max(1e-14, floor64);
        coarse_done = std::isfinite(hres[0]) && hres[0] <= target;
        C->stats.coarse_path = coarse_done ? 1 : 0;
    }
    NDPlan ndp;
    if (nPi > 0 && !coarse_done && !C->o.coarse_elim) {
        BDDC_TRY(coarse_nd_setup(C, SPi, ndp));
        coarse_done = true;
        C->stats.coarse_path = 2;
    }
    if (nPi > 0 && !coarse_done) {
        if (!C->SPiInv) BDDC_TRY(C->alloc(&C->SPiInv, (size_t)std::max(nPi, 1) * ldc));
        double* Xc = nullptr;
        BDDC_TRY(C->alloc(&Xc, 4LL * nPi * nPi));
        BDDC_TRY(coarse_ext_run(SPi, Xc, nPi, st));
        std::vector<EngItem<double>> it1{EngItem<double>{Xc, 2 * nPi, nPi, 2 * nPi}};
        BDDC_TRY(run_engine<double>(C, it1));
        std::vector<CopyJob> cj{CopyJob{Xc, 2 * nPi, nPi, nPi, nPi, nPi, C->SPiInv, ldc, 1.0}};
        CopyJob* d_cj;
        BDDC_TRY(C->upload(&d_cj, cj));
        BDDC_TRY((copy_blocks_run<double, double>(d_cj, 1, 64, st)));
    }
    ktimer_end(KT_COARSE, st, 0.0, 0.0);
    BDDC_TRY(build_apply_tasks<T>(C, iM1res, iM1loc, iCt, iM3, C->coarse_nd ? &ndp : nullptr));
    C->phase_mark(6);
    return BDDC_OK;
}

// ---------------------------------------------------------------------------
// operators
// ---------------------------------------------------------------------------
template <class T>
static int op_S(bddc_ctx* C, const double* x, double* y, const int* skip) {
    BDDC_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * C->nG, C->st));
    return gemv_run<T>((const T*)C->ST, C->itS, C->nitS, C->gidx_pool, x, y, C->maxcols, 1, 0, 0, C->st, skip,
                       C->bytesS);
}

// zc[0:nG] = M^-1 x with caller-chosen work vectors: zc (nG + nPi; zc[nG:]
// receives the coarse residual) and upi (nPi, the coarse solution), where
// upi == zc + nG + nPi (the nested-dissection sweeps address both through one
// base pointer).
template <class T>
static int op_M_into(bddc_ctx* C, const double* x, double* zc, double* upi, const int* skip) {
    if (C->o.apply_launch == 0 && C->apTasks) {
        BDDC_CUDA_TRY(cudaMemsetAsync(zc, 0, sizeof(double) * (C->nG + 2 * (size_t)C->nPi), C->st));
        return apply_tasks_run<T>(C->apTasks, C->nApRes, C->nApTasks, C->nApLocal, C->apBlocks, C->apCtr, C->nApCtr,
                                  (const T*)C->MA,
                                  C->coarse_nd ? C->ndOps : C->SPiInv, (const T*)C->MC, C->gidx_pool, C->ndIdx, x,
                                  zc, C->nG, C->nPi, C->err, skip, C->apBytes, C->st);
    }
    BDDC_CUDA_TRY(cudaMemsetAsync(zc, 0, sizeof(double) * (C->nG + C->nPi), C->st));
    BDDC_TRY(gemv_run<T>((const T*)C->MA, C->itM1, C->nitM1, C->gidx_pool, x, zc, C->maxcols, 1, 0, 0, C->st, skip,
                         C->bytesM1));
    if (C->nPi > 0) {
        if (C->coarse_nd) {
            BDDC_TRY(coarse_nd_solve(C, zc + C->nG, skip));
        } else {
            BDDC_CUDA_TRY(cudaMemsetAsync(upi, 0, sizeof(double) * C->nPi, C->st));
            BDDC_TRY(gemv_run<double>(C->SPiInv, C->itC, C->nitC, C->gidx_pool, zc, upi, C->maxcols, 1, 0, 0, C->st,
                                      skip, C->bytesC));
        }
        BDDC_TRY(gemv_t_run<T>((const T*)C->MC, C->itM3, C->nitM3, C->gidx_pool, upi, zc, 1, 0, 0, C->st, skip,
                               C->bytesM3));
    }
    return BDDC_OK;
}

template <class T>
static int op_M(bddc_ctx* C, const double* x, const int* skip) {
    return op_M_into<T>(C, x, C->zc, C->uPi, skip);
}

// Executable GMRES graphs of destroyed contexts, per host thread.  A new context
// takes one and updates it from its own capture (cudaGraphExecUpdate succeeds
// when only kernel parameters differ); each executable graph belongs to one live
// context at a time.
namespace {
struct GraphPool {
    std::vector<std::pair<int, cudaGraphExec_t>> execs;     // (device, graph)
    ~GraphPool() {
        for (auto& e : execs) cudaGraphExecDestroy(e.second);
    }
};
thread_local GraphPool g_graph_pool;
}  // namespace

static cudaGraphExec_t graph_pool_take(cudaGraph_t g) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    auto& v = g_graph_pool.execs;
    for (size_t i = v.size(); i-- > 0;) {
        if (v[i].first != dev) continue;
        cudaGraphExec_t e = v[i].second;
        v.erase(v.begin() + (long)i);
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(e, g, &info) == cudaSuccess) return e;
        cudaGetLastError();
        cudaGraphExecDestroy(e);
    }
    return nullptr;
}

static void graph_pool_give(cudaGraphExec_t e) {
    if (!e) return;
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && g_graph_pool.execs.size() < 4)
        g_graph_pool.execs.push_back({dev, e});
    else
        cudaGraphExecDestroy(e);
}

static int norm2(bddc_ctx* C, const double* x, long long n, double* out_host) {
    // uses the spare state slot (never stopped)
    int nchunk = gm_nchunk(n);
    BDDC_TRY(gm_norm2(x, n, C->gst + 1, C->partial, C->st));
    (void)nchunk;
    BDDC_CUDA_TRY(cudaMemcpyAsync(C->hst + 1, C->gst + 1, sizeof(GmState), cudaMemcpyDeviceToHost, C->st));
    BDDC_CUDA_TRY(cudaStreamSynchronize(C->st));
    *out_host = std::sqrt(std::max(C->hst[1].nrm2, 0.0));
    return BDDC_OK;
}

template <class T>
static int gm_iteration(bddc_ctx* C) {
    const long long n = C->nG;
    const int* skip = &C->gst->stop;
    // vcur = V[j] (written by the cycle start or the previous normalisation)
    BDDC_TRY(op_M<T>(C, C->vcur, skip));
    BDDC_TRY(op_S<T>(C, C->zc, C->w, skip));
    BDDC_TRY(gm_pass(0, C->V, n, C->w, n, C->gst, nullptr, C->hh, C->partial, C->st));
    BDDC_TRY(gm_pass(1, C->V, n, C->w, n, C->gst, C->hh, C->hh2, C->partial, C->st));
    BDDC_TRY(gm_pass(2, C->V, n, C->w, n, C->gst, C->hh2, nullptr, C->partial, C->st));
    BDDC_TRY(gm_givens(C->gst, C->H, C->cs, C->sn, C->gv, C->hh, C->hh2, C->st));
    BDDC_TRY(gm_normalize(C->V, n, C->w, n, C->gst, C->vcur, C->st));
    return BDDC_OK;
}

// GMRES on S x = b (device vectors of length nG); x is overwritten.
template <class T>
static int gmres(bddc_ctx* C, const double* b, double* x, double rtol, int max_iter, int* iters,
                 double* relres, int* converged) {
    const long long n = C->nG;
    cudaStream_t st = C->st;
    double bnorm = 0.0;
    BDDC_TRY(norm2(C, b, n, &bnorm));
    BDDC_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    *iters = 0;
    *converged = 0;
    *relres = 0.0;
    if (bnorm == 0.0) {
        *converged = 1;
        return BDDC_OK;
    }
    const int m = C->gm_m;
    GmState init;
    memset(&init, 0, sizeof(init));
    init.m = m;
    init.max_iter = max_iter;
    init.tol = rtol * bnorm;
    BDDC_CUDA_TRY(cudaMemcpyAsync(C->gst, &init, sizeof(init), cudaMemcpyHostToDevice, st));
    const int K = 4;
    const bool use_graph = getenv("BDDC_NO_GRAPH") == nullptr;
    if (use_graph && (C->graph == nullptr || C->graph_iters != K)) {
        if (C->graph) cudaGraphExecDestroy(C->graph);
        C->graph = nullptr;
        cudaGraph_t g;
        BDDC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        g_capturing = true;
        int rc = BDDC_OK;
        for (int q = 0; q < K && rc == BDDC_OK; ++q) rc = gm_iteration<T>(C);
        g_capturing = false;
        cudaError_t ce = cudaStreamEndCapture(st, &g);
        if (rc != BDDC_OK) return rc;
        BDDC_CUDA_TRY(ce);
        size_t nn = 0;
        BDDC_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        BDDC_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &nn));
        C->graph_kernels = 0;
        for (auto& nd : nodes) {
            cudaGraphNodeType ty;
            BDDC_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
            if (ty == cudaGraphNodeTypeKernel) ++C->graph_kernels;
        }
        // an executable graph left by a destroyed context of the same shape is
        // retargeted to this context's buffers (no new instantiation)
        C->graph = graph_pool_take(g);
        if (!C->graph) BDDC_CUDA_TRY(cudaGraphInstantiate(&C->graph, g, 0));
        cudaGraphDestroy(g);
        C->graph_iters = K;
    }
    int total = 0;
    bool first = true;
    while (true) {
        // r = b - S x
        if (first) {
            BDDC_CUDA_TRY(cudaMemcpyAsync(C->r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        } else {
            BDDC_TRY(op_S<T>(C, x, C->r, nullptr));
            BDDC_TRY(vec_axpby(C->r, b, 1.0, -1.0, n, st));
        }
        first = false;
        BDDC_TRY(gm_cycle_start(C->r, n, C->gst, C->gst + 1, C->gv, C->partial, C->V, C->vcur, st));
        for (int guard = 0; guard < 100000; ++guard) {
            BDDC_CUDA_TRY(cudaMemcpyAsync(C->hst, C->gst, sizeof(GmState), cudaMemcpyDeviceToHost, st));
            BDDC_CUDA_TRY(cudaStreamSynchronize(st));
            if (C->hst->stop) break;
            if (use_graph) {
                BDDC_CUDA_TRY(cudaGraphLaunch(C->graph, st));
                bddc_note_launches(C->graph_kernels);
            } else {
                for (int q = 0; q < K; ++q) BDDC_TRY(gm_iteration<T>(C));
            }
        }
        total = C->hst->total;
        if (C->hst->j > 0) {
            if (C->o.cond_est) BDDC_TRY(gm_cond(C->gst, C->H, C->gm_m, C->kmax, st));
            BDDC_TRY(gm_finish(C->V, n, C->gst, C->H, C->gv, C->yy, C->t, n, st));
            BDDC_TRY(op_M<T>(C, C->t, nullptr));
            BDDC_TRY(vec_axpby(x, C->zc, 1.0, 1.0, n, st));
        }
        if (C->hst->converged || total >= max_iter) break;
    }
    // true residual
    BDDC_TRY(op_S<T>(C, x, C->r, nullptr));
    BDDC_TRY(vec_axpby(C->r, b, 1.0, -1.0, n, st));
    double rn = 0.0;
    BDDC_TRY(norm2(C, C->r, n, &rn));
    *iters = total;
    *relres = rn / bnorm;
    *converged = C->hst->converged;
    return BDDC_OK;
}

template <class T>
static int solve_one(bddc_ctx* C, const double* Fdev, double* udev, bddc_stats* stt) {
    cudaStream_t st = C->st;
    HostMesh& hm = C->hm;
    const long long nG = C->nG, ndof = hm.ndof;
    int iters_total = 0, conv = 0, steps = 0;
    double relres = 0.0;
    double Fn = 0.0;
    BDDC_TRY(norm2(C, Fdev, ndof, &Fn));
    if (!C->mixed) {
        BDDC_TRY(condense_all<T>(C, Fdev, C->g, C->ystore, C->Fc, C->yc, 1, st));
        int it = 0;
        BDDC_TRY(gmres<T>(C, C->g, C->xG, C->o.rtol, C->o.max_iter, &it, &relres, &conv));
        iters_total = it;
        BDDC_TRY(recover_all<T>(C, C->xG, C->ystore, udev, C->yc, 1, st));
        steps = 1;
    } else {
        // FP64 iterative refinement on the global system with FP32 BDDC-GMRES as inner solver
        BDDC_CUDA_TRY(cudaMemsetAsync(udev, 0, sizeof(double) * ndof, st));
        BDDC_CUDA_TRY(cudaMemcpyAsync(C->res, Fdev, sizeof(double) * ndof, cudaMemcpyDeviceToDevice, st));
        double rn = Fn;
        for (steps = 0; steps < C->o.max_refine; ++steps) {
            if (Fn == 0.0 || rn <= C->o.rtol * Fn) {
                conv = 1;
                break;
            }
            BDDC_TRY(condense_all<T>(C, C->res, C->g, C->ystore, C->Fc, C->yc, 1, st));
            int it = 0, cv = 0;
            double rr = 0.0;
            // the loosest inner tolerance that still reaches rtol (with a factor-2 margin)
            const double tol_k = std::max(C->o.inner_rtol, 0.5 * C->o.rtol * Fn / rn);
            BDDC_TRY(gmres<T>(C, C->g, C->xG, std::min(tol_k, 0.5), C->o.max_iter - iters_total, &it, &rr, &cv));
            iters_total += it;
            BDDC_TRY(recover_all<T>(C, C->xG, C->ystore, C->corr, C->yc, 1, st));
            BDDC_TRY(vec_axpby(udev, C->corr, 1.0, 1.0, ndof, st));
            BDDC_TRY(stencil_residual(hm, C->stencil, udev, Fdev, C->res, 1, st));
            BDDC_TRY(norm2(C, C->res, ndof, &rn));
            if (iters_total >= C->o.max_iter) {
                ++steps;
                break;
            }
        }
        if (rn <= C->o.rtol * Fn) conv = 1;
        relres = Fn > 0 ? rn / Fn : 0.0;
    }
    // global FP64 residual
    BDDC_TRY(stencil_residual(hm, C->stencil, udev, Fdev, C->res, 1, st));
    double rg = 0.0;
    BDDC_TRY(norm2(C, C->res, ndof, &rg));
    stt->iters = iters_total;
    stt->refine_steps = steps;
    stt->converged = conv;
    stt->relres = relres;
    stt->relres_global = Fn > 0 ? rg / Fn : 0.0;
    return conv ? BDDC_OK : BDDC_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------
// Several right-hand sides at once: independent GMRES runs (one Krylov space
// per column) in lockstep.  Every operator launch streams each subdomain's
// matrices once for all columns (the GEMV kernels loop over the columns of a
// work item while its matrix slice is in cache); the Arnoldi / Givens kernels
// carry a column grid dimension with one GmState per column, and a column that
// has converged or reached the cap stops through its own stop flag.
// ---------------------------------------------------------------------------
constexpr int BDDC_BATCH_MAX = 64;   // columns per batched solve

struct BatchWS {
    int nb = 0;
    long long ldz = 0;                 // column stride of zc: [z (nG) | y (nPi) | x (nPi)]
    GmBatch B;
    double *V = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *gv = nullptr, *hh = nullptr, *hh2 = nullptr,
           *yy = nullptr, *partial = nullptr, *w = nullptr, *vcur = nullptr, *t = nullptr, *r = nullptr,
           *zc = nullptr, *g = nullptr, *xG = nullptr, *ystore = nullptr, *res = nullptr, *corr = nullptr,
           *Fin = nullptr, *uglob = nullptr, *Fc = nullptr, *yc = nullptr;
    GmState* gst = nullptr;            // nb states, then nb spare states (plain reductions)
    GmState* hst = nullptr;            // pinned host copy of the nb states
    int* allstop = nullptr;
    cudaGraphExec_t graph = nullptr;
    unsigned long long graph_kernels = 0;
    ~BatchWS() {
        if (graph) cudaGraphExecDestroy(graph);
        if (hst) cudaFreeHost(hst);
    }
};

static int batch_ws(bddc_ctx* C, int nb, BatchWS** out) {
    if (C->bw && C->bw->nb == nb) {
        *out = C->bw;
        return BDDC_OK;
    }
    delete C->bw;
    C->bw = nullptr;
    BatchWS* W = new BatchWS();
    const long long nG = C->nG, ndof = C->hm.ndof, m = C->gm_m;
    const long long nchunk = gm_nchunk(std::max(nG, ndof));
    W->nb = nb;
    W->ldz = nG + 2LL * C->nPi;
    W->B = GmBatch{nb, (m + 1) * nG, nG, (m + 1) * (m + 1), m + 2, (m + 9) * (nchunk + 1)};
    int rc = BDDC_OK;
    auto A = [&](double** p, long long n) {
        if (rc == BDDC_OK) rc = C->alloc(p, (size_t)n);
    };
    A(&W->V, W->B.sV * nb);
    A(&W->H, W->B.sH * nb);
    A(&W->cs, W->B.sSm * nb);
    A(&W->sn, W->B.sSm * nb);
    A(&W->gv, W->B.sSm * nb);
    A(&W->hh, W->B.sSm * nb);
    A(&W->hh2, W->B.sSm * nb);
    A(&W->yy, W->B.sSm * nb);
    A(&W->partial, W->B.sP * nb);
    A(&W->w, nG * nb);
    A(&W->vcur, nG * nb);
    A(&W->t, nG * nb);
    A(&W->r, nG * nb);
    A(&W->g, nG * nb);
    A(&W->xG, nG * nb);
    A(&W->zc, W->ldz * nb);
    A(&W->ystore, C->tp.ny * nb);
    if (C->lnd) {
        A(&W->Fc, ndof * nb);
        A(&W->yc, C->tc.ny * nb);
    }
    A(&W->res, ndof * nb);
    A(&W->corr, ndof * nb);
    A(&W->Fin, ndof * nb);
    A(&W->uglob, ndof * nb);
    if (rc == BDDC_OK) rc = C->alloc(&W->gst, 2 * (size_t)nb);
    if (rc == BDDC_OK && cudaMemsetAsync(W->gst, 0, sizeof(GmState) * 2 * nb, C->st) != cudaSuccess) rc = BDDC_ECUDA;
    if (rc == BDDC_OK) rc = C->alloc(&W->allstop, 1);
    if (rc == BDDC_OK && cudaMallocHost(&W->hst, sizeof(GmState) * nb) != cudaSuccess) rc = BDDC_ENOMEM;
    if (rc != BDDC_OK) {
        delete W;
        return rc;
    }
    C->bw = W;
    *out = W;
    return BDDC_OK;
}

template <class T>
static int op_S_multi(bddc_ctx* C, const double* x, long long ldx, double* y, int nb, const int* skip) {
    BDDC_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * C->nG * nb, C->st));
    return gemv_run<T>((const T*)C->ST, C->itS, C->nitS, C->gidx_pool, x, y, C->maxcols, nb, (int)ldx, C->nG, C->st,
                       skip, C->bytesS);
}

// zc (column stride ldz) = [M^-1 x | coarse residual | coarse solution] for nb columns
template <class T>
static int op_M_multi(bddc_ctx* C, const double* x, double* zc, long long ldz, int nb, const int* skip) {
    cudaStream_t st = C->st;
    BDDC_CUDA_TRY(cudaMemsetAsync(zc, 0, sizeof(double) * ldz * nb, st));
    BDDC_TRY(gemv_run<T>((const T*)C->MA, C->itM1, C->nitM1, C->gidx_pool, x, zc, C->maxcols, nb, C->nG, (int)ldz, st,
                         skip, C->bytesM1));
    if (C->nPi == 0) return BDDC_OK;
    double* y2 = zc + C->nG;
    double* upi = y2 + C->nPi;
    if (C->coarse_nd) {
        for (size_t h = 0; h + 1 < C->ndFwdOff.size(); ++h) {
            const int a = C->ndFwdOff[h], b = C->ndFwdOff[h + 1];
            if (b > a)
                BDDC_TRY(gemv_run<double>(C->ndOps, C->ndFwd + a, b - a, C->ndIdx, y2, y2, 0, nb, (int)ldz, (int)ldz,
                                          st, skip, C->ndFwdBytes[h]));
        }
        for (size_t d = 0; d + 1 < C->ndBwdOff.size(); ++d) {
            const int a = C->ndBwdOff[d], b = C->ndBwdOff[d + 1];
            if (b > a)
                BDDC_TRY(gemv_run<double>(C->ndOps, C->ndBwd + a, b - a, C->ndIdx, y2, y2, 0, nb, (int)ldz, (int)ldz,
                                          st, skip, C->ndBwdBytes[d]));
        }
    } else {
        BDDC_TRY(gemv_run<double>(C->SPiInv, C->itC, C->nitC, C->gidx_pool, zc, upi, C->maxcols, nb, (int)ldz,
                                  (int)ldz, st, skip, C->bytesC));
    }
    return gemv_t_run<T>((const T*)C->MC, C->itM3, C->nitM3, C->gidx_pool, upi, zc, nb, (int)ldz, (int)ldz, st, skip,
                         C->bytesM3);
}

template <class T>
static int gm_iteration_batch(bddc_ctx* C, BatchWS* W) {
    const long long n = C->nG;
    const int* skip = W->allstop;
    BDDC_TRY(op_M_multi<T>(C, W->vcur, W->zc, W->ldz, W->nb, skip));
    BDDC_TRY(op_S_multi<T>(C, W->zc, W->ldz, W->w, W->nb, skip));
    BDDC_TRY(gm_pass(0, W->V, n, W->w, n, W->gst, nullptr, W->hh, W->partial, C->st, W->B));
    BDDC_TRY(gm_pass(1, W->V, n, W->w, n, W->gst, W->hh, W->hh2, W->partial, C->st, W->B));
    BDDC_TRY(gm_pass(2, W->V, n, W->w, n, W->gst, W->hh2, nullptr, W->partial, C->st, W->B));
    BDDC_TRY(gm_givens(W->gst, W->H, W->cs, W->sn, W->gv, W->hh, W->hh2, C->st, W->B));
    BDDC_TRY(gm_normalize(W->V, n, W->w, n, W->gst, W->vcur, C->st, W->B));
    return gm_all_stopped(W->gst, W->nb, W->allstop, C->st);
}

// Column norms ||x_c|| of nb vectors of length n (stride ld = n) through the spare states.
static int norms_batch(bddc_ctx* C, BatchWS* W, const double* x, long long n, int nb, double* out) {
    GmBatch B = W->B;
    B.ncol = nb;
    B.sW = n;
    BDDC_TRY(gm_norm2(x, n, W->gst + W->nb, W->partial, C->st, B));
    BDDC_CUDA_TRY(cudaMemcpyAsync(W->hst, W->gst + W->nb, sizeof(GmState) * nb, cudaMemcpyDeviceToHost, C->st));
    BDDC_CUDA_TRY(cudaStreamSynchronize(C->st));
    for (int c = 0; c < nb; ++c) out[c] = std::sqrt(std::max(W->hst[c].nrm2, 0.0));
    return BDDC_OK;
}

// GMRES on S X = Bm for the columns of Bm (nG x nb); tol[c] is the absolute
// residual target of column c (< 0: the column is left at zero).  X is
// overwritten; iters[c], conv[c] and the true relative residuals are returned.
template <class T>
static int gmres_batch(bddc_ctx* C, BatchWS* W, const double* Bm, double* X, const double* tol, const double* bnorm,
                       const int* max_iter, int* iters, int* conv, double* relres) {
    const long long n = C->nG;
    const int nb = W->nb;
    cudaStream_t st = C->st;
    BDDC_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(double) * n * nb, st));
    std::vector<GmState> init(2 * (size_t)nb);
    memset(init.data(), 0, sizeof(GmState) * init.size());
    bool any = false;
    for (int c = 0; c < nb; ++c) {
        init[c].m = C->gm_m;
        init[c].max_iter = max_iter[c];
        init[c].tol = tol[c];
        init[c].done = (tol[c] < 0.0 || bnorm[c] == 0.0) ? 1 : 0;
        init[c].converged = init[c].done;
        iters[c] = 0;
        conv[c] = init[c].done;
        relres[c] = 0.0;
        any = any || !init[c].done;
    }
    if (!any) return BDDC_OK;
    BDDC_CUDA_TRY(cudaMemcpyAsync(W->gst, init.data(), sizeof(GmState) * 2 * nb, cudaMemcpyHostToDevice, st));
    const int K = 4;
    const bool use_graph = getenv("BDDC_NO_GRAPH") == nullptr;
    if (use_graph && W->graph == nullptr) {
        cudaGraph_t gr;
        BDDC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        g_capturing = true;
        int rc = BDDC_OK;
        for (int q = 0; q < K && rc == BDDC_OK; ++q) rc = gm_iteration_batch<T>(C, W);
        g_capturing = false;
        cudaError_t ce = cudaStreamEndCapture(st, &gr);
        if (rc != BDDC_OK) return rc;
        BDDC_CUDA_TRY(ce);
        size_t nn = 0;
        BDDC_CUDA_TRY(cudaGraphGetNodes(gr, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        BDDC_CUDA_TRY(cudaGraphGetNodes(gr, nodes.data(), &nn));
        W->graph_kernels = 0;
        for (auto& nd : nodes) {
            cudaGraphNodeType ty;
            BDDC_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
            if (ty == cudaGraphNodeTypeKernel) ++W->graph_kernels;
        }
        BDDC_CUDA_TRY(cudaGraphInstantiate(&W->graph, gr, 0));
        cudaGraphDestroy(gr);
    }
    std::vector<GmState> hs(nb);
    bool first = true;
    while (true) {
        if (first) {
            BDDC_CUDA_TRY(cudaMemcpyAsync(W->r, Bm, sizeof(double) * n * nb, cudaMemcpyDeviceToDevice, st));
        } else {
            BDDC_TRY(op_S_multi<T>(C, X, n, W->r, nb, nullptr));
            BDDC_TRY(vec_axpby_cols(W->r, n, Bm, n, 1.0, -1.0, n, nb, st));
        }
        first = false;
        BDDC_TRY(gm_cycle_start(W->r, n, W->gst, W->gst + nb, W->gv, W->partial, W->V, W->vcur, st, W->B));
        BDDC_TRY(gm_all_stopped(W->gst, nb, W->allstop, st));
        for (int guard = 0; guard < 100000; ++guard) {
            BDDC_CUDA_TRY(cudaMemcpyAsync(W->hst, W->gst, sizeof(GmState) * nb, cudaMemcpyDeviceToHost, st));
            BDDC_CUDA_TRY(cudaStreamSynchronize(st));
            bool all = true;
            for (int c = 0; c < nb; ++c) all = all && W->hst[c].stop;
            if (all) break;
            if (use_graph) {
                BDDC_CUDA_TRY(cudaGraphLaunch(W->graph, st));
                bddc_note_launches(W->graph_kernels);
            } else {
                for (int q = 0; q < K; ++q) BDDC_TRY(gm_iteration_batch<T>(C, W));
            }
        }
        if (C->o.cond_est) BDDC_TRY(gm_cond(W->gst, W->H, C->gm_m, C->kmax, st, W->B));
        BDDC_TRY(gm_finish(W->V, n, W->gst, W->H, W->gv, W->yy, W->t, n, st, W->B));
        BDDC_TRY(op_M_multi<T>(C, W->t, W->zc, W->ldz, nb, nullptr));
        BDDC_TRY(vec_axpby_cols(X, n, W->zc, W->ldz, 1.0, 1.0, n, nb, st));
        // columns that converged or reached the cap are done; the others restart
        BDDC_CUDA_TRY(cudaMemcpyAsync(hs.data(), W->gst, sizeof(GmState) * nb, cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        bool all_done = true;
        for (int c = 0; c < nb; ++c) {
            if (!hs[c].done && (hs[c].converged || hs[c].total >= max_iter[c])) hs[c].done = 1;
            all_done = all_done && hs[c].done;
        }
        if (all_done) break;
        BDDC_CUDA_TRY(cudaMemcpyAsync(W->gst, hs.data(), sizeof(GmState) * nb, cudaMemcpyHostToDevice, st));
    }
    // true residuals
    BDDC_TRY(op_S_multi<T>(C, X, n, W->r, nb, nullptr));
    BDDC_TRY(vec_axpby_cols(W->r, n, Bm, n, 1.0, -1.0, n, nb, st));
    std::vector<double> rn(nb);
    BDDC_TRY(norms_batch(C, W, W->r, n, nb, rn.data()));
    for (int c = 0; c < nb; ++c) {
        iters[c] = hs[c].total;
        conv[c] = init[c].done ? 1 : hs[c].converged;
        relres[c] = bnorm[c] > 0 ? rn[c] / bnorm[c] : 0.0;
    }
    return BDDC_OK;
}

// The whole solve (condensation, GMRES, recovery; MIXED: FP64 refinement) for
// nb columns F (ndof x nb, device) -> U (ndof x nb, device).
template <class T>
static int solve_batch(bddc_ctx* C, BatchWS* W, const double* F, double* U, bddc_stats* stt) {
    cudaStream_t st = C->st;
    HostMesh& hm = C->hm;
    const long long nG = C->nG, ndof = hm.ndof;
    const int nb = W->nb;
    std::vector<double> Fn(nb), rn(nb), bn(nb), tol(nb), rr(nb);
    std::vector<int> it(nb), cv(nb), itot(nb, 0), steps(nb, 0), convd(nb, 0);
    BDDC_TRY(norms_batch(C, W, F, ndof, nb, Fn.data()));
    auto condense_cols = [&](const double* R) -> int {
        return condense_all<T>(C, R, W->g, W->ystore, W->Fc, W->yc, nb, st);
    };
    double relres_max = 0.0;
    if (!C->mixed) {
        BDDC_TRY(condense_cols(F));
        BDDC_TRY(norms_batch(C, W, W->g, nG, nb, bn.data()));
        std::vector<int> caps(nb, C->o.max_iter);
        for (int c = 0; c < nb; ++c) tol[c] = C->o.rtol * bn[c];
        BDDC_TRY(gmres_batch<T>(C, W, W->g, W->xG, tol.data(), bn.data(), caps.data(), it.data(), cv.data(),
                                rr.data()));
        BDDC_TRY(recover_all<T>(C, W->xG, W->ystore, U, W->yc, nb, st));
        for (int c = 0; c < nb; ++c) {
            itot[c] = it[c];
            steps[c] = 1;
            convd[c] = cv[c];
            relres_max = std::max(relres_max, rr[c]);
        }
    } else {
        BDDC_CUDA_TRY(cudaMemsetAsync(U, 0, sizeof(double) * ndof * nb, st));
        BDDC_CUDA_TRY(cudaMemcpyAsync(W->res, F, sizeof(double) * ndof * nb, cudaMemcpyDeviceToDevice, st));
        for (int c = 0; c < nb; ++c) rn[c] = Fn[c];
        for (int step = 0; step < C->o.max_refine; ++step) {
            bool any = false;
            for (int c = 0; c < nb; ++c) {
                const bool done = Fn[c] == 0.0 || rn[c] <= C->o.rtol * Fn[c] || itot[c] >= C->o.max_iter;
                if (done) convd[c] = convd[c] || Fn[c] == 0.0 || rn[c] <= C->o.rtol * Fn[c];
                any = any || !done;
            }
            if (!any) break;
            BDDC_TRY(condense_cols(W->res));
            BDDC_TRY(norms_batch(C, W, W->g, nG, nb, bn.data()));
            std::vector<int> caps(nb, 0);
            for (int c = 0; c < nb; ++c) {
                const bool done = Fn[c] == 0.0 || rn[c] <= C->o.rtol * Fn[c] || itot[c] >= C->o.max_iter;
                const double tk = std::min(std::max(C->o.inner_rtol, 0.5 * C->o.rtol * Fn[c] / rn[c]), 0.5);
                tol[c] = done ? -1.0 : tk * bn[c];
                caps[c] = C->o.max_iter - itot[c];
                if (!done) ++steps[c];
            }
            BDDC_TRY(gmres_batch<T>(C, W, W->g, W->xG, tol.data(), bn.data(), caps.data(), it.data(), cv.data(),
                                    rr.data()));
            for (int c = 0; c < nb; ++c)
                if (tol[c] >= 0.0) itot[c] += it[c];
            BDDC_TRY(recover_all<T>(C, W->xG, W->ystore, W->corr, W->yc, nb, st));
            BDDC_TRY(vec_axpby_cols(U, ndof, W->corr, ndof, 1.0, 1.0, ndof, nb, st));
            BDDC_TRY(stencil_residual(hm, C->stencil, U, F, W->res, nb, st));
            BDDC_TRY(norms_batch(C, W, W->res, ndof, nb, rn.data()));
        }
        for (int c = 0; c < nb; ++c) {
            convd[c] = convd[c] || Fn[c] == 0.0 || rn[c] <= C->o.rtol * Fn[c];
            relres_max = std::max(relres_max, Fn[c] > 0 ? rn[c] / Fn[c] : 0.0);
        }
    }
    BDDC_TRY(stencil_residual(hm, C->stencil, U, F, W->res, nb, st));
    BDDC_TRY(norms_batch(C, W, W->res, ndof, nb, rn.data()));
    double rg = 0.0;
    int conv_all = 1, iters = 0, nsteps = 0;
    for (int c = 0; c < nb; ++c) {
        rg = std::max(rg, Fn[c] > 0 ? rn[c] / Fn[c] : 0.0);
        conv_all = conv_all && convd[c];
        iters += itot[c];
        nsteps += steps[c];
    }
    stt->iters = iters;
    stt->refine_steps = nsteps;
    stt->converged = conv_all;
    stt->relres = relres_max;
    stt->relres_global = rg;
    return conv_all ? BDDC_OK : BDDC_NOT_CONVERGED;
}

int bddc_ctx_device(const bddc_ctx* C) { return C ? C->device : -1; }

int bddc_apply_into(bddc_ctx* C, const double* r, double* z, int nrhs, double* work, size_t work_doubles) {
    if (!C || !r || !z || nrhs < 1 || !work) return BDDC_EINVAL;
    const size_t need = (size_t)C->nG + 2 * (size_t)C->nPi;
    if (need > work_doubles) {
        bddc_set_last_error("interface + 2 x coarse size exceeds the static work array", __FILE__, __LINE__);
        return BDDC_EINVAL;
    }
    double* zc = work;
    double* upi = work + C->nG + C->nPi;
    for (int c = 0; c < nrhs; ++c) {
        if (C->mixed) BDDC_TRY(op_M_into<float>(C, r + (long long)c * C->nG, zc, upi, nullptr));
        else BDDC_TRY(op_M_into<double>(C, r + (long long)c * C->nG, zc, upi, nullptr));
        BDDC_CUDA_TRY(cudaMemcpyAsync(z + (long long)c * C->nG, zc, sizeof(double) * C->nG,
                                      cudaMemcpyDeviceToDevice, C->st));
    }
    return BDDC_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void bddc_default_opts(bddc_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->theta_E = 10.0;
    o->theta_F = 0.0;
    o->tau = 0.7;
    o->precision = BDDC_PREC_FP64;
    o->restart = 0;
    o->max_iter = 300;
    o->rtol = 1e-8;
    o->edge_gep = BDDC_EDGE_NEW;
    o->face_gep = 1;
    o->all_primal = 0;
    o->inner_rtol = 1e-6;
    o->max_refine = 8;
    o->learned_skip_p = -1.0;
    o->mlp_params = nullptr;
    o->tensor_cores = 1;
    o->coarse_elim = 0;
    o->apply_launch = 0;
    o->cond_est = 1;
    o->element = BDDC_ELEM_Q1;
    o->local_nd = 0;
}

const char* bddc_last_error(void) { return g_last_error.c_str(); }

const char* bddc_strerror(int code) {
    switch (code) {
        case BDDC_OK: return "ok";
        case BDDC_NOT_CONVERGED: return "GMRES did not reach the tolerance";
        case BDDC_EINVAL: return "invalid argument";
        case BDDC_ENOMEM: return "out of device or host memory";
        case BDDC_ECUDA: return g_last_error.empty() ? "CUDA error" : g_last_error.c_str();
        case BDDC_EGEP: return "eigen iteration cap reached";
        case BDDC_ETIMEOUT: return "bounded device wait gave up";
        case BDDC_ENUMERIC: return "zero or non-finite pivot";
        default: return "unknown error";
    }
}

void bddc_destroy(bddc_ctx* C) {
    if (!C) return;
    if (C->st) cudaStreamSynchronize(C->st);     // the graph may still be running
    delete C->bw;
    graph_pool_give(C->graph);
    for (void* p : C->allocs) cudaFreeAsync(p, C->st);
    if (C->st) cudaStreamSynchronize(C->st);
    for (cudaEvent_t e : C->phase_ev)
        if (e) cudaEventDestroy(e);
    if (C->own) cudaStreamDestroy(C->own);
    delete C;
}

// Pinned host slots for the small device->host reads of the solve; one block
// per host thread, reused by every context the thread drives (each call
// synchronises before it reads them).
static int pinned_scratch(GmState** out) {
    static thread_local GmState* block = nullptr;
    if (!block) BDDC_CUDA_TRY(cudaMallocHost(&block, 4 * sizeof(GmState)));
    *out = block;
    return BDDC_OK;
}

// Keep freed device memory in the stream-ordered pool of each device so that
// repeated setups reuse it instead of returning it to the driver.
static int keep_pool_memory() {
    int dev = 0;
    BDDC_CUDA_TRY(cudaGetDevice(&dev));
    static std::mutex mu;
    static bool done[256] = {false};
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 256 && !done[dev]) {
        cudaMemPool_t pool;
        BDDC_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
        unsigned long long thr = ~0ULL;
        BDDC_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        done[dev] = true;
    }
    return BDDC_OK;
}

static int copy_coeff(bddc_ctx* C, double** dst, const double* src, size_t n, int mem) {
    *dst = nullptr;
    if (!src) return BDDC_OK;
    BDDC_TRY(C->alloc(dst, n));
    BDDC_CUDA_TRY(cudaMemcpyAsync(*dst, src, n * sizeof(double),
                                  mem == BDDC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, C->st));
    return BDDC_OK;
}

static int setup_body(bddc_ctx* C, const bddc_mesh* mesh, const bddc_coeffs* k, const bddc_partition* part) {
    const auto t0 = std::chrono::steady_clock::now();
    BDDC_TRY(stage_reset());
    BDDC_TRY(build_host_boxes(mesh, part, C->hm));
    HostMesh& hm = C->hm;
    if (C->o.local_nd != 0 && C->o.local_nd != 1) {
        bddc_set_last_error("local_nd must be 0 or 1", __FILE__, __LINE__);
        return BDDC_EINVAL;
    }
    if (!C->o.local_nd)          // (with local_nd the children and separators are checked at setup)
        for (const SubInfo& S : hm.sub)
            if (S.nI > BDDC_MAX_INTERIOR) {
                bddc_set_last_error("subdomain interior larger than the interior-solve limit", __FILE__, __LINE__);
                return BDDC_EINVAL;
            }
    if (!k || !k->nu_elem) return BDDC_EINVAL;
    if (k->mem != BDDC_MEM_HOST && k->mem != BDDC_MEM_DEVICE) return BDDC_EINVAL;
    if (C->o.element != BDDC_ELEM_Q1 && C->o.element != BDDC_ELEM_P1) {
        bddc_set_last_error("element must be BDDC_ELEM_Q1 or BDDC_ELEM_P1", __FILE__, __LINE__);
        return BDDC_EINVAL;
    }
    if (!std::isfinite(k->c) || !std::isfinite(k->beta_const[0]) || !std::isfinite(k->beta_const[1]) ||
        !std::isfinite(k->beta_const[2])) {
        bddc_set_last_error("reaction and constant velocity must be finite", __FILE__, __LINE__);
        return BDDC_EINVAL;
    }
    BDDC_TRY(copy_coeff(C, &C->nu, k->nu_elem, hm.nelem, k->mem));
    BDDC_TRY(copy_coeff(C, &C->beta, k->beta_node, 3 * (size_t)hm.nnodes, k->mem));
    BDDC_TRY(copy_coeff(C, &C->f, k->f_node, hm.nnodes, k->mem));
    BDDC_TRY(copy_coeff(C, &C->divb, k->divb_node, hm.nnodes, k->mem));
    BDDC_TRY(copy_coeff(C, &C->gdir, k->g_node, hm.nnodes, k->mem));
    {
        // the coefficient arrays (host or device) are checked on the device before any other work
        int* vflag = nullptr;
        BDDC_TRY(C->alloc(&vflag, 1));
        BDDC_TRY(validate_coeffs_run(C->nu, hm.nelem, C->beta, C->f, C->divb, C->gdir, hm.nnodes, vflag, C->st));
        int hv = 0;
        BDDC_CUDA_TRY(cudaMemcpyAsync(&hv, vflag, sizeof(int), cudaMemcpyDeviceToHost, C->st));
        BDDC_CUDA_TRY(cudaStreamSynchronize(C->st));
        if (hv) {
            bddc_set_last_error("nu must be positive and finite; beta, f, div(beta) and the Dirichlet values finite",
                                __FILE__, __LINE__);
            return BDDC_EINVAL;
        }
    }
    for (int d = 0; d < 3; ++d) C->bconst[d] = k->beta_const[d];
    C->c = k->c;
    if (C->o.mlp_params && C->o.learned_skip_p >= 0.0) {
        std::vector<float> hp(C->o.mlp_params, C->o.mlp_params + BDDC_MLP_PARAMS);
        BDDC_TRY(C->upload(&C->mlp_params, hp));
    }
    BDDC_TRY(C->alloc(&C->err, 2));        // [0] error flags, [1] largest Jacobi sweep count
    BDDC_CUDA_TRY(cudaMemsetAsync(C->err, 0, 2 * sizeof(int), C->st));
    BDDC_TRY(pinned_scratch(&C->hst));
    C->stats.t_mesh_ms = ms_since(t0);
    if (C->mixed) BDDC_TRY(setup_impl<float>(C));
    else BDDC_TRY(setup_impl<double>(C));
    // solve buffers
    const long long nG = C->nG, ndof = hm.ndof;
    BDDC_TRY(C->alloc(&C->zc, nG + 2 * (long long)C->nPi + 1));
    C->uPi = C->zc + nG + C->nPi;
    BDDC_TRY(C->alloc(&C->g, nG));
    BDDC_TRY(C->alloc(&C->xG, nG));
    BDDC_TRY(C->alloc(&C->r, nG));
    BDDC_TRY(C->alloc(&C->w, nG));
    BDDC_TRY(C->alloc(&C->vcur, nG));
    BDDC_TRY(C->alloc(&C->t, nG));
    BDDC_TRY(C->alloc(&C->res, ndof));
    BDDC_TRY(C->alloc(&C->corr, ndof));
    BDDC_TRY(C->alloc(&C->uglob, ndof));
    BDDC_TRY(C->alloc(&C->Fin, ndof));
    BDDC_TRY(C->alloc(&C->ystore, C->tp.ny));
    if (C->lnd) {
        BDDC_TRY(C->alloc(&C->Fc, ndof));
        BDDC_TRY(C->alloc(&C->yc, C->tc.ny));
    }
    BDDC_TRY(C->upload(&C->gamma_dofs, hm.gamma));
    int m = C->o.restart > 0 ? std::min(C->o.restart, C->o.max_iter) : C->o.max_iter;
    m = std::max(m, 1);
    C->gm_m = m;
    BDDC_TRY(C->alloc(&C->V, (size_t)(m + 1) * nG));
    BDDC_TRY(C->alloc(&C->H, (size_t)(m + 1) * (m + 1)));
    BDDC_TRY(C->alloc(&C->cs, m + 1));
    BDDC_TRY(C->alloc(&C->sn, m + 1));
    BDDC_TRY(C->alloc(&C->gv, m + 2));
    BDDC_TRY(C->alloc(&C->hh, m + 2));
    BDDC_TRY(C->alloc(&C->hh2, m + 2));
    BDDC_TRY(C->alloc(&C->yy, m + 1));
    BDDC_TRY(C->alloc(&C->partial, (size_t)(m + 9) * (gm_nchunk(std::max(nG, ndof)) + 1)));
    BDDC_TRY(C->alloc(&C->gst, 2));
    BDDC_TRY(C->alloc(&C->kmax, 1));
    BDDC_CUDA_TRY(cudaMemsetAsync(C->gst, 0, 2 * sizeof(GmState), C->st));
    int herr2[2] = {0, 0};
    BDDC_CUDA_TRY(cudaMemcpyAsync(herr2, C->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, C->st));
    BDDC_CUDA_TRY(cudaStreamSynchronize(C->st));
    const int herr = herr2[0];
    C->stats.jacobi_sweeps_max = herr2[1];
    C->stats.t_assemble_ms = C->phase_ms(0, 1);
    C->stats.t_factor_ms = C->phase_ms(1, 2);
    C->stats.t_face_ms = C->phase_ms(2, 3);
    C->stats.t_edge_ms = C->phase_ms(3, 4);
    C->stats.t_basis_ms = C->phase_ms(4, 5);
    C->stats.t_coarse_ms = C->phase_ms(4, 6);
    if (herr & (ERR_TIMEOUT_ENGINE | ERR_TIMEOUT_TC | ERR_TIMEOUT_APPLY)) {
        bddc_set_last_error("a bounded device wait gave up", __FILE__, __LINE__);
        return BDDC_ETIMEOUT;
    }
    if (herr & ERR_PIVOT) return BDDC_ENUMERIC;
    if (herr & ERR_JACOBI) return BDDC_EGEP;
    if (herr) return BDDC_ECUDA;
    return BDDC_OK;
}

int bddc_setup(const bddc_mesh* mesh, const bddc_coeffs* coeffs, const bddc_partition* part,
               double tol_eig, const bddc_opts* opts, void* stream, bddc_ctx** out) {
    g_last_error.clear();
    if (!out || !part || !coeffs) return BDDC_EINVAL;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        bddc_set_last_error("no CUDA device", __FILE__, __LINE__);
        return BDDC_ECUDA;
    }
    int prc = keep_pool_memory();
    if (prc != BDDC_OK) return prc;
    bddc_ctx* C = new bddc_ctx();
    C->device = dev;
    if (opts) C->o = *opts;
    else bddc_default_opts(&C->o);
    if (tol_eig > 0) C->o.theta_E = tol_eig;
    if (C->o.max_iter <= 0 || !(C->o.rtol >= 0) || C->o.restart < 0 || C->o.precision < BDDC_PREC_FP64 ||
        C->o.precision > BDDC_PREC_BF16) {
        delete C;
        return BDDC_EINVAL;
    }
    C->mixed = C->o.precision != BDDC_PREC_FP64;
    C->st = (cudaStream_t)stream;
    if (C->st == nullptr) {
        // a blocking stream: ordered with the legacy default stream, and capturable
        if (cudaStreamCreate(&C->own) != cudaSuccess) {
            delete C;
            return BDDC_ECUDA;
        }
        C->st = C->own;
    }
    memset(&C->stats, 0, sizeof(C->stats));
    auto t0 = std::chrono::steady_clock::now();
    int rc = setup_body(C, mesh, coeffs, part);
    if (rc != BDDC_OK) {
        cudaStreamSynchronize(C->st);
        bddc_destroy(C);
        return rc;
    }
    C->stats.setup_ms = ms_since(t0);
    C->stats.n_pi = C->nPi;
    C->stats.n_gamma = C->nG;
    C->stats.ndof = C->hm.ndof;
    C->stats.nsub = C->hm.nsd;
    *out = C;
    return BDDC_OK;
}

int bddc_schur_apply(bddc_ctx* C, const double* x, double* y, int nrhs) {
    if (!C || !x || !y || nrhs < 1) return BDDC_EINVAL;
    for (int c = 0; c < nrhs; ++c) {
        if (C->mixed) BDDC_TRY(op_S<float>(C, x + (long long)c * C->nG, y + (long long)c * C->nG, nullptr));
        else BDDC_TRY(op_S<double>(C, x + (long long)c * C->nG, y + (long long)c * C->nG, nullptr));
    }
    BDDC_CUDA_TRY(cudaGetLastError());
    return BDDC_OK;
}

int bddc_apply(bddc_ctx* C, const double* r, double* z, int nrhs) {
    if (!C || !r || !z || nrhs < 1) return BDDC_EINVAL;
    for (int c = 0; c < nrhs; ++c) {
        if (C->mixed) BDDC_TRY(op_M<float>(C, r + (long long)c * C->nG, nullptr));
        else BDDC_TRY(op_M<double>(C, r + (long long)c * C->nG, nullptr));
        BDDC_CUDA_TRY(cudaMemcpyAsync(z + (long long)c * C->nG, C->zc, sizeof(double) * C->nG,
                                      cudaMemcpyDeviceToDevice, C->st));
    }
    return BDDC_OK;
}

int bddc_gmres_solve(bddc_ctx* C, const double* load, double* u, int nrhs, int mem, bddc_stats* stats) {
    if (!C || !u || nrhs < 1) return BDDC_EINVAL;
    if (mem != BDDC_MEM_DEVICE && mem != BDDC_MEM_HOST) return BDDC_EINVAL;
    auto t0 = std::chrono::steady_clock::now();
    const long long ndof = C->hm.ndof;
    int worst = BDDC_OK;
    bddc_stats agg = C->stats;
    agg.iters = 0;
    agg.converged = 1;
    agg.relres = 0;
    agg.relres_global = 0;
    agg.refine_steps = 0;
    BDDC_CUDA_TRY(cudaMemsetAsync(C->kmax, 0, sizeof(double), C->st));
    // several columns: batched solves of up to BDDC_BATCH_MAX columns each
    for (int c0 = 0; nrhs > 1 && c0 < nrhs; c0 += BDDC_BATCH_MAX) {
        const int nb = std::min(BDDC_BATCH_MAX, nrhs - c0);
        BatchWS* W = nullptr;
        BDDC_TRY(batch_ws(C, nb, &W));
        const double* Fd = W->Fin;
        for (int c = 0; c < nb; ++c) {
            const double* src = load ? load + (long long)(c0 + c) * ndof : C->F;
            const cudaMemcpyKind kind = (load && mem == BDDC_MEM_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
            if (load && mem == BDDC_MEM_DEVICE && c == 0) {
                Fd = load + (long long)c0 * ndof;   // device loads are used in place
                break;
            }
            BDDC_CUDA_TRY(cudaMemcpyAsync(W->Fin + c * ndof, src, sizeof(double) * ndof, kind, C->st));
        }
        double* ud = mem == BDDC_MEM_HOST ? W->uglob : u + (long long)c0 * ndof;
        bddc_stats one = C->stats;
        int rc = C->mixed ? solve_batch<float>(C, W, Fd, ud, &one) : solve_batch<double>(C, W, Fd, ud, &one);
        if (rc < 0) return rc;
        if (rc != BDDC_OK) worst = rc;
        if (mem == BDDC_MEM_HOST)
            BDDC_CUDA_TRY(cudaMemcpyAsync(u + (long long)c0 * ndof, W->uglob, sizeof(double) * ndof * nb,
                                          cudaMemcpyDeviceToHost, C->st));
        agg.iters += one.iters;
        agg.refine_steps += one.refine_steps;
        agg.converged = agg.converged && one.converged;
        agg.relres = std::max(agg.relres, one.relres);
        agg.relres_global = std::max(agg.relres_global, one.relres_global);
    }
    for (int c = 0; nrhs == 1 && c < nrhs; ++c) {
        const double* Fd = C->F;
        if (load) {
            if (mem == BDDC_MEM_HOST) {
                BDDC_CUDA_TRY(cudaMemcpyAsync(C->Fin, load + c * ndof, sizeof(double) * ndof, cudaMemcpyHostToDevice, C->st));
                Fd = C->Fin;
            } else {
                Fd = load + c * ndof;
            }
        }
        double* ud = mem == BDDC_MEM_HOST ? C->uglob : u + c * ndof;
        bddc_stats one = C->stats;
        int rc = C->mixed ? solve_one<float>(C, Fd, ud, &one) : solve_one<double>(C, Fd, ud, &one);
        if (rc < 0) return rc;
        if (rc != BDDC_OK) worst = rc;
        if (mem == BDDC_MEM_HOST)
            BDDC_CUDA_TRY(cudaMemcpyAsync(u + c * ndof, C->uglob, sizeof(double) * ndof, cudaMemcpyDeviceToHost, C->st));
        agg.iters += one.iters;
        agg.refine_steps += one.refine_steps;
        agg.converged = agg.converged && one.converged;
        agg.relres = std::max(agg.relres, one.relres);
        agg.relres_global = std::max(agg.relres_global, one.relres_global);
    }
    int herr = 0;
    double hk = 0.0;
    BDDC_CUDA_TRY(cudaMemcpyAsync(&herr, C->err, sizeof(int), cudaMemcpyDeviceToHost, C->st));
    BDDC_CUDA_TRY(cudaMemcpyAsync(&hk, C->kmax, sizeof(double), cudaMemcpyDeviceToHost, C->st));
    BDDC_CUDA_TRY(cudaStreamSynchronize(C->st));
    C->stats.kappa_est = C->o.cond_est ? hk : 0.0;
    agg.solve_ms = ms_since(t0);
    if (herr & ERR_TIMEOUT_APPLY) {
        bddc_set_last_error("a bounded wait of the preconditioner's task kernel gave up", __FILE__, __LINE__);
        return BDDC_ETIMEOUT;
    }
    C->stats.iters = agg.iters;
    C->stats.refine_steps = agg.refine_steps;
    C->stats.converged = agg.converged;
    C->stats.relres = agg.relres;
    C->stats.relres_global = agg.relres_global;
    C->stats.solve_ms = agg.solve_ms;
    if (stats) *stats = C->stats;
    return worst;
}

int bddc_get_stats(const bddc_ctx* C, bddc_stats* s) {
    if (!C || !s) return BDDC_EINVAL;
    *s = C->stats;
    return BDDC_OK;
}

int bddc_get_numbering(const bddc_ctx* C, int* gamma_dofs) {
    if (!C || !gamma_dofs) return BDDC_EINVAL;
    memcpy(gamma_dofs, C->hm.gamma.data(), sizeof(int) * C->hm.gamma.size());
    return BDDC_OK;
}

int bddc_get_schur(const bddc_ctx* C, int s, double* out, int* n_b) {
    if (!C || s < 0 || s >= C->hm.nsd || !n_b) return BDDC_EINVAL;
    const int nB = C->hm.sub[s].nB;
    *n_b = nB;
    if (!out) return BDDC_OK;
    BDDC_CUDA_TRY(cudaStreamSynchronize(C->st));
    BDDC_CUDA_TRY(cudaMemcpy2D(out, sizeof(double) * nB, C->S64 + C->soff[s], sizeof(double) * C->sld[s],
                               sizeof(double) * nB, nB, cudaMemcpyDeviceToHost));
    return BDDC_OK;
}

int bddc_get_entity_count(const bddc_ctx* C, int kind) {
    if (!C || kind < 0 || kind > 2) return BDDC_EINVAL;
    return (int)C->hm.by_kind[kind].size();
}

int bddc_get_entity(const bddc_ctx* C, int kind, int index, int* subs, int* dofs, int* n, int* k,
                    double* Q, double* lambda, int* n_eig) {
    if (!C || kind < 0 || kind > 2 || index < 0 || index >= (int)C->hm.by_kind[kind].size()) return BDDC_EINVAL;
    const int e = C->hm.by_kind[kind][index];
    const Entity& E = C->hm.ent[e];
    const int nn = (int)E.dofs.size();
    if (n) *n = nn;
    if (k) *k = E.k;
    if (subs)
        for (int a = 0; a < 8; ++a) subs[a] = a < (int)E.subs.size() ? E.subs[a] : -1;
    if (dofs) memcpy(dofs, E.dofs.data(), sizeof(int) * nn);
    if (n_eig) *n_eig = C->neig[e];
    BDDC_CUDA_TRY(cudaStreamSynchronize(C->st));
    if (Q && kind > 0) {
        // device Q is row-major (row = entity dof, column = basis vector); return column-major n x k
        std::vector<double> h((size_t)nn * nn);
        BDDC_CUDA_TRY(cudaMemcpy(h.data(), C->Q[e], sizeof(double) * nn * nn, cudaMemcpyDeviceToHost));
        for (int l = 0; l < E.k; ++l)
            for (int a = 0; a < nn; ++a) Q[(size_t)l * nn + a] = h[(size_t)a * nn + l];
    } else if (Q && kind == 0) {
        Q[0] = 1.0;
    }
    if (lambda && kind > 0 && C->neig[e] > 0)
        BDDC_CUDA_TRY(cudaMemcpy(lambda, C->lam[e], sizeof(double) * C->neig[e], cudaMemcpyDeviceToHost));
    return BDDC_OK;
}

unsigned long long bddc_kernel_launches(void) { return g_launches.load(); }

int bddc_tc_selftest(const float* A, const float* B, float* C, int nr, int nc, int K) {
    if (!A || !B || !C || nr < 1 || nc < 1 || nr > 128 || nc > 128 || K < 1 || K > 32) return BDDC_EINVAL;
    cudaStream_t st;
    BDDC_CUDA_TRY(cudaStreamCreate(&st));
    float *dA = nullptr, *dB = nullptr, *dC = nullptr;
    int* derr = nullptr;
    int rc = BDDC_OK;
    int herr = 0;
    if (cudaMallocAsync((void**)&dA, 128 * 32 * sizeof(float), st) != cudaSuccess ||
        cudaMallocAsync((void**)&dB, 32 * 128 * sizeof(float), st) != cudaSuccess ||
        cudaMallocAsync((void**)&dC, 128 * 128 * sizeof(float), st) != cudaSuccess ||
        cudaMallocAsync((void**)&derr, sizeof(int), st) != cudaSuccess) {
        rc = BDDC_ENOMEM;
    } else {
        cudaMemcpyAsync(dA, A, 128 * 32 * sizeof(float), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dB, B, 32 * 128 * sizeof(float), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dC, C, 128 * 128 * sizeof(float), cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(derr, 0, sizeof(int), st);
        rc = tc_selftest_run(dA, dB, dC, nr, nc, K, derr, st);
        cudaMemcpyAsync(C, dC, 128 * 128 * sizeof(float), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
    }
    cudaFreeAsync(dA, st);
    cudaFreeAsync(dB, st);
    cudaFreeAsync(dC, st);
    cudaFreeAsync(derr, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        bddc_set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
        return BDDC_ECUDA;
    }
    if (rc == BDDC_OK && herr) rc = BDDC_ETIMEOUT;
    return rc;
}

int bddc_wait_selftest(int limit) {
    if (limit < 1 || limit > (1 << 24)) return BDDC_EINVAL;
    int to = 0;
    BDDC_TRY(wait_selftest_run(limit, &to));
    return to ? BDDC_ETIMEOUT : BDDC_OK;
}

int bddc_kernel_timer(int kind) {
    if (kind < KT_NONE || kind > KT_LAST) return BDDC_EINVAL;
    std::lock_guard<std::mutex> lk(g_kt_mu);
    for (auto& pr : g_kt.ev) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    g_kt = KTimer();
    g_kt.kind = kind;
    return BDDC_OK;
}

int bddc_kernel_timer_read(double* total_ms, long long* launches, double* flops, double* bytes) {
    std::lock_guard<std::mutex> lk(g_kt_mu);
    double tot = 0.0;
    for (auto& pr : g_kt.ev) {
        BDDC_CUDA_TRY(cudaEventSynchronize(pr.second));
        float ms = 0.f;
        BDDC_CUDA_TRY(cudaEventElapsedTime(&ms, pr.first, pr.second));
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = g_kt.launches;
    if (flops) *flops = g_kt.flops;
    if (bytes) *bytes = g_kt.bytes;
    return BDDC_OK;
}

int bddc_get_edge_features(const bddc_ctx* C, float* feats, int* counts) {
    if (!C) return BDDC_EINVAL;
    const std::vector<int>& edges = C->hm.by_kind[1];
    BDDC_CUDA_TRY(cudaStreamSynchronize(C->st));
    if (feats && !edges.empty())
        BDDC_CUDA_TRY(cudaMemcpy(feats, C->d_feat, sizeof(float) * edges.size() * BDDC_MLP_FEATURES,
                                 cudaMemcpyDeviceToHost));
    if (counts)
        for (size_t ei = 0; ei < edges.size(); ++ei) counts[ei] = C->edge_skipped[ei] ? -1 : C->kk[edges[ei]];
    return BDDC_OK;
}

}  // extern "C"
