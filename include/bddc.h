/*
 * bddc.h -- C ABI of libbddc: adaptive BDDC-preconditioned GMRES for the
 * stabilised advection-diffusion system of arXiv 2501.01676 on one GB300.
 *
 * The model problem (Sect. 2) is -div(nu grad u) + beta.grad u + c u = f on a
 * box with u = 0 on its boundary, discretised by trilinear hexahedra with the
 * stabilised forms a = b + z and load g of Sect. 2.  The box is cut into a
 * tensor partition of subdomains (Sect. 3); the library solves the interface
 * Schur system (eq. Schur-complex-sys) with GMRES preconditioned by
 * M^-1 = R~^T D~ S~^-1 D~^T R~ (Sect. 3) whose coarse space holds vertex
 * constraints, adaptive face constraints (face GEP, eq. equ-4-8) and adaptive
 * edge constraints from the edge GEP on prior-selected primal constraints
 * (eq. equ-5-21, constraints eq. equ-5-22), then recovers the interior
 * unknowns.
 *
 * Conventions shared by every entry point
 *   - Return value: 0 (BDDC_OK) on success, BDDC_NOT_CONVERGED (positive, the
 *     result is still written), or a negative error code.  Nothing aborts or
 *     traps; every device wait and iteration is bounded.
 *   - Numbering: elements e = ex + Ex*(ey + Ey*ez); nodes
 *     n = ix + (Ex+1)*(iy + (Ey+1)*iz); free (non-Dirichlet) dofs
 *     d = (ix-1) + (Ex-1)*((iy-1) + (Ey-1)*(iz-1)).  Interface vectors
 *     (length n_gamma) list the interface dofs in ascending dof id.
 *   - Calls are ordered on the CUDA stream given at setup.  All device memory
 *     the solver needs is owned by the context; the caller owns its own
 *     buffers.  One context must not be used by two host threads at once.
 *   - There is no CPU fallback: without a usable GPU every call fails with
 *     BDDC_ECUDA.
 */
#ifndef BDDC_H
#define BDDC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BDDC_OK              0
#define BDDC_NOT_CONVERGED   1
#define BDDC_EINVAL        (-1)   /* bad argument                                  */
#define BDDC_ENOMEM        (-2)   /* device or host allocation failed              */
#define BDDC_ECUDA         (-3)   /* CUDA runtime error / no GPU                   */
#define BDDC_EGEP          (-4)   /* eigen iteration cap reached in a GEP          */
#define BDDC_ETIMEOUT      (-5)   /* bounded device wait gave up                   */
#define BDDC_ENUMERIC      (-6)   /* zero or non-finite pivot in a factorisation   */

#define BDDC_MEM_DEVICE 0
#define BDDC_MEM_HOST   1

#define BDDC_PREC_FP64  0   /* every factor and operator in FP64                  */
#define BDDC_PREC_MIXED 1   /* FP32 factors/operators + FP64 iterative refinement  */
#define BDDC_PREC_BF16  2   /* as MIXED, the trailing updates of the FP32 dense
                               eliminations on the tensor cores with BF16 operands
                               (FP32 accumulation); the refinement restores FP64
                               accuracy of the solution, at more iterations        */

#define BDDC_EDGE_NONE 0
#define BDDC_EDGE_NEW  1    /* edge GEP on prior-selected primal constraints      */
#define BDDC_EDGE_OLD  2    /* conventional edge GEP (Sect. 3, eq. equ-4-8-E):
                               B_E v = lambda B~_E v with B_E = sum_i sum_{k != i}
                               D^(k)T B_E^(i) D^(k) and B~_E the parallel sum of the
                               Schur complements of B^(k) onto E; the comparison
                               method of the paper's ABDDC-OLD columns            */

#define BDDC_ELEM_Q1   0    /* trilinear hexahedra (bricks)                        */
#define BDDC_ELEM_P1   1    /* linear tetrahedra: each brick split into the six
                               tetrahedra around its main diagonal (Sect. 4)       */

/* Box [lo, hi]^3; the unit cube when both are zero. */
typedef struct { double lo[3], hi[3]; } bddc_mesh;

/* Tensor partition: direction d is cut into nsub[d] slabs, slab s holding
 * elems_per_slab[d][s] >= 1 elements (host pointers, copied). Element
 * spacing is uniform per direction. */
typedef struct { int nsub[3]; const int* elems_per_slab[3]; } bddc_partition;

/* Coefficients (Sect. 2).  All arrays are FP64, in host or device memory as
 * `mem` says, and are copied at setup; bddc_setup rejects (BDDC_EINVAL) a
 * nu <= 0 or non-finite, and non-finite beta, f, div(beta), c or beta_const.
 *   nu_elem   [nelem]      viscosity per element, > 0
 *   beta_node [3*nnodes]   velocity at the nodes (x,y,z interleaved) or NULL,
 *                          in which case beta_const is used everywhere
 *   f_node    [nnodes]     source at the nodes, or NULL (f = 0)
 *   divb_node [nnodes]     div(beta) at the nodes, or NULL (0)
 *   g_node    [nnodes]     Dirichlet values at the nodes (only the boundary
 *                          nodes' are used), or NULL (homogeneous); they enter
 *                          the loads of the neighbouring free nodes
 * beta, f and div(beta) are interpolated trilinearly inside each element (Q1),
 * or linearly inside each tetrahedron (element BDDC_ELEM_P1). */
typedef struct {
    const double* nu_elem;
    const double* beta_node;
    double beta_const[3];
    double c;
    const double* f_node;
    const double* divb_node;
    int mem;
    const double* g_node;
} bddc_coeffs;

typedef struct {
    double theta_E;        /* edge threshold Theta_E (Sect. 4: 10)                 */
    double theta_F;        /* face threshold; <= 0: 1 + ln(H/h) per face (Sect. 4) */
    double tau;            /* stabilisation constant (Sect. 2: 0.7)               */
    int precision;         /* BDDC_PREC_FP64, BDDC_PREC_MIXED or BDDC_PREC_BF16    */
    int restart;           /* GMRES restart length, 0: no restart                 */
    int max_iter;          /* iteration cap (Sect. 4: 300)                        */
    double rtol;           /* relative residual target (Sect. 4: 1e-8)            */
    int edge_gep;          /* BDDC_EDGE_NONE, BDDC_EDGE_NEW or BDDC_EDGE_OLD       */
    int face_gep;          /* 1: adaptive face constraints, 0: none               */
    int all_primal;        /* 1: every interface dof primal (exact solver check)   */
    double inner_rtol;     /* MIXED: inner GMRES tolerance per refinement step     */
    int max_refine;        /* MIXED: refinement step cap                           */
    double learned_skip_p; /* < 0: no learned skip; else skip an edge GEP when the
                              network gives P(no constraint) >= this               */
    const float* mlp_params; /* host, BDDC_MLP_PARAMS floats (layout below), copied at
                                setup; NULL: no learned skip                        */
    int tensor_cores;      /* MIXED: 1 = trailing updates of the FP32 eliminations on
                              the tensor cores (tcgen05, split TF32), 0 = FP32 CUDA
                              cores; ignored by the FP64 and BF16 paths             */
    int coarse_elim;       /* 1: invert S_Pi explicitly by the elimination engine
                              always (dense, 4.7 n_Pi^3 flops); 0: small S_Pi
                              (n_Pi <= 128) by FP32 Gauss-Jordan + FP64 Newton-
                              Schulz when its residual check passes, otherwise the
                              nested-dissection sparse LU of S_Pi (coarse_path 2)   */
    int apply_launch;      /* 0: M^-1 r as one persistent launch (local part, coarse
                              restriction, coarse solve and prolongation as work
                              items with completion counters); 1: one launch per
                              phase (the reference path of the tests)              */
    int cond_est;          /* 1: estimate the condition number of the preconditioned
                              operator from every GMRES cycle's Hessenberg
                              (stats.kappa_est); 0: skip                           */
    int element;           /* BDDC_ELEM_Q1: trilinear bricks; BDDC_ELEM_P1: linear
                              elements on the six tetrahedra of each brick around
                              its main diagonal (Sect. 4, Example 4.1)            */
    int local_nd;          /* 0: each subdomain's interior eliminated as one dense
                              block; 1: one level of nested dissection: the
                              subdomain box split into up to 2 x 2 x 2 child boxes
                              (every slab of 2 or more elements halved), the
                              children's interiors eliminated first (dense, in a
                              batch), their Schur complements summed into the
                              subdomain's matrix over its separator planes and
                              interface, then the separators eliminated; S^(i) is
                              the same operator (Sect. 3), with ~1/12 of the
                              flops and ~1/5 of the memory at H/h = 16         */
} bddc_opts;

typedef struct {
    int iters;               /* GMRES iterations (all refinement steps)           */
    int refine_steps;        /* MIXED: outer steps, FP64: 1                        */
    int converged;
    double relres;           /* FP64: ||g - S u_G|| / ||g|| on the Schur system;
                                MIXED: ||F - A u|| / ||F|| of the global system   */
    double relres_global;    /* ||F - A u|| / ||F|| in FP64 (both modes)           */
    int pnumF, pnumE;        /* face / edge primal unknowns (Sect. 4 tables)       */
    int n_pi;                /* coarse size: vertices + pnumF + pnumE             */
    int n_gamma, ndof, nsub;
    int edges_skipped;       /* edge GEPs skipped by the learned predictor         */
    double setup_ms, solve_ms;
    double t_assemble_ms, t_factor_ms, t_face_ms, t_edge_ms, t_coarse_ms;
    int jacobi_sweeps_max;   /* most sweeps any GEP eigen-decomposition needed   */
    double t_mesh_ms;        /* host numbering / entity lists / coefficient staging */
    double t_basis_ms;       /* change of basis + extended elimination (part of
                                t_coarse_ms)                                      */
    int coarse_path;         /* coarse problem by 0: explicit FP64 inverse from the
                                elimination of [[S_Pi, -I], [I, 0]], 1: FP32 Gauss-
                                Jordan + FP64 Newton-Schulz (n_Pi <= 128), 2: FP64
                                sparse LU by nested dissection of the subdomain grid
                                (multifrontal; the apply runs its forward and
                                backward sweeps)                                   */
    int coarse_fronts;       /* path 2: dense fronts (separators) of the tree       */
    int coarse_levels;       /* path 2: height of the tree (sweep launches per side) */
    double coarse_factor_gflop; /* path 2: flops of the front eliminations / 1e9    */
    double kappa_est;        /* largest sigma_max / sigma_min of the Hessenberg over
                                the last solve's GMRES cycles of at most 128
                                iterations: an estimate of the condition number
                                of S M^-1 (0: not computed)                       */
    int gemv_rows;           /* rows per work item of the S x kernel, picked at
                                setup by timing 32, 64, 128 and 256 on the
                                context's own operators (the first setup of a
                                shape class in the process measures; later ones
                                reuse the choice)                                  */
    double gemv_tune_us;     /* the chosen list's time per product when this setup
                                measured it (0: the choice was reused)             */
    int nd_children;         /* local_nd = 1: child boxes over all subdomains (0: off) */
    double factor_gflop;     /* flops of the subdomain eliminations / 1e9 (children
                                and separators with local_nd = 1)                 */
} bddc_stats;

typedef struct bddc_ctx bddc_ctx;

/* Fill `o` with the defaults of Sect. 4: Theta_E = 10, Theta_F = 1 + ln(H/h),
 * tau = 0.7, FP64, no restart, 300 iterations, rtol 1e-8, new edge GEP,
 * face GEP on, inner_rtol 1e-6, max_refine 8, no learned skip, tensor-core
 * trailing updates in the MIXED path (tensor_cores 1), coarse_elim 0,
 * apply_launch 0, cond_est 1, element BDDC_ELEM_Q1, local_nd 0. */
void bddc_default_opts(bddc_opts* o);

/* Setup (call stack: assembly, batched Dirichlet factorisation + Schur
 * complements S^(i) (Sect. 3), deluxe scaling, face GEPs, new edge GEPs,
 * constrained local solvers, coarse matrix and its FP64 inverse).
 * tol_eig > 0 overrides opts->theta_E.  stream: a cudaStream_t or NULL for
 * the legacy default stream.  On success *out owns all device memory.
 * Subdomains with more than 8192 interior dofs (a box of more than 21
 * elements in every direction) and faces of more than 256 dofs (more than
 * 17 x 17 elements) are rejected with BDDC_EINVAL. */
int bddc_setup(const bddc_mesh* mesh, const bddc_coeffs* coeffs,
               const bddc_partition* part, double tol_eig,
               const bddc_opts* opts, void* stream, bddc_ctx** out);

/* z = M^-1 r on the interface (Sect. 3, M_BDDC^-1).  r, z: device FP64,
 * n_gamma x nrhs column blocks (column j at offset j*n_gamma). */
int bddc_apply(bddc_ctx* ctx, const double* r_dev, double* z_dev, int nrhs);

/* z = M^-1 r exactly as bddc_apply, for callers that cannot allocate device
 * memory where they apply the preconditioner (a host framework that owns all
 * device memory and forbids libraries from allocating behind its back, or
 * code where an allocation call could synchronise the device).  The paper has
 * no counterpart; it is a property of this library only.  The context's
 * device must be the current device (BDDC_EINVAL otherwise).  The call
 * allocates nothing: its work vectors
 * (n_gamma + 2 * n_pi doubles) live in one file-scope device array of
 * 2^20 doubles (8 MiB) that every GPU loading the library holds until the
 * process exits; larger problems are rejected with BDDC_EINVAL.  The first
 * call on a device looks up the array's device address, so make that first
 * call before any stream capture.  All calls share the array and it keeps
 * the last call's contents (the kernels clear what must start at zero);
 * calls that overlap on the GPU race on it.  r, z: device FP64 as in
 * bddc_apply; the work runs on the context's stream. */
int bddc_apply_static(bddc_ctx* ctx, const double* r_dev, double* z_dev, int nrhs);

/* y = S x = sum_i R_i^T S^(i) R_i x on the interface (eq. Schur-complex-sys).
 * Device FP64, n_gamma x nrhs. */
int bddc_schur_apply(bddc_ctx* ctx, const double* x_dev, double* y_dev, int nrhs);

/* Full solve: condense the load onto the interface, right-preconditioned
 * GMRES (Sect. 4 stopping rule), recover the interior unknowns.
 * load: assembled nodal loads on the free dofs (ndof x nrhs) or NULL to use
 * the load of the coefficients (Sect. 2, g(v)); u: ndof x nrhs output.
 * mem: BDDC_MEM_DEVICE or BDDC_MEM_HOST for both pointers (host pointers are
 * staged through device buffers inside the call).  stats may be NULL. */
int bddc_gmres_solve(bddc_ctx* ctx, const double* load, double* u, int nrhs,
                     int mem, bddc_stats* stats);

int  bddc_get_stats(const bddc_ctx* ctx, bddc_stats* stats);
void bddc_destroy(bddc_ctx* ctx);
const char* bddc_strerror(int code);
/* The message of the last failure recorded on the calling thread (what was
 * rejected or which CUDA call failed, with the source location), or "" when
 * none was recorded since the thread's last bddc_setup.  The string is owned by
 * the library and valid until the thread's next call. */
const char* bddc_last_error(void);

/* ---- introspection (tests and benchmarks; host output buffers) ---------- */

/* Process-wide number of kernels the library has launched so far (a CUDA
 * graph replay counts its kernel nodes).  Host-only, never fails. */
unsigned long long bddc_kernel_launches(void);

/* Self-test of the tensor-core trailing update (no counterpart in the paper):
 * C (128 x 128, row-major, host) -= A (128 x 32, row-major) * B (32 x 128,
 * row-major) restricted to rows < nr, columns < nc and the first K (<= 32)
 * columns of A / rows of B, computed by one CTA with tcgen05.mma (split TF32:
 * hi*hi + hi*lo + lo*hi, FP32 accumulation in tensor memory).  Host buffers;
 * BDDC_ETIMEOUT if the bounded wait for the MMAs gave up. */
int bddc_tc_selftest(const float* A, const float* B, float* C, int nr, int nc, int K);

/* Self-test of the bounded device waits (no counterpart in the paper): one
 * CTA runs the wait that the one-launch preconditioner apply uses on its
 * completion counters, on a counter that nothing increments, with `limit`
 * polls (1 .. 2^24, about 0.1 us each).  The wait must give up by itself:
 * the call returns BDDC_ETIMEOUT (the expected outcome) with the device
 * still usable, BDDC_OK if the wait ended otherwise, BDDC_EINVAL for a limit
 * out of range.  Synchronous; allocates and frees a few bytes. */
int bddc_wait_selftest(int limit);

/* Kernel timer for roofline reporting: after bddc_kernel_timer(kind) every
 * launch of that kernel class (1 engine trailing update, 2 engine panel,
 * 3 apply GEMV, 4 face GEP, 5 edge GEP, 6 element assembly, 7 change of basis,
 * 8 interior condense / recover solves, 9 coarse inverse, 10 the engine's
 * persistent task kernel, 11 the one-launch preconditioner apply (1 and 2
 * switch the engine to per-panel launches);
 * 0 off) is bracketed by CUDA events on
 * its stream (launches captured into graphs are not).  _read synchronises on
 * the recorded events and returns their summed duration, the number of
 * launches and, where the library knows them, the algorithmic flops and
 * bytes of those launches.  Process-wide; not thread-safe with concurrent
 * solves. */
int bddc_kernel_timer(int kind);
int bddc_kernel_timer_read(double* total_ms, long long* launches, double* flops, double* bytes);

/* Global dof id of each interface position (n_gamma ints). */
int bddc_get_numbering(const bddc_ctx* ctx, int* gamma_dofs);

/* S^(s) (n_B x n_B, row-major, local interface order = ascending dof id) in
 * FP64 (converted when MIXED).  Pass out = NULL to query *n_b only. */
int bddc_get_schur(const bddc_ctx* ctx, int s, double* out, int* n_b);

/* Entities: kind 0 vertex, 1 edge, 2 face; index within its kind in the
 * library's order.  Writes the sorted subdomain set (subs[8], -1 padded),
 * the entity's dof ids (dofs[n]), its primal count k and, for faces and
 * edges, the orthonormal constraint basis Q (n x k, column-major) and the
 * GEP eigenvalues lambda (ascending sigma order reversed: largest first,
 * +inf for infinite; up to n values for faces and conventional edge GEPs,
 * (|n(E)| - 1) n for the new edge GEP; count in *n_eig).  NULL outputs are
 * skipped.  *n returns the entity size. */
int bddc_get_entity_count(const bddc_ctx* ctx, int kind);
int bddc_get_entity(const bddc_ctx* ctx, int kind, int index, int* subs,
                    int* dofs, int* n, int* k, double* Q, double* lambda,
                    int* n_eig);

/* ---- learned edge-GEP skip ---------------------------------------------
 * Not in the paper.  A small FP32 network predicts from local coefficient
 * features how many constraints the edge GEP (eq. equ-5-21 and the selection
 * below it) will select on an edge; at setup, edges whose predicted
 * probability of selecting none is >= learned_skip_p skip the GEP (no edge
 * constraint; deluxe scaling is still computed); every other edge runs the
 * full GEP.  Features of an edge (a line of n_E interior dofs along axis a;
 * "touching" elements are the 4 (n_E + 1) elements holding the segment):
 *   0-2 min / max / mean log10 nu over touching elements,
 *   3   max - min over n(E) of the per-subdomain mean log10 nu,
 *   4-6 mean |beta_a|, max |beta_a|, mean |beta| over the edge nodes,
 *   7   edge length (n_E + 1) h_a, 8 (H/h)/10, 9 log10(h_a * f6 / (2 * 10^f2)),
 *   10  log10(Theta_E) (the GEP's selection threshold).
 * Network: 11 -> 64 -> 64 -> 64 (ReLU) -> 8 logits (class = min(k_E, 7)),
 * loss = mean softmax cross-entropy.  Parameters are one FP32 array:
 * W1[11][64], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[64][8],
 * b4[8] (row-major, input index first). */

#define BDDC_MLP_FEATURES 11
#define BDDC_MLP_HIDDEN   64
#define BDDC_MLP_CLASSES  8
#define BDDC_MLP_PARAMS   9608

/* Edge features of the context (n_edges x BDDC_MLP_FEATURES, FP32 host) and
 * the edge GEP's constraint counts (n_edges ints, -1 where it was skipped),
 * edges in the order of bddc_get_entity(kind 1). */
int bddc_get_edge_features(const bddc_ctx* ctx, float* feats, int* counts);

/* Class probabilities (rows x 8, device) of feature rows X (rows x 10,
 * device) for the parameters params (host).  Synchronous on `stream`. */
int bddc_mlp_forward(const float* params, const float* X_dev, int rows, float* probs_dev, void* stream);

/* Mean cross-entropy over the rows (labels y_dev in 0..7) and its gradient
 * (BDDC_MLP_PARAMS floats, host) by the library's backward kernels. */
int bddc_mlp_loss_grad(const float* params, const float* X_dev, const int* y_dev, int rows,
                       float* grad, float* loss, void* stream);

/* Full-batch Adam training on the GPU (beta1 0.9, beta2 0.999, eps 1e-8):
 * params (host) are read and overwritten; loss (host, epochs + 1 values,
 * may be NULL) receives the loss before every step and after the last. */
int bddc_mlp_train(float* params, const float* X_dev, const int* y_dev, int rows, int epochs,
                   float lr, float* loss, void* stream);

#ifdef __cplusplus
}
#endif
#endif
