/*
 * ieti.h -- C ABI of the GB300 tree-cotree IETI-DP eddy-current solver.
 *
 * Method: Mally, Vazquez, Schoeps, "Tree-Cotree-Based IETI-DP for Eddy Current
 * Problems in Time-Domain".  The library advances the implicit-Euler scheme of
 * Eq. (11),  [W, dt B^T; dt B, 0][a; m] = [M a^l + dt j^{l+1}; 0],  W = M + dt K,
 * for the A*-formulation (Eq. (5)) discretised with spline edge elements on a
 * structured grid of conforming patches (Sec. 2.2), gauged by the hierarchical
 * tree-cotree splitting of Sec. 3 (e / p / r DOFs), and solves each step by the
 * dual-primal method of Sec. 3 (two Schur complements, PCG on the interface
 * problem with a Dirichlet preconditioner, Sec. 4) on one CUDA device.
 *
 * Conventions (all entry points):
 *  - Return 0 on success or a negative IETI_ERR_* code; ieti_last_error() gives
 *    a message.  Nothing is thrown across the ABI; no call aborts the process.
 *  - Input arrays are owned by the caller and copied during the call.  Output
 *    buffers are allocated by the caller.
 *  - "host or device" arguments: IETI_MEM_HOST means a host pointer (pageable or
 *    pinned), IETI_MEM_DEVICE a pointer into memory of the context's device.
 *  - Device work runs on options.cuda_stream (0 = legacy default stream).  A call
 *    returns after its device work has completed.
 *  - A context is not thread-safe; distinct contexts are independent.
 *
 * Global DOF numbering (the control-mesh lattice of all patches, Sec. 2.2/3):
 *  slab a in direction d has n_el[d][a] elements and degree[d][a]; its lattice
 *  offset is off_d(a) = sum_{b<a} (n_el[d][b] + degree[d][b] - 1); N_d is the total
 *  number of lattice points in direction d.  Edge ids: direction-0 edges first,
 *  id = I + (N0-1)*(J + N1*K); then direction 1 from E0 = (N0-1)*N1*N2,
 *  id = E0 + I + N0*(J + (N1-1)*K); then direction 2 from E0 + E1 with
 *  E1 = N0*(N1-1)*N2, id = E0 + E1 + I + N0*(J + N1*K).  Vectors of length
 *  ieti_num_dofs() use this numbering; eliminated DOFs (Dirichlet and gauge) hold 0.
 */
#ifndef IETI_H
#define IETI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IETI_OK 0
#define IETI_ERR_INVALID_ARG -1     /* bad sizes, pointers, knot vectors, options */
#define IETI_ERR_NONCONFORMING -2   /* knot vectors / degrees that do not match on a shared face */
#define IETI_ERR_NOT_SPD -3         /* a local or coarse block is not positive definite (patch id in message) */
#define IETI_ERR_CG_NOT_CONVERGED -4 /* PCG hit cg_max_it (or outer refinement max_sweeps) */
#define IETI_ERR_CUDA -5            /* a CUDA runtime error (message has the text) */
#define IETI_ERR_OOM -6             /* device or host allocation failed */
#define IETI_ERR_NO_DEVICE -7       /* compute requested on a host-only context */
#define IETI_ERR_TOO_LARGE -8       /* size beyond a documented fixed maximum */
#define IETI_ERR_TIMEOUT -9         /* a bounded device wait (grid barrier of the dual-primal kernel) ran out;
                                       the launch ended cleanly and the context stays usable */

#define IETI_MEM_HOST 0
#define IETI_MEM_DEVICE 1

/* Precision of the factor-derived operators (Sec. 3 Schur complements). */
#define IETI_PREC_FP64 0   /* everything FP64 */
#define IETI_PREC_MIXED 1  /* FP32 local operators, FP64 CG / coarse / residuals, outer FP64 refinement */

/* Arithmetic of the setup factorizations of the patch blocks (the partial Cholesky
 * behind both Schur complements of Sec. 3) in the MIXED precision mode; the FP64
 * mode always factors in FP64.  The coarse block is always factored in FP64.  The
 * outer FP64 refinement of every step recovers the accuracy of the reduced factors. */
#define IETI_FACTOR_FP64 0    /* FP64 on the FP64 pipe, operators rounded to FP32 afterwards */
#define IETI_FACTOR_FP32 1    /* FP32 on the SIMT pipe */
#define IETI_FACTOR_TF32X3 2  /* FP32 panels, trailing updates on the tensor cores as three TF32 products
                                 (hi*hi + hi*lo + lo*hi, FP32 accumulation): FP32-class accuracy */
#define IETI_FACTOR_TF32 3    /* as TF32X3 with one TF32 product (ablation: 11-bit operands) */
#define IETI_FACTOR_BF16X3 4  /* as TF32X3 with BF16 hi and lo planes (kind::f16 MMAs, FP32 accumulation):
                                 about 16 significant bits per operand (ablation) */
#define IETI_FACTOR_BF16 5    /* one BF16 product (ablation: 8-bit operands) */

/* Solve of the primal coarse problem S_c q = c (Sec. 3, the second Schur complement) in
 * every PCG iteration.  DENSE: S_c^{-1} is formed at setup (FP64 partial Cholesky of
 * [[S_c, I], [I, 0]]) and applied as dense rows (8 nc^2 bytes per solve).  ND: S_c is
 * factored along a nested dissection of the patch grid (multifrontal, FP64) and solved by
 * one forward and one backward sweep over the tree levels (bytes ~ the factor's entries).
 * AUTO: ND once the dense inverse exceeds 64 MB, for linear problems with pcg_mode 0. */
#define IETI_COARSE_AUTO 0
#define IETI_COARSE_DENSE 1
#define IETI_COARSE_ND 2

/* Dirichlet preconditioner variants (Sec. 4 uses the unscaled one; Sec. 5 asks for scaling). */
#define IETI_PRECOND_NONE 0
#define IETI_PRECOND_DIRICHLET 1       /* unscaled: B_D = B (the paper's experiments) */
#define IETI_PRECOND_DIRICHLET_MULT 2  /* multiplicity scaling delta = 1/|N_x| */
#define IETI_PRECOND_DIRICHLET_STIFF 3 /* stiffness scaling with the local diagonal of W */

/* Problem: unit cube split into a structured P0 x P1 x P2 grid of patches, patch
 * s = a + P0*(b + P1*c) (Sec. 2.2, conforming spline spaces on each patch). */
typedef struct {
  int32_t n_patches[3];         /* P0, P1, P2 >= 1 */
  const int32_t *n_el[3];       /* [d][slab]: elements per slab, >= 1 */
  const int32_t *degree[3];     /* [d][slab]: H^1 degree p >= 1 (edge space: p-1 along the edge) */
  const double *knots[3];       /* [d]: concatenated open knot vectors on [0,1] of each slab,
                                   n_el + 2p + 1 values each, p+1 repeated ends, simple interior knots */
  const double *ctrl_pts;       /* concatenated geometry control nets, per patch (n2,n1,n0,3), i fastest,
                                   n_d = n_el + p; the map uses the degree-p splines of the same knots */
  const double *sigma_el;       /* per element, patch-major, (e2,e1,e0) e0 fastest; >= 0 */
  const double *nu_el;          /* per element, same layout; > 0 */
  double dt;                    /* implicit-Euler step (Eq. (11)), > 0 */
  int32_t primal_mode;          /* 0: tree DOFs on Gamma + cotree wirebasket edges of Omega_I (Sec. 3) */
  const double *reluctivity;    /* NULL: linear (nu_el everywhere).  Else 4 values nu0, k1, k2, k3 of the law
                                   nu(|B|) = nu0 (k1 exp(k2 |B|^2) + k3), which replaces nu_el in the
                                   conducting elements (sigma_el > 0); nu0 > 0, k1, k2, k3 >= 0, k1 + k3 > 0.
                                   The nonlinear material the paper names as an extension (Sec. 2): every
                                   ieti_step then runs Newton's method (see ieti_options.refactor). */
} ieti_problem;

typedef struct {
  int32_t device;        /* CUDA device ordinal; -1 = host-only context (setup queries, no compute) */
  int32_t precision;     /* IETI_PREC_* */
  int32_t precond;       /* IETI_PRECOND_* */
  double cg_tol;         /* PCG stop: ||r_k|| <= cg_tol * ||d||, lambda_0 = 0 */
  int32_t cg_max_it;
  double outer_tol;      /* refinement stop: ||f - W a|| <= outer_tol * ||f|| (FP64 residual) */
  int32_t max_sweeps;    /* refinement sweeps per step (FP64 mode: 1 suffices) */
  int32_t pcg_mode;      /* 0: PCG as one persistent cooperative kernel (default); 1: one launch per phase */
  int32_t host_threads;  /* threads for the host setup (0 = all cores) */
  void *cuda_stream;     /* cudaStream_t (0 = legacy default stream) */
  int32_t profile;       /* 1: time every launch of the operator kernels with CUDA events (ieti_kernel_stats) */
  int32_t l2_persist;    /* L2 use by the per-iteration operators (H, Psi, S_bb, coarse), re-read every
                            PCG iteration.  0: plain streaming.  1: a persisting L2 carve-out (access-policy
                            window) during a step.  2: eviction-priority hints on their TMA loads: a fraction
                            of the lines (about 60% of the L2 worth) loaded evict-last, the per-sweep operators
                            evict-first.  Modes 1 and 2 return the lines to normal priority at the end of
                            every step. */
  int32_t factor;        /* IETI_FACTOR_* (MIXED precision only; must be IETI_FACTOR_FP64 with FP64) */
  /* Newton's method for a nonlinear reluctivity (ignored for linear problems).  Each
   * iteration evaluates the FP64 residual R(a) = W a + dt N(a) - f of the nonlinear
   * system on the device and solves J d = -R with one dual-primal PCG solve (cg_tol);
   * max_sweeps bounds the iterations.  The step stops when ||R|| <= outer_tol ||f|| or,
   * with newton_tol > 0, when ||d|| <= newton_tol ||a|| after an update. */
  int32_t refactor;      /* IETI_REFACTOR_*: when the nonlinear patches and the coarse block are refactored */
  double newton_tol;     /* relative-update stop (0: residual test only) */
  /* Initial iterate of each step's refinement sweeps.  0: the previous state a^l.
   * 1: the linear extrapolation in time 2 a^l - a^{l-1}; 2: the quadratic one
   * 3 a^l - 3 a^{l-1} + a^{l-2} (lower orders while fewer states exist after setup or
   * ieti_set_state).  The right-hand side M a^l + dt j^{l+1} and the stopping test are
   * unchanged, so the step reaches the same outer_tol, usually in fewer sweeps. */
  int32_t predictor;
  /* Schedule of the persistent dual-primal kernel (pcg_mode 0): CTAs per SM, TMA
   * ring stages and bytes per stage.  0: the rule (one CTA per SM, three stages of
   * at most 64 KB).  1: autotune at setup: every feasible schedule of a fixed
   * candidate list runs a few PCG iterations on a synthetic right-hand side and the
   * fastest is kept, then partitions of the Psi rows of their own are tried on it
   * (results do not depend on the schedule beyond rounding order).
   * tune_cache (NULL: none) names a text file of earlier choices keyed by device name,
   * precision and problem sizes: a matching entry is used without timing, a new
   * choice is added to it.  An unreadable or malformed cache is ignored (tuned
   * afresh); a failed write leaves setup successful (ieti_info.pcg_sched_source). */
  int32_t autotune;
  const char *tune_cache;
  /* 1: run the refinement sweeps of each step of a linear problem as one CUDA graph
   * (a while node whose condition a device kernel sets from the assembled residual
   * norm and the PCG status: no host round trip per sweep); 0: the host loop.  The
   * graph is built at setup and needs pcg_mode 0, profile 0 and l2_persist != 1; if
   * building it fails the host loop runs (ieti_info.step_graph).  Same sweeps, same
   * stopping rules, same results. */
  int32_t graph;
  /* Bound of every grid-barrier wait of the persistent dual-primal kernel, in polls of
   * the arrival counter.  0: the default (about 1-3 s).  A wait that runs out sets an
   * error flag, every CTA waits for its own copies in flight and returns, and the step
   * returns IETI_ERR_TIMEOUT.  Small values exist to test that path. */
  int32_t wait_limit;
  int32_t coarse;        /* IETI_COARSE_*: solve of the coarse problem (ND: linear problems, pcg_mode 0) */
  int32_t coarse_leaf;   /* nested dissection: boxes of at most this many patches are not cut further
                            (0: the tree shape of least modelled solve time over a candidate list) */
  int32_t factor_arena_mb; /* budget of the setup factorization's arena of dense patch blocks, MiB: the
                              patches are factored in batches that fit it (0: 64 GB or 40% of the free
                              device memory, whichever is smaller) */
  int32_t coarse_top;    /* nested dissection: k >= 2 merges the separators of the top k levels of the
                            bisection into one dense root block, 1 merges none; 0: none when coarse_leaf
                            is given, else chosen with the leaf size by the same model */
  /* 1: the preconditioner (any precond, also NONE) in balancing form, the reading of
   * the deflation that Sec. 5 recommends for the Dirichlet preconditioner:
   *   M_bal = (I - P) M (I - P)^T + U E^{-1} U^T,  P = U E^{-1} U^T F,  E = U^T F U,
   * with U one column per pair of patches joined by multipliers (the indicator of that
   * pair's multipliers).  M_bal is symmetric and the solution is unchanged.  Setup
   * applies F to the k columns of U (k = ieti_info.deflation_dim) and keeps F U (k x m
   * FP64) on the device; every PCG iteration streams it twice.  The dual problem then
   * runs in the host-loop PCG (pcg_mode 1, no graph), so the coarse problem uses the
   * dense inverse (coarse = ND is refused).  IETI_ERR_TOO_LARGE when 8 k m > 8 GB or
   * k > 4096.  0: off. */
  int32_t deflation;
  /* n >= 2: the nested-dissection tree is cut where ieti_shard_plan cuts the patch grid
   * for n ranks (then the rest by midpoints), so that every rank's patches form whole
   * subtrees and the shared top of ieti_shard_coarse is only the ranks' separators;
   * 0 or 1: midpoint cuts.  At most 31 and at most the number of patches. */
  int32_t coarse_ranks;
} ieti_options;

#define IETI_REFACTOR_EVERY 0  /* at every Newton iterate (Newton's method) */
#define IETI_REFACTOR_STEP 1   /* at the first iterate of every step, frozen within the step (modified Newton) */
#define IETI_REFACTOR_NEVER 2  /* never after setup (the tangent at a = 0) */

/* Coil source through its potential T = T_z(r) chi(|z - zc| < hz) e_z (J = curl T):
 * T_z = J0 (r_out - r) on r_in < r < r_out, J0 (r_out - r_in) for r <= r_in, 0 beyond;
 * r = distance to the axis x = xc, y = yc.  j_k = <T, curl w_k> (Sec. 2.2 load vector). */
typedef struct {
  double J0, r_in, r_out, xc, yc, zc, hz;
} ieti_coil;

typedef struct {
  int32_t cg_its;        /* PCG iterations of the step (all refinement sweeps) */
  int32_t sweeps;        /* refinement sweeps taken */
  double rel_res;        /* last PCG relative residual */
  double outer_res;      /* ||f - W a|| / ||f|| after the step (FP64) */
  double t_step_ms;      /* device time of the step (CUDA events) */
  int64_t kernel_launches; /* kernels this library launched for the step */
  int32_t refactors;     /* refactorizations of the nonlinear patches in the step (nonlinear problems) */
} ieti_stats;

typedef struct {
  int64_t n_dofs;        /* global lattice edges (ieti_num_dofs) */
  int64_t n_free;        /* r + p edges */
  int64_t n_lambda;      /* multipliers (one per pair of copies of a shared r-DOF) */
  int64_t n_coarse;      /* primal unknowns */
  int64_t sum_ni, sum_nb, sum_np;  /* interior / interface / primal copies over patches */
  int64_t max_n;         /* largest local block n_i + n_b + n_p */
  int64_t bytes_iter;    /* algorithmic bytes one PCG iteration streams (operators + coarse) */
  int64_t bytes_device;  /* device memory held by the context */
  double t_setup_host_ms, t_setup_device_ms;
  int64_t kernel_launches_setup;
  int64_t l2_window_bytes;   /* per-iteration operators covered by the persisting L2 window (0: off) */
  double l2_hit_ratio;       /* fraction of that window marked persisting */
  int64_t iter_operator_bytes; /* size of the per-iteration operator arena */
  double t_factor_ms;        /* device time of the patch-block partial Cholesky (both phases, CUDA events) */
  double tc_ms;              /* of which in the tensor-core trailing updates (IETI_FACTOR_TF32X3 / TF32) */
  double tc_flops;           /* tensor-core flops those updates issued (3 products per update for TF32X3) */
  double tc_useful_flops;    /* the multiply-adds of the updated entries, x 2 */
  int64_t tc_launches;       /* tensor-core update launches */
  double factor_flops;       /* useful flops of the patch-block partial Cholesky (both phases) */
  int64_t nl_patches;        /* patches refactored by Newton (holding elements of the nonlinear law) */
  int64_t nl_elements;       /* elements of the nonlinear law */
  int64_t refactors;         /* refactorizations since setup */
  int64_t nl_coarse_block;   /* coarse unknowns of those patches, updated by the block formula at every
                                refactorization (0: the whole coarse block is refactored) */
  double t_refactor_ms[4];   /* with options.profile = 1: device time of all refactorizations since setup in
                                the tangent assembly, the local factorization + extraction, the coarse update,
                                and in total (CUDA events) */
  int32_t pcg_grid;          /* CTAs of the persistent dual-primal kernel */
  int32_t pcg_stages;        /* TMA ring stages per CTA */
  int32_t pcg_stage_bytes;   /* bytes per stage */
  int32_t pcg_psi_partition; /* 0: the Psi rows share the S_bb rows' partition; > 0: their own, balanced with
                                this per-row overhead (elements) */
  int32_t pcg_sched_source;  /* 0: rule, 1: autotuned, 2: autotuned and written to tune_cache, 3: from tune_cache */
  int32_t tune_candidates;   /* schedules timed by the autotuner */
  double tune_ms;            /* host time of the autotuning */
  double tune_us_per_it[2];  /* measured time per PCG iteration: the rule's schedule, the chosen one */
  int32_t step_graph;        /* 1: the sweeps of a step run as one CUDA graph (ieti_options.graph) */
  int32_t coarse_mode;       /* IETI_COARSE_DENSE or IETI_COARSE_ND (0 without coarse unknowns) */
  int32_t coarse_nodes;      /* nodes of the nested-dissection tree */
  int32_t coarse_levels;     /* grid-synchronised phases of one coarse solve */
  double coarse_bytes;       /* algorithmic bytes of one coarse solve */
  double t_coarse_ms;        /* host time of the coarse assembly and factorization at setup */
  int32_t factor_batches;    /* patch batches of the setup factorization */
  int32_t pcg_seg_weight;    /* per-segment weight of the persistent kernel's row partitions (elements; the
                                autotuner tries a few, 0 by the rule) */
  int32_t coarse_flow;       /* 1: the nested-dissection levels wait on per-node completion counters instead of
                                grid barriers (the autotuner's choice; 0 by the rule) */
  int32_t deflation_dim;     /* columns of the balanced preconditioner's pair space (0: off) */
} ieti_info;

/* Kernel classes timed when options.profile = 1 (CUDA events on the step stream). */
#define IETI_K_GEMV_H 0   /* [F_s; Psi_s^T] u: dual operator and primal right-hand side, one launch per F apply */
#define IETI_K_GEMV_Q 1   /* Psi_s q: primal correction */
#define IETI_K_GEMV_P 2   /* S_bb u: Dirichlet preconditioner */
#define IETI_K_GEMV_S 3   /* S_c^{-1} c: coarse solve */
#define IETI_K_GEMV_Y 4   /* interior condensation / recovery GEMVs */
#define IETI_K_TRI 5      /* interior substitutions: batched triangular GEMVs with X = L_ii^{-1} and X^T */
#define IETI_K_SPMV 6     /* FP64 sparse M a, W a */
#define IETI_K_VEC 7      /* gathers, jumps, dots, axpys (not timed) */
#define IETI_K_PCG 8      /* the persistent PCG kernel (bytes = iterations x algorithmic bytes per iteration) */
#define IETI_K_NCLASS 9

typedef struct {
  int64_t launches;
  double total_ms;       /* sum of CUDA-event durations */
  double bytes;          /* algorithmic bytes moved by those launches (operator entries + vectors, once) */
} ieti_kernel_stat;

typedef struct ieti_ctx ieti_ctx;

/* Sec. 2.2-3: assemble K, M per patch, build the tree-cotree gauge and e/p/r
 * classes, the multipliers B and primal map N, then (device >= 0) factor all local
 * blocks and the coarse Schur complement on the GPU.  *out is set on success.
 * Errors: INVALID_ARG, NONCONFORMING, NOT_SPD, CUDA, OOM. */
int ieti_setup(const ieti_problem *problem, const ieti_options *options, ieti_ctx **out);

/* Number of global DOFs (lattice edges, the length of all global vectors). */
int64_t ieti_num_dofs(const ieti_ctx *ctx);

int ieti_get_info(const ieti_ctx *ctx, ieti_info *info);

/* Load vector j (Sec. 2.2, (j_i)_k = <J, w_k>) of a coil source, via j_k = <T, curl w_k>,
 * assembled over patches into the global numbering.  Host computation; j_out is a host
 * buffer of ieti_num_dofs() doubles.  Works on host-only contexts. */
int ieti_load_vector(const ieti_ctx *ctx, const ieti_coil *coil, double *j_out);

/* Quadrature points of the assembly, for sources given as functions of space
 * (Sec. 2.2 load vector (j_i)_k = <J, w_k> with a general J): the physical coordinates
 * (x, y, z) of every point, patch after patch, within a patch element after element
 * (x fastest) and within an element the (p_d + 2)^3 Gauss points (x fastest).
 * Two-call protocol: with xyz NULL only *n_points is written; otherwise xyz holds
 * 3 * (*n_points) doubles (host) and *n_points must be at least the count.  Works on
 * host-only contexts.  Errors: INVALID_ARG. */
int ieti_quad_points(const ieti_ctx *ctx, double *xyz, int64_t *n_points);

/* Load vector j_k = <J, w_k> of a current density J sampled at the quadrature points
 * of ieti_quad_points (J_xyz: 3 doubles per point, same order; host), assembled into
 * the global numbering (j_out: ieti_num_dofs() doubles, host).  For J = curl T of a
 * coil, ieti_load_vector is the exact alternative.  Works on host-only contexts. */
int ieti_load_vector_points(const ieti_ctx *ctx, const double *J_xyz, double *j_out);

/* Host-side classification (works on host-only contexts): per global DOF,
 * cls[g] = 0 (e), 1 (p), 2 (r) and tree[g] = 1 for tree edges (Sec. 3).  Either
 * pointer may be NULL. */
int ieti_dof_classes(const ieti_ctx *ctx, int8_t *cls, int8_t *tree);

/* Patch matrices of Sec. 2.2 in the patch-local edge numbering (component-major,
 * i fastest): which = 0 for K_s (nu curl-curl), 1 for M_s (sigma mass).  Two-call
 * protocol: with ptr/col/val NULL only *nnz is written; otherwise ptr has n_s+1
 * entries and col/val *nnz entries (host buffers).  Works on host-only contexts. */
int ieti_patch_csr(const ieti_ctx *ctx, int32_t patch, int32_t which, int32_t *n_rows, int64_t *nnz,
                   int32_t *ptr, int32_t *col, double *val);

/* One implicit-Euler step (Eq. (11)): a^{l+1} from the stored a^l and the load
 * vector j^{l+1} (global numbering, ieti_num_dofs() doubles, in host or device
 * memory per j_mem).  stats may be NULL.  Errors: NO_DEVICE, CG_NOT_CONVERGED
 * (the state is still advanced with the last iterate), CUDA. */
int ieti_step(ieti_ctx *ctx, const double *j_next, int32_t j_mem, ieti_stats *stats);

/* Copy the current a^l (global numbering, e entries 0) to a_out (len doubles). */
int ieti_solution(const ieti_ctx *ctx, double *a_out, int64_t len, int32_t out_mem);

/* Replace the state a^l (checkpoint resume); e entries are ignored. */
int ieti_set_state(ieti_ctx *ctx, const double *a, int64_t len, int32_t a_mem);

/* Nested-dissection tree of the coarse problem (host query; built for every context
 * with coarse unknowns, with options.coarse_leaf).  Nodes in postorder; node p owns the
 * coarse unknowns at elimination positions [k0[p], k0[p] + nk[p]) and couples to the
 * ancestor positions s_idx[s_off[p] .. s_off[p+1]); parent[p] = -1 for a root.
 * elim_pos[g] (ieti_num_dofs() entries) is the elimination position of the primal edge
 * g, -1 for other edges.  Two-call protocol: with the arrays NULL only *n_nodes and
 * *n_s are written; otherwise k0, nk, parent hold *n_nodes entries, s_off *n_nodes + 1,
 * s_idx *n_s.  Any array may be NULL.  Errors: INVALID_ARG. */
int ieti_coarse_tree(const ieti_ctx *ctx, int32_t *n_nodes, int64_t *n_s, int32_t *elim_pos, int32_t *k0,
                     int32_t *nk, int32_t *parent, int64_t *s_off, int32_t *s_idx);

/* Patch-sharded layout of the dual-primal solve for n_ranks ranks (host query, 1 <=
 * n_ranks <= min(31, patches)).  The patches are independent units (Sec. 3); the
 * interface problem couples them through the multiplier jumps, the coarse right-hand
 * side and the PCG dot products.  rank_of_patch[n_patches]: recursive coordinate
 * bisection of the patch grid balanced by the local sizes.  lam_owner[n_lambda]: the rank
 * holding the multiplier's lower patch; lam_peer[n_lambda]: the rank of its upper patch
 * when that is another rank (the multiplier is cut: its partial jump crosses once per
 * PCG iteration), else -1.  coarse_owner[n_coarse]: the lowest rank holding a copy of
 * the primal unknown.  Any array may be NULL.  Errors: INVALID_ARG. */
int ieti_shard_plan(const ieti_ctx *ctx, int32_t n_ranks, int32_t *rank_of_patch, int32_t *lam_owner,
                    int32_t *lam_peer, int32_t *coarse_owner);

/* The coarse solve (Sec. 3: the primal Schur complement S_c) on the ranks of
 * ieti_shard_plan (host query).  node_rank[n_nodes of ieti_coarse_tree]: the rank that
 * computes node p of the nested-dissection tree when every patch of the node's box is on
 * that rank (its whole subtree then is too), else -1: a shared node of the top, computed
 * by every rank after one sum over the ranks of the owned subtrees' updates into the
 * shared fronts.  Each rank then holds the coarse values its patches need without a
 * further exchange.  Errors: INVALID_ARG (n_ranks out of range, NULL). */
int ieti_shard_coarse(const ieti_ctx *ctx, int32_t n_ranks, int32_t *node_rank);

/* Multipliers and patch blocks (host queries): multiplier l joins the interface copy
 * pos_s[l] of patch s[l] to the copy pos_t[l] of patch t[l] (s < t, lambda = copy in s -
 * copy in t; positions index the patch's interface block); per patch the block sizes
 * ni, nb, np (interior, interface, primal copies) and, patch after patch, the coarse
 * unknown of every primal copy (coarse ids ascending with the primal edges).  Arrays of
 * n_lambda, n_patches and sum np entries; any may be NULL.  Errors: INVALID_ARG. */
int ieti_multipliers(const ieti_ctx *ctx, int32_t *s, int32_t *pos_s, int32_t *t, int32_t *pos_t);
int ieti_patch_blocks(const ieti_ctx *ctx, int32_t *ni, int32_t *nb, int32_t *np, int32_t *coarse_of_copy);

/* Per-class kernel statistics accumulated since the last reset (options.profile = 1);
 * out has IETI_K_NCLASS entries.  reset != 0 clears the counters after reading. */
int ieti_kernel_stats(ieti_ctx *ctx, ieti_kernel_stat *out, int32_t reset);

/* Per-phase timing of the persistent PCG kernel (options.profile = 1): mean over the
 * traced iterations of the work time of CTA 0 in each of its six phases and of its
 * wait at the grid barrier that ends the phase, in microseconds (%globaltimer).
 * work_us and wait_us have 6 entries each.  sub_us (NULL or 12 entries) splits the
 * work of the four operator-streaming phases (the dual operator, the coarse solve,
 * the primal correction, the preconditioner; 3 entries each): from the phase start to
 * the staged first vector segment, from there to the first operator chunk in shared
 * memory, and from there to the last row.  reset != 0 clears the accumulators. */
int ieti_pcg_phase_times(ieti_ctx *ctx, double *work_us, double *wait_us, double *sub_us, int32_t reset);

/* Per-level timing of the nested-dissection coarse solve (options.profile = 1, coarse
 * mode ND): mean over the traced PCG iterations of CTA 0's time in each level of one
 * coarse solve (forward levels by height, then backward levels by depth), in
 * microseconds (%globaltimer): entries 4 lv .. 4 lv + 3 of level lv hold the staging of
 * its first vector segment (from the end of the previous level's barrier), the wait for
 * its first operator chunk, the rows, and the wait at its grid barrier.  us receives n
 * entries (0 beyond the tree's levels).  reset != 0 clears the accumulators.  Errors:
 * INVALID_ARG, NO_DEVICE. */
int ieti_coarse_level_times(ieti_ctx *ctx, double *us, int32_t n, int32_t reset);

/* Batched dense partial Cholesky, the kernel family behind both Schur complements
 * of Sec. 3 (local W_rr eliminations and the coarse block), exposed for callers and
 * kernel-level tests.  Matrix b is row-major n[b] x n[b] at base_dev + offsets[b]
 * (device memory of the current device, offsets in doubles, caller-owned; only the
 * lower triangle is read and written).  The first n_pivots[b] pivots are eliminated
 * in place: those columns hold the factor L (A = L L^T on the leading block,
 * L21 = A21 L11^{-T}) and the trailing lower triangle holds the Schur complement
 * A22 - L21 L21^T.  status_out[b] (host) is 0, or 1 + the index of the first
 * non-positive pivot (the factorization then continues with a unit pivot).
 * offsets, n, n_pivots, status_out are host arrays of length batch; stream is a
 * cudaStream_t (0 = legacy default).  Allocates and frees its device scratch (the
 * descriptor copies and the status words) on every call.  Returns 0, INVALID_ARG
 * (batch < 1, n < 1, n_pivots outside [0, n], NULL pointers), CUDA or OOM. */
int ieti_potrf_batched(int32_t batch, double *base_dev, const int64_t *offsets, const int32_t *n,
                       const int32_t *n_pivots, int32_t *status_out, void *stream);

/* The FP32 variant of ieti_potrf_batched in the arithmetic `factor` (IETI_FACTOR_FP32,
 * IETI_FACTOR_TF32X3, IETI_FACTOR_TF32, IETI_FACTOR_BF16X3 or IETI_FACTOR_BF16: the
 * data stays FP32, only the trailing-update operands are rounded).  Matrix b is
 * row-major n[b] x n[b] with
 * leading dimension ld[b] >= n[b] at base_dev + offsets[b] (floats).  The tensor-core
 * variants need 16-byte rows and bases: ld[b] and offsets[b] multiples of 4.  Same
 * results, status and ownership rules as ieti_potrf_batched; the error is that of
 * the FP32 (or TF32 / BF16) arithmetic.  Allocates its scratch (tile list, the panel
 * buffer of 2 x sum(n) x 256 operand words) per call.  Returns 0, INVALID_ARG (also for a bad
 * factor or misaligned ld / offsets), CUDA or OOM. */
int ieti_potrf_batched_f32(int32_t batch, float *base_dev, const int64_t *offsets, const int32_t *n,
                           const int32_t *ld, const int32_t *n_pivots, int32_t factor, int32_t *status_out,
                           void *stream);

/* ieti_potrf_batched for callers that must not allocate device memory: code that
 * runs under a fixed memory budget (an application that reserved all device memory
 * for its own pool), inside a host callback or library hook where cudaMalloc is not
 * allowed, or that must avoid the implicit device synchronisation cudaFree causes.
 * The paper has no counterpart; this is a library convenience.
 *
 * Same arguments, results and errors as ieti_potrf_batched.  Its scratch (the
 * descriptor copies and status words, 40 bytes per matrix) lives in one static
 * device array of IETI_NOALLOC_MAX_BATCH entries, which every device that loads the
 * library holds until the process exits; batch > IETI_NOALLOC_MAX_BATCH returns
 * IETI_ERR_TOO_LARGE.  It calls no cudaMalloc or cudaFree.  Every call looks up
 * the array's device address in the current device's context
 * (cudaGetSymbolAddress).  The call copies its descriptors from pageable host
 * memory and waits for its stream, so it cannot be called on a stream that is
 * being captured into a CUDA graph.  Every call shares the one array (the status
 * words are cleared at each call), so calls whose GPU work overlaps, on different
 * streams or threads, race. */
#define IETI_NOALLOC_MAX_BATCH 4096
int ieti_potrf_batched_noalloc(int32_t batch, double *base_dev, const int64_t *offsets, const int32_t *n,
                               const int32_t *n_pivots, int32_t *status_out, void *stream);

const char *ieti_last_error(const ieti_ctx *ctx);
/* Message of the last failed ieti_setup or ieti_potrf_batched[_noalloc] (no context exists then). */
const char *ieti_setup_error(void);

void ieti_destroy(ieti_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* IETI_H */
