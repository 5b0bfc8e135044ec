/*
 * pff.h -- C ABI of the GB300 solver for pressurized phase-field fracture.
 *
 * The library solves, on one GPU, the loading steps of Formulation 1 of
 * Heister & Wick (arXiv 1806.09924, Section 2): displacements u and a phase
 * field phi on a tensor-product Q1 mesh (Section 3), with the irreversibility
 * constraint phi <= phi_old, by the combined semi-smooth Newton / primal-dual
 * active-set method of Section 3 whose linear systems are solved by FGMRES with
 * the block-diagonal preconditioner of Section 3.1 (one smoothed-aggregation
 * AMG V-cycle per diagonal block).  The crack functionals TCV and COD of
 * Section 4 are evaluated on the device.
 *
 * Conventions shared by every entry point
 *   - Return value: PFF_OK (0) on success, a negative PFF_ERR_* code on failure;
 *     pff_last_error() then returns a thread-local message.  A failed call
 *     leaves the problem usable unless the code is PFF_ERR_CUDA.
 *   - Ownership: a pff_problem is created and owned by the library and holds
 *     all its state in device memory until pff_destroy.  Input arrays are
 *     copied, never retained.  Output arrays are owned by the caller.
 *   - "host" pointers point to CPU memory; "_dev" entry points take pointers
 *     to device memory of the current CUDA device (for example tensors
 *     allocated by PyTorch) and enqueue work on the problem's stream without
 *     synchronizing.  All other entry points synchronize the stream before
 *     they return.
 *   - Layout: node (i,j,k) has index i + (nx+1)(j + (ny+1)k) (x fastest);
 *     u is [n_nodes][dim] row-major; phi, phi_old are [n_nodes].  A full
 *     solution / residual vector is [u (dim*n_nodes) ; phi (n_nodes)], the
 *     basis order of Section 3.1 (all displacement DoFs, then the phase field).
 *   - Thread safety: calls on one problem must not overlap; distinct problems
 *     are independent.
 */
#ifndef PFF_H
#define PFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PFF_OK 0
#define PFF_ERR_INVALID_ARG (-1)   /* bad size, pointer, option or call order */
#define PFF_ERR_OOM (-2)           /* device allocation failed */
#define PFF_ERR_NOT_CONVERGED (-3) /* Newton or Krylov iteration cap reached */
#define PFF_ERR_LINESEARCH (-4)    /* reserved: line-search failures are reported, not fatal */
#define PFF_ERR_CYCLE (-5)         /* reserved: active-set locks are reported, not fatal */
#define PFF_ERR_NAN (-6)           /* a NaN / Inf appeared in a residual or norm */
#define PFF_ERR_TIMEOUT (-7)       /* a bounded device-side wait gave up */
#define PFF_ERR_CUDA (-8)          /* CUDA runtime error; the problem may be unusable */
#define PFF_ERR_CAPACITY (-9)      /* an internal fixed-size table overflowed */

#define PFF_PREC_FP64 0   /* FP64 everywhere */
#define PFF_PREC_MIXED 1  /* FP32 AMG preconditioner inside FP64 FGMRES / Newton */

#define PFF_APPLY_AUTO 0        /* pick the faster FP64 Jacobian apply (timed once) */
#define PFF_APPLY_ASSEMBLED 1   /* stencil-assembled Section 3.1 blocks */
#define PFF_APPLY_MATFREE 2     /* matrix-free element-batched apply */

#define PFF_PC_AMG 0     /* block-diagonal preconditioner, one SA-AMG V-cycle per block */
#define PFF_PC_JACOBI 1  /* point Jacobi (diagnostics only) */
#define PFF_PC_AMG_TRI 2 /* block lower-triangular: the phase-field V-cycle acts on
                            r_phi - M_phi_u z_u (uses the M_phi_u coupling the
                            block-diagonal form of Section 3.1 leaves out) */

typedef struct pff_problem pff_problem;

/* Solver options.  pff_default_options fills the defaults given here. */
typedef struct pff_options {
  int precision;        /* PFF_PREC_FP64 (default) or PFF_PREC_MIXED */
  double c;             /* active-set constant c > 0 (Section 3 algorithm, step 2), in units
                           of G_c/eps: indicator = F_phi/m + c (G_c/eps)(phi - phi_old); 0.1 */
  double tol_newton;    /* stop when the scaled reduced residual (inf-norm) fell by this
                           (or below atol_newton); 1e-10 */
  double tol_step;      /* ... and the last Newton step is below this, relative per block; 1e-9 */
  double tol_linear;    /* FGMRES relative residual (Table 1 uses 1e-8); 1e-8 */
  int max_newton;       /* Newton / active-set iterations per loading step; 50 */
  int max_halvings;     /* line-search halvings; 10 */
  int cycle_lock;       /* lock an index active after this many membership changes; 3 */
  int krylov_restart;   /* FGMRES restart length m; 40 */
  int max_krylov;       /* FGMRES iterations per linear solve; 600 */
  int cheb_degree;      /* Chebyshev smoother degree on the finest level; 4 */
  double amg_theta;     /* strength threshold on the distance Laplacian of the mesh nodes
                           (w_ij = 1/|x_i - x_j|^2 strong iff w_ij^2 >= theta^2 wmax_i wmax_j);
                           0.02 (0 treats every coupling as strong and fails on graded
                           meshes; 0.06 and above coarsen the graded meshes less
                           effectively: +10 % time on the graded 2d and 3d workloads) */
  int amg_coarse_max;   /* largest coarse level (scalar rows) solved directly; 1000 */
  int apply_variant;    /* PFF_APPLY_*; PFF_APPLY_AUTO */
  int precond;          /* PFF_PC_*; PFF_PC_AMG */
  double cheb_ratio;    /* Chebyshev smoothing interval [lmax/ratio, 1.1 lmax]; 8 */
  double tol_active;    /* active-set threshold tau, in units of G_c/eps; 1e-10 */
  double atol_newton;   /* absolute floor of the scaled reduced residual test; 1e-14 */
  double tol_change;    /* the active set counts as unchanged when every index that changed
                           membership has |indicator| <= tol_change G_c/eps (such an index is
                           a tie: both memberships satisfy the complementarity test); 1e-9 */
  int spmv_group;       /* block-sparse kernel of the AMG hierarchy: lanes per block row of
                           the vector-CSR kernels, 1, 2, 4, 8, 16 or 32; 64 = SELL-32 layout
                           (one thread per block row, FP32 hierarchies; FP64 ones fall back
                           to vector-CSR); -1 = one thread per scalar row (reference);
                           0 = timed per matrix at hierarchy build (default; the choice is
                           cached per block shape and size class) */
  int amg_reuse;        /* 1: a displacement hierarchy carries over to the next loading step
                           while phi~ moved by at most amg_reuse_tol (max norm) since its
                           build; 0: rebuilt every loading step; 1 */
  double amg_reuse_tol; /* see amg_reuse; 0.05 */
  int precond_overlap;  /* 1: the displacement and phase-field V-cycles of the block
                           preconditioner run concurrently on two streams; 0: one after the
                           other; 1 */
  int cheb_degree_coarse; /* Chebyshev degree on AMG levels >= 1; 0 = cheb_degree; -1 = by
                           dimension: 2 in 2d, 3 in 3d; -1 */
  double forcing_max;   /* > 0: inexact Newton with the Eisenstat-Walker forcing term: the
                           first linear solve of a loading step to forcing_max, later ones to
                           0.9 (rho_k / rho_k-1)^2, never tighter than tol_linear; 0: every
                           solve to tol_linear (as in Table 1); 0.  Faster (1e-3 halves the
                           3d penny step), but along the other Newton path the cycle rule
                           locks other indices and the converged phi can move by ~1e-5 */
  int iter_graph;       /* 1: problems up to 10^6 DoFs on a non-default stream run each
                           FGMRES iteration's preconditioner and Jacobian apply as one CUDA
                           graph (same kernels, same order); 0: ordinary launches; 1 */
  double amg_rebuild_phi; /* the phase-field hierarchy is rebuilt when the active set differs
                           from the one it was built for in more than this fraction of the
                           nodes (otherwise only its finest level is refreshed); 1e-3 */
  int amg_age_phi;      /* ... or once it has served this many Newton iterations; 8 */
  int amg_levels_phi;   /* at most this many levels in the phase-field hierarchy, the last
                           one smoothing only (1: Chebyshev smoothing on the assembled
                           stencil, no coarse levels); 0 = coarsen down to amg_coarse_max;
                           -1 = by resolution: 1 while the smallest cell is at least eps/4
                           (the block is dominated by its mass term G_c/eps M), else 0
                           (finer cells: its eps-scaled Laplacian takes over, which
                           smoothing alone resolves poorly); -1 */
  int cheb_degree_phi;  /* Chebyshev degree on the finest level of the phase-field block;
                           0 = cheb_degree; 4 */
  int amg_rotations;    /* near-null space of the displacement hierarchy: 1 = rigid-body
                           modes (translations and rotations; coarse blocks of 3 x 3 in
                           2d, 6 x 6 in 3d), 0 = translations only (d x d blocks),
                           -1 = by dimension: 1 in 2d, 0 in 3d (measured faster there:
                           the 6 x 6 coarse operators cost more than the iterations
                           they save); -1 */
} pff_options;

/* Per loading step (or per Newton iteration for pff_newton_step) report. */
typedef struct pff_step_report {
  int status;           /* PFF_OK or the error code of the step */
  int converged;        /* 1 when the stopping test of the Section 3 algorithm held */
  int newton_its;       /* Newton / active-set iterations taken */
  int krylov_its;       /* total FGMRES iterations */
  int krylov_its_max;   /* largest FGMRES iteration count of one Newton step (cf. Table 1) */
  int active;           /* size of the final active set */
  int changed;          /* active-set changes in the last iteration */
  int locked;           /* indices locked active by the cycle rule */
  int ties;             /* nodes whose active-set indicator is within round-off of 0 */
  int linesearch_fails; /* line searches that fell back to the full step */
  double rho0;          /* scaled reduced residual (inf-norm) at the first iteration */
  double rho;           /* ... at the last iteration */
  double time_ms;       /* wall time of the step */
  int amg_builds_u;     /* displacement hierarchies built during the step (0: carried over) */
  int amg_builds_phi;   /* phase-field hierarchies built during the step */
} pff_step_report;

void pff_default_options(pff_options* opts);

/* Checks opts (NULL: the defaults) against the ranges documented above without
 * touching the device.  Returns PFF_OK, or PFF_ERR_INVALID_ARG with the first
 * violated rule in pff_last_error().  Every solver entry point applies the same
 * check; pff_server_create applies it to the server's options. */
int pff_check_options(const pff_options* opts);

/* Mesh and problem set-up -------------------------------------------------- */

/* Tensor-product Q1 mesh of the box spanned by axis_coords (Section 3: Q1^c on
 * quadrilaterals / hexahedra).  dim is 2 or 3; n_cells[a] >= 1 cells along
 * axis a; axis_coords[a] points to n_cells[a]+1 strictly increasing host
 * doubles (copied).  Homogeneous Dirichlet conditions on u at the whole outer
 * boundary (Section 2).  Initial state: u = 0, phi = phi_old = 1.
 * *out receives the new problem (owned by the library until pff_destroy). */
int pff_create_mesh(int dim, const int32_t* n_cells, const double* const* axis_coords,
                    pff_problem** out);

/* Material of Formulation 1 (Section 2): Young's modulus E > 0, Poisson ratio
 * 0 <= nu < 0.5 (Lame coefficients; plane strain in 2d), critical energy
 * release rate G_c > 0, stiffness floor kappa >= 0, regularization eps > 0. */
int pff_set_material(pff_problem* prob, double E, double nu, double Gc, double kappa, double eps);

/* Start a loading step with constant pressure p (Section 4 uses p = 1e-3):
 * forms the extrapolation phi~ of Section 2 (phi_old in the first two steps,
 * whose history starts at the initial crack field rather than a computed
 * solution; clamp(2 phi_old - phi_prev, 0, 1) afterwards) and resets the
 * per-step Newton state. */
int pff_set_pressure(pff_problem* prob, double p);

/* Crack of half length / radius l0 centred at the origin (Section 4): phi =
 * phi_old = 0 on all nodes of cells cut by the segment |x| < l0, y = 0 (2d)
 * or the disc x^2+y^2 < l0^2, z = 0 (3d), 1 elsewhere; u = 0; history reset. */
int pff_set_crack(pff_problem* prob, double l0);

/* General state (host arrays, copied; NULL keeps the current value).
 * steps_done = number of completed loading steps (selects phi~). */
int pff_set_state(pff_problem* prob, const double* u, const double* phi, const double* phi_old,
                  const double* phi_prev, int steps_done);

/* Solver entry points ------------------------------------------------------ */

/* One iteration of the Section 3 algorithm within the current loading step:
 * residual, active set, reduced Jacobian, FGMRES solve, line search, update.
 * report->converged = 1 (and no update) once the stopping test holds. */
int pff_newton_step(pff_problem* prob, const pff_options* opts, pff_step_report* report);

/* Finish the current loading step: phi_prev <- phi_old, phi_old <- phi. */
int pff_end_loading_step(pff_problem* prob);

/* Solve n_steps loading steps with pressures p_schedule[0..n_steps-1] (host),
 * each to convergence; reports[n_steps] (host, caller-owned) may be NULL.
 * Returns PFF_ERR_NOT_CONVERGED if a step hit max_newton (reports say which). */
int pff_solve_loading_steps(pff_problem* prob, int n_steps, const double* p_schedule,
                            const pff_options* opts, pff_step_report* reports);

/* TCV_h = int u . grad phi over the domain and the crack opening
 * COD_h = int u . grad phi along lines normal to the crack (Section 4).
 * pts: n_pts abscissae x (2d) or (x, y) pairs (3d), host; a point on a mesh
 * line averages the adjacent cells.  tcv (1 double) and cod (n_pts doubles)
 * are host outputs; either may be NULL. */
int pff_eval_tcv_cod(pff_problem* prob, int n_pts, const double* pts, double* tcv, double* cod);

/* Copy the state out to host arrays (any may be NULL): u [n_nodes*dim],
 * phi [n_nodes], active [n_nodes] (1 = phase-field index in the last active set). */
int pff_get_solution(pff_problem* prob, double* u, double* phi, uint8_t* active);

/* Use this CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream()) for
 * all later work of the problem; NULL selects the legacy default stream. */
int pff_set_stream(pff_problem* prob, void* stream);

int pff_get_sizes(const pff_problem* prob, int* dim, int64_t* n_nodes, int64_t* n_dofs);

void pff_destroy(pff_problem* prob);

const char* pff_last_error(void);

/* Component entry points (device pointers, asynchronous on the problem's
 * stream).  They expose the steps of the hot path one by one for parity tests
 * and benchmarks; all vectors use the full [u ; phi] layout of n_dofs doubles. */

/* F = -r(U): Eq. (E22ATW) and (E33ATW) tested with every basis function at the
 * current state, pressure and phi~ (no elimination). */
int pff_residual_dev(pff_problem* prob, double* F_dev);

/* Active set of the Section 3 algorithm (step 2) at the current state:
 * indicator[i] = F_phi,i / m_i + c (phi_i - phi_old,i) with the lumped mass m;
 * active[i] = indicator > 0.  Stores the set in the problem (used by the
 * reduced Jacobian below).  Either output may be NULL. */
int pff_active_set_dev(pff_problem* prob, double c, uint8_t* active_dev, double* indicator_dev);

/* Assemble the Section 3.1 Jacobian blocks (M_uu, M_phi_u, M_phi_phi) at the
 * current state in the node-stencil format, reduced by the Dirichlet set and
 * the stored active set. */
int pff_assemble(pff_problem* prob);

/* y = G~ x, the reduced Jacobian (identity rows and zero columns for Dirichlet
 * displacement DoFs and active phase-field DoFs; M_u_phi = 0).  variant:
 * PFF_APPLY_ASSEMBLED (needs pff_assemble) or PFF_APPLY_MATFREE. */
int pff_apply_jacobian_dev(pff_problem* prob, int variant, const double* x_dev, double* y_dev);

/* Build the block-diagonal SA-AMG preconditioner of the assembled blocks and
 * apply it: z = diag(V_uu, V_phiphi) r (one V-cycle per block). */
int pff_precond_setup(pff_problem* prob, const pff_options* opts);
int pff_precond_apply_dev(pff_problem* prob, const double* r_dev, double* z_dev);

/* Solve G~ x = b with preconditioned FGMRES (relative tolerance tol_linear on
 * the Jacobi-scaled residual).  *iters receives the iteration count. */
int pff_linear_solve_dev(pff_problem* prob, const pff_options* opts, const double* b_dev,
                         double* x_dev, int* iters);

/* Same as pff_set_state with device arrays of the current device (copied
 * device-to-device on the problem's stream; NULL keeps the current value). */
int pff_set_state_dev(pff_problem* prob, const double* u_dev, const double* phi_dev,
                      const double* phi_old_dev, const double* phi_prev_dev, int steps_done);

/* Adaptive refinement (Section 3, refinement strategy) ------------------------
 *
 * The paper refines octree meshes with hanging nodes: cells of the crack region
 * until eps = 2h holds there, the rest by a gradient-jump estimator for the
 * displacements.  Here the mesh stays a tensor product, so refinement splits
 * whole axis intervals (slabs of cells); a refined mesh is a new problem, and
 * the state moves to it by Q1 interpolation. */

/* Gradient-jump (Kelly-type) indicator of the current displacements per cell,
 * eta2[c] = (h_c / 24) * sum over the interior faces F of cell c of the
 * integral over F of |[du/dn]|^2 (h_c the cell diameter, [du/dn] the jump of
 * the normal derivative of every component; boundary faces contribute
 * nothing).  eta2_dev: n_cells doubles on the device, cells numbered like
 * nodes (x fastest).  Asynchronous on the problem's stream. */
int pff_cell_indicators_dev(pff_problem* prob, double* eta2_dev);

/* One refinement pass of the axes.  With S_a[i] the sum of eta2 over the
 * cells whose a-index is i, and minphi_a[i] the smallest phi on those cells'
 * nodes, interval i of axis a is split at its midpoint when
 *   S_a[i] > 0 and S_a[i] >= theta * max_i S_a[i]          (estimator), or
 *   minphi_a[i] < phi_band and its length exceeds h_band   (crack region:
 *                                                         h_band = eps / 2).
 * theta >= 0 (theta > 1 disables the estimator rule), h_band >= 0.
 * Outputs (host, caller-owned): n_cells_out[dim] and coords_out[a], each with
 * room for 2 * n_cells[a] + 1 doubles, strictly increasing and containing the
 * old coordinates.  The problem is not changed.  Synchronous. */
int pff_refine_axes(pff_problem* prob, double theta, double h_band, double phi_band,
                    int32_t* n_cells_out, double* const* coords_out);

/* The marking and splitting step of pff_refine_axes on host arrays, without a
 * problem or a device: for callers that form the slab quantities themselves.
 * Per axis a (dim of them): coords[a] (n_cells[a] + 1 strictly increasing
 * values), slab_eta2[a] and slab_minphi[a] (n_cells[a] values each); outputs
 * as for pff_refine_axes.  All arrays host, caller-owned. */
int pff_mark_axes(int dim, const int32_t* n_cells, const double* const* coords,
                  const double* const* slab_eta2, const double* const* slab_minphi, double theta,
                  double h_band, double phi_band, int32_t* n_cells_out, double* const* coords_out);

/* Move nodal fields of src onto the nodes of dst by Q1 interpolation (the
 * finite element function of src evaluated at dst's nodes; each value is the
 * corner sum of prod(t or 1 - t) times the corner values, in corner order,
 * rounded product by product).  dst's box must lie inside src's; both problems
 * must have the same dimension.  fields: any of the flags below.  With
 * PFF_FIELD_PHI_OLD, dst also takes src's count of finished loading steps (the
 * phi~ extrapolation).  Clears dst's assembled operators and preconditioner.
 * Synchronizes both streams. */
#define PFF_FIELD_U 1
#define PFF_FIELD_PHI 2
#define PFF_FIELD_PHI_OLD 4
#define PFF_FIELD_PHI_PREV 8
int pff_transfer_state(pff_problem* src, pff_problem* dst, int fields);

/* Allocation-free TCV / COD ------------------------------------------------ */

/* The paper has no counterpart of this entry point.  It exists for callers
 * that cannot let a library allocate device memory: an application whose
 * device memory is all handed out by its own pool allocator, or that reserved
 * the whole GPU up front, would see an unplanned cudaMalloc fail or upset its
 * own accounting.  pff_eval_tcv_cod allocates a small buffer for the COD line
 * descriptors on every call; this variant does not.
 *
 * Same results as pff_eval_tcv_cod (same kernels, same arguments and
 * layouts), but all scratch memory (COD line descriptors, per-line integrals,
 * TCV partial sums) lives in one fixed array of the library (about 200 KB,
 * declared with __device__ storage) that every GPU using the library holds
 * until the process exits; nothing is allocated with cudaMalloc, cudaFree or
 * any allocating library routine.  At most PFF_NOALLOC_MAX_POINTS COD points
 * per call: larger n_pts returns PFF_ERR_CAPACITY without doing any work.
 * The call synchronizes the problem's stream before it returns: tcv and cod
 * are ordinary (pageable) host memory that holds the results on return.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, checked) with that device current.  Every call on a
 * device shares the one array and it keeps the last call's contents: calls
 * whose work overlaps on the GPU (several problems or threads on different
 * streams at once) race and must be serialized by the caller.  No part of the
 * array needs to start at zero: each slot a call reads was written earlier in
 * the same call. */
#define PFF_NOALLOC_MAX_POINTS 1024
int pff_eval_tcv_cod_noalloc(pff_problem* prob, int n_pts, const double* pts, double* tcv,
                             double* cod);

/* Batched solves (many independent problems) ------------------------------
 * The paper solves one problem at a time; these entry points have no
 * counterpart there.  They exist because small instances (a few thousand to a
 * few hundred thousand DoFs) leave most of the GPU idle: their kernels are
 * launch- and latency-bound.  Running many of them at once lets their kernels
 * overlap on the device.
 *
 * pff_batch_solve solves the loading-step schedules of n independent problems
 * with n_workers host threads (0: one per problem, at most 16).  Each worker
 * owns a non-blocking CUDA stream; it takes the next unsolved problem (largest
 * first), moves it onto its stream for the duration of the call (the
 * problem's own stream is restored afterwards) and solves it exactly as
 * pff_solve_loading_steps would, so every problem reaches the result it reaches
 * alone, up to the summation order of the autotuned sparse kernels.
 * problems[i] must be distinct.  n_steps[i] pressures are read from
 * schedules[i] (host); reports[i] (host, caller-owned, n_steps[i] entries) and
 * status[i] (may be NULL) receive the outcome of problem i.  Returns PFF_OK when
 * every problem converged, else the first nonzero status (all problems are
 * still attempted). */
int pff_batch_solve(int n, pff_problem* const* problems, const int* n_steps,
                    const double* const* schedules, const pff_options* opts,
                    pff_step_report* const* reports, int n_workers, int* status);

/* Request server (continuous batching) --------------------------------------
 * Also without counterpart in the paper.  A server owns n_workers host
 * threads and streams and a device-memory budget.  Submitted requests wait in
 * FIFO order; the head of the queue is admitted as soon as a worker is free and
 * its memory estimate (pff_request_bytes) fits into what the running requests
 * leave of the budget (a request larger than the whole budget is admitted
 * alone).  An admitted request builds its problem on the worker's stream,
 * solves its pressure schedule, evaluates TCV and the requested COD points,
 * optionally copies its solution to the host, and frees its device memory;
 * requests that arrive meanwhile are admitted as memory and workers free up,
 * so the kernels of all running requests overlap on the GPU. */
typedef struct pff_server pff_server;

typedef struct pff_request {
  int dim;                        /* 2 or 3 */
  int32_t n_cells[3];             /* cells per axis */
  const double* axis_coords[3];   /* host, n_cells[a] + 1 increasing values each; copied */
  double E, nu, Gc, kappa, eps;   /* material (pff_set_material) */
  double l0;                      /* crack half-length (2d) / radius (3d) (pff_set_crack) */
  int n_steps;                    /* loading steps */
  const double* schedule;         /* host, n_steps pressures; copied */
  int n_cod;                      /* COD lines, may be 0 */
  const double* cod_x;            /* host, n_cod abscissae x; copied.  Each gives one COD
                                     line: along y at x (2d), along z at (x, y = 0) (3d) */
  int keep_solution;              /* 1: keep u, phi, active on the host (pff_server_solution) */
  int reserved;
} pff_request;

typedef struct pff_request_result {
  int status;            /* PFF_OK or the error code of the request */
  int done;              /* 1 once finished (successfully or not) */
  int newton_its;        /* summed over the loading steps */
  int krylov_its;        /* summed over the loading steps */
  int converged_steps;   /* loading steps that met the stopping test */
  int reserved;
  int64_t n_dofs;
  int64_t bytes;         /* admission estimate */
  double t_submit;       /* seconds since the server was created */
  double t_admit;
  double t_finish;
  double tcv;
} pff_request_result;

typedef struct pff_server_stats {
  int64_t budget_bytes;
  int64_t reserved_bytes;       /* estimates of the running requests */
  int64_t peak_reserved_bytes;  /* never above the budget unless one request exceeds it alone */
  int queued, running, finished;
  int max_running;              /* most requests running at once */
} pff_server_stats;

/* Device bytes reserved for a problem of this size by the admission test. */
int64_t pff_request_bytes(int dim, const int32_t* n_cells);

int pff_server_create(int64_t budget_bytes, int n_workers, const pff_options* opts,
                      pff_server** out);
/* Queue a request (its arrays are copied); *id identifies it. */
int pff_server_submit(pff_server* srv, const pff_request* req, int64_t* id);
/* Non-blocking state of a request (res->done = 0 while queued or running). */
int pff_server_result(pff_server* srv, int64_t id, pff_request_result* res);
/* Wait up to timeout_s seconds (< 0: no limit) for a request to finish;
 * PFF_ERR_TIMEOUT if it has not. */
int pff_server_wait(pff_server* srv, int64_t id, double timeout_s, pff_request_result* res);
/* COD values of a finished request (n_cod doubles, host). */
int pff_server_cod(pff_server* srv, int64_t id, double* cod);
/* Solution of a finished request submitted with keep_solution = 1 (host
 * buffers as for pff_get_solution; any may be NULL). */
int pff_server_solution(pff_server* srv, int64_t id, double* u, double* phi, uint8_t* active);
/* Forget a finished request (its host copies are freed). */
int pff_server_release(pff_server* srv, int64_t id);
int pff_server_stats_get(pff_server* srv, pff_server_stats* st);
/* Stop admitting, drop queued requests, wait for the running ones, free all. */
void pff_server_destroy(pff_server* srv);

/* Instrumentation (process-wide, all problems) ----------------------------- */

/* Enable (1) or disable (0) per-kernel timing and reset its totals.  When
 * enabled, each instrumented launch records a CUDA event pair on its stream
 * and is credited with its algorithmic bytes (every input and output array
 * moved once).  Adds a few microseconds per launch. */
int pff_profile_enable(int on);

/* Autotuner choices (sparse-kernel formats of the AMG hierarchy, element-kernel
 * tiles, Jacobian apply variant) are timed with CUDA events at first use.  With
 * the environment variable PFF_TUNE_CACHE naming a file, every choice is also
 * written there and choices found there are reused without timing, so a run under
 * a profiler (whose serialised, instrumented launches make such timings
 * meaningless) executes the kernels of the plain run that wrote the file. */

/* Restrict the timing to launches of the named kernels (as reported by
 * pff_profile_report; several names separated by commas); NULL times every
 * instrumented launch again.  Timing a few kernels keeps the event overhead
 * off the rest of the run.  The replays of a captured coarse-level graph
 * ("coarse_levels_graph_u" / "_phi") are credited with the summed algorithmic
 * bytes of the kernels captured in them. */
int pff_profile_select(const char* name);

/* Synchronize the device and write per-kernel totals as a JSON object
 * {"name": {"count": launches, "ms": total time, "bytes": algorithmic bytes}}
 * into buf (NUL-terminated, truncated to buflen).  Returns the length needed
 * including the NUL. */
int pff_profile_report(char* buf, int buflen);

/* Number of kernels launched by the library since it was loaded. */
long long pff_launch_count(void);

/* Device bytes the library holds now and at most since the last reset (all
 * problems and servers of the process; reset_peak = 1 restarts the peak from
 * the current value). */
int pff_memory_usage(int64_t* current, int64_t* peak, int reset_peak);

#ifdef __cplusplus
}
#endif
#endif /* PFF_H */
