/*
 * npfem.h - C ABI of the B300 npFEM batched deformable-body step.
 *
 * What the library computes (paper: Palabos-npFEM, arXiv 2011.04332)
 * ------------------------------------------------------------------
 * One implicit time step of npFEM - the mass-lumped linear finite-element solver
 * for triangulated cell membranes (Introduction) - for a batch of independent
 * red blood cells and platelets.  The step advances every cell from (x_n, v_n)
 * under per-vertex external forces to (x_{n+1}, v_{n+1}); in the coupled code
 * these forces come from the immersed-boundary coupling and the positions and
 * velocities go back to the fluid (Implementation and architecture section).
 * The step minimises the implicit-Euler objective of Eq. (2)
 *     f(x) = (x-y)^T M (x-y)/(2 dt^2) + sum_t E_t + sum_e E_e + E_A + E_V,
 *     y    = x_n + dt v_n + dt^2 M^-1 f_ext,
 * with the quasi-Newton projective-dynamics iteration the paper adopts from Liu
 * et al. 2017 (Implementation and architecture, first bullet): L-BFGS with
 * history 5 whose initial inverse Hessian is the prefactored projective-dynamics
 * matrix A = M/dt^2 + sum_t w_t G_t^T G_t + sum_e w_e c_e c_e^T (one Cholesky
 * factor per cell type), plus a backtracking line search.  The elemental
 * energies (per-triangle strain, per-hinge bending, global area and volume) are
 * the per-element energies with weights of the material file (Setting up new
 * materials section).
 *
 * Units: um, us, pg (force nN, energy nN*um, weights nN/um).
 *
 * Conventions
 * -----------
 * - Status codes: 0 = OK, negative = error (see NPFEM_ERR_*).  Errors of
 *   arguments or setup are returned synchronously; the message is available
 *   from npfem_last_error_string().  Per-cell numerical outcomes of a step are
 *   written to the device array status_out as bit flags (NPFEM_CELL_*); device
 *   code never traps.
 * - State layout is structure-of-arrays, coordinate-major: x[c*N_total + k] is
 *   coordinate c (0=x,1=y,2=z) of global vertex k; the vertices of cell i are
 *   k in [offset_i, offset_{i+1}) in batch order, each cell's vertices in its
 *   type's mesh order.
 * - Ownership: the caller owns every state array (device memory for
 *   npfem_step, host memory for npfem_step_host).  The library owns cell types,
 *   batches and their device workspace.  Types are immutable after creation and
 *   may be shared by several batches; a type must outlive its batches.
 * - Streams: npfem_step and npfem_step_adjoint are asynchronous on the given
 *   stream (0 = legacy default stream) and perform no host synchronisation, so
 *   they can be captured into a CUDA graph.  A batch must not be used on two
 *   streams at the same time (its workspace is shared by its calls).
 */
#ifndef NPFEM_H
#define NPFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int npfem_status;

#define NPFEM_OK 0
#define NPFEM_ERR_INVALID_ARG (-1)  /* null pointer, bad size or enum */
#define NPFEM_ERR_BAD_MESH (-2)     /* open / non-manifold mesh or degenerate rest triangle */
#define NPFEM_ERR_NOT_SPD (-3)      /* global matrix not positive definite (e.g. negative weight) */
#define NPFEM_ERR_CUDA (-4)         /* a CUDA runtime call failed */
#define NPFEM_ERR_OOM (-5)          /* device or host allocation failed */
#define NPFEM_ERR_UNSUPPORTED (-6)  /* size beyond a compiled limit */

/* Per-cell status bits written by a step (device array status_out). */
#define NPFEM_CELL_OK 0
#define NPFEM_CELL_LINESEARCH_FAIL 1  /* no acceptable step after 20 halvings (last trial kept) */
#define NPFEM_CELL_DEGENERATE 2       /* a triangle collapsed (det F^T F <= 1e-30) */
#define NPFEM_CELL_NONFINITE 4        /* NaN/Inf in the result */
#define NPFEM_CELL_ITER_LIMIT 8       /* iteration count above the supported bound (adjoint: 16;
                                         split step: opts->max_iters); the cell stopped there */
#define NPFEM_CELL_CG_NOT_CONVERGED 16 /* implicit adjoint: CG stopped before its tolerance */

typedef enum { NPFEM_FP64 = 0, NPFEM_FP32FORM = 1 } npfem_precision;

/* Closed, consistently outward-oriented triangle mesh of a cell type at rest
 * (host memory, read during the call only). */
typedef struct {
  int32_t n_verts;
  int32_t n_tris;
  const double* rest_xyz; /* [n_verts][3] rest positions, um */
  const int32_t* tris;    /* [n_tris][3] vertex indices, counter-clockwise seen from outside */
} npfem_mesh;

/* Per-type material: the weights of the per-element energies. */
typedef struct {
  double w_strain; /* nN/um: E_t = w_strain*A_t/2 |F - R(F)|^2 per triangle (A_t rest area) */
  double w_bend;   /* nN*um: E_e = w_bend*3/(A_A+A_B)/2 |K - |K0| K/|K||^2 per interior edge */
  double w_area;   /* nN/um: E_A = w_area/2 (A - A0)^2 / A0 */
  double w_vol;    /* nN/um^2: E_V = w_vol/2 (V - V0)^2 / V0 */
  double density;  /* pg/um^3: cell mass density*V0, lumped by vertex area share */
  /* Viscoelastic (Rayleigh) damping, C = c_alpha M + c_beta L with M the lumped mass
   * matrix and L = A - M/dt^2 the elastic part of the projective-dynamics matrix.  The
   * paper sets the bodies' viscous behaviour with two parameters, Calpha and Cbeta
   * (Setting up new materials section), without a formula; here the implicit step
   * minimises f(x) + (x - x_n)^T C (x - x_n) / (2 dt) per coordinate, i.e. implicit Euler
   * for M a + C v + grad E = f, and the prefactored matrix becomes
   * (1/dt^2 + c_alpha/dt) M + (1 + c_beta/dt) L.  Both 0: no damping. */
  double c_alpha;  /* 1/us, >= 0 */
  double c_beta;   /* us, >= 0 */
  /* Strain limits: the membrane-strain constraint set of a triangle is the set of
   * deformation gradients whose singular values lie in [s_min, s_max] (ShapeOp-style
   * strain limiting; the solver's origin, Implementation and architecture section), so
   * R(F) = U clamp(Sigma, s_min, s_max) V^T for F = U Sigma V^T.  Both 0 (or both 1):
   * the rotations, R = F (F^T F)^(-1/2).  Otherwise 0 < s_min <= 1 <= s_max, finite
   * (the rest shape lies in the set); else INVALID_ARG.  The adjoints differentiate
   * the clamped projection (by regime: both singular values inside the limits, both
   * clamped to one limit, or one on each side). */
  double s_min;
  double s_max;
} npfem_material;

typedef struct {
  int32_t iters;           /* quasi-Newton iterations per cell when iters array is NULL */
  int32_t alpha_log_len;   /* entries per cell in alpha_log (0 = no log) */
  double* alpha_log;       /* device [ncells][alpha_log_len] accepted step lengths, or NULL */
  int32_t max_iters;       /* upper bound of the per-cell counts of an iters array (split mode
                              launches that many iterations; 0 = unknown: fused mode) */
  double tol;              /* converged-residual mode (the solver run towards a converged
                              solution, Implementation and architecture section): > 0 ends a
                              cell's step after the first iteration whose gradient norm is below
                              tol * |grad f(x_0)|, compared in FP64; the iteration count is then
                              a budget.  0 = fixed counts.  Must be finite and >= 0. */
  int32_t* iters_done;     /* out [ncells] iterations each cell ran, or NULL: device memory for
                              npfem_step / npfem_step_noalloc, host memory for npfem_step_host */
} npfem_solver_opts;

typedef struct npfem_cell_type npfem_cell_type;
typedef struct npfem_batch npfem_batch;

/* Sizes and factor statistics of a cell type (host-side query). */
typedef struct {
  int32_t n_verts, n_tris, n_hinges;
  int64_t nnz_factor;      /* off-diagonal nonzeros of the unit lower factor */
  int64_t solve_chunks;    /* 32-entry chunks per triangular solve */
  double rest_area, rest_volume, total_mass;
  /* colour classes of the triangles and of the hinges (no two elements of a class share a
   * vertex; the CTA iteration kernels visit them class by class), 0 when the mesh needs
   * more than 64 (the type then runs the one-warp iteration kernels) */
  int32_t tri_colours, hinge_colours;
} npfem_type_info;

/* Build a cell type once: rest geometry, lumped masses, the global matrix A and
 * its FP64 Cholesky factor (fill-reducing ordering, A = P^T L D L^T P), uploaded to
 * the current CUDA device.  dt in us.  *out is owned by the caller and released
 * with npfem_destroy_cell_type.  Errors: INVALID_ARG, BAD_MESH, NOT_SPD, CUDA, OOM. */
npfem_status npfem_create_cell_type(const npfem_mesh* mesh, const npfem_material* mat,
                                    double dt, npfem_cell_type** out);
npfem_status npfem_destroy_cell_type(npfem_cell_type* type);
/* Host-only dry run of npfem_create_cell_type: validates the mesh and material,
 * builds and factors the global matrix on the host and fills *info, without touching
 * any GPU.  Same error codes as npfem_create_cell_type (except CUDA/OOM). */
npfem_status npfem_cell_type_analyze(const npfem_mesh* mesh, const npfem_material* mat, double dt,
                                     npfem_type_info* info);

npfem_status npfem_cell_type_info(const npfem_cell_type* type, npfem_type_info* info);

/* Group cells into a batch: cell i has type types[type_of_cell[i]] (host arrays,
 * read during the call).  Computes vertex offsets, per-type work queues and the
 * launch shape, and allocates the device workspace.  Errors: INVALID_ARG, CUDA, OOM. */
npfem_status npfem_batch_create(const npfem_cell_type* const* types, int32_t ntypes,
                                const int32_t* type_of_cell, int32_t ncells,
                                npfem_precision prec, npfem_batch** out);
npfem_status npfem_batch_destroy(npfem_batch* batch);
/* Total vertex count N_total and the vertex offsets [ncells+1] (host copy). */
npfem_status npfem_batch_layout(const npfem_batch* batch, int64_t* n_total, int64_t* offsets);

/* One time step for every cell of the batch (device memory, caller-owned).
 *   x, v  in/out [3][N_total] positions (um) and velocities (um/us): double for
 *         NPFEM_FP64, float for NPFEM_FP32FORM; overwritten with x_{n+1}, v_{n+1}.
 *   f_ext in [3][N_total] external forces (nN), same type as x.
 *   iters in [ncells] int32 per-cell iteration counts (>= 0), or NULL to use opts->iters.
 *   residual_out out [ncells] |grad f(x_final)| / |grad f(x_0)| (FP64; 0 when grad f(x_0)
 *                is exactly zero), or NULL.
 *   status_out   out [ncells] NPFEM_CELL_* bit flags, or NULL.
 * With opts->tol > 0 a cell that meets the tolerance stops early and its remaining
 * iterations are skipped (split mode keeps launching up to the budget over the
 * shrinking list of cells still iterating).  The result of a cell that stops after k
 * iterations equals that of a fixed-count step of k iterations.
 * Asynchronous on `stream` (a cudaStream_t).  Errors: INVALID_ARG (also a negative or
 * non-finite tol), CUDA. */
npfem_status npfem_step(npfem_batch* batch, void* x, void* v, const void* f_ext,
                        const int32_t* iters, const npfem_solver_opts* opts,
                        double* residual_out, int32_t* status_out, void* stream);

/* Reverse mode of one step (FP64 batches only): given dL/dx_{n+1} and dL/dv_{n+1},
 * returns dL/dx_n, dL/dv_n, dL/df_ext and, per cell, dL/d(w_strain, w_bend, w_area,
 * w_vol) of its type's material.  The derivative is that of the unrolled
 * quasi-Newton iteration of npfem_step (Liu et al. 2017, the iteration named in the
 * paper's Implementation and architecture section) with its accepted line-search
 * step lengths held fixed; the forward step is recomputed from (x, v, f_ext).
 *   x, v, f_ext   in  [3][N_total] double: the state the step started from.
 *   iters         in  [ncells] int32 or NULL (opts->iters); at most 16 per cell.
 *   gx_next       in  [3][N_total] dL/dx_{n+1};  gv_next in [3][N_total] or NULL (zero).
 *   gx, gv, gf    out [3][N_total] (overwritten).
 *   gw            out [ncells][4] (overwritten).
 *   status_out    out [ncells] or NULL: 0, or 8 when a cell's iteration count exceeds 16.
 * The first call on a batch allocates its adjoint workspace (about 2 MB per warp
 * slot for a 642-vertex type).  Asynchronous on `stream`.
 * opts->tol must be 0 (the adjoint differentiates fixed iteration counts); opts->iters_done
 * is ignored.  With Rayleigh damping the dissipation term of every iterate's gradient
 * depends on x_n directly, and the matrix weight terms carry the (1 + c_beta/dt) factor.
 * Errors: INVALID_ARG (null pointer, FP32-form batch, tol != 0, collisions on), CUDA, OOM. */
npfem_status npfem_step_adjoint(npfem_batch* batch, const void* x, const void* v, const void* f_ext,
                                const int32_t* iters, const npfem_solver_opts* opts,
                                const double* gx_next, const double* gv_next, double* gx, double* gv,
                                double* gf, double* gw, int32_t* status_out, void* stream);

/* Reverse mode of a whole rollout of `nsteps` steps with constant external forces (FP64
 * batches): the membrane-calibration use of the adjoint (Setting up new materials
 * section: a material's per-element weights; the derivative is that of the unrolled
 * quasi-Newton iteration of npfem_step, Implementation and architecture section).
 * Starting from (x0, v0), the library runs the forward rollout, keeping (x, v) before
 * every ckpt_every-th step, then sweeps the segments backwards: each segment's states
 * are recomputed from its checkpoint and the step adjoints (npfem_step_adjoint) run in
 * reverse.  Memory grows with nsteps/ckpt_every + ckpt_every states, not nsteps.
 *   x0, v0, f_ext   in  [3][N_total] double: initial state and the forces of every step.
 *   iters, opts     as in npfem_step_adjoint (fixed counts, at most 16, tol 0).
 *   nsteps >= 1, ckpt_every >= 1.
 *   gx_end          in  [3][N_total] dL/dx_N;  gv_end in [3][N_total] dL/dv_N or NULL (zero).
 *   gx0, gv0, gf    out [3][N_total] dL/dx0, dL/dv0, dL/df_ext (the sum over all steps).
 *   gweights        out [ntypes][4] dL/d(w_strain, w_bend, w_area, w_vol) of each cell type
 *                   (summed over its cells and all steps in a fixed order: reproducible).
 *   status_out      out [ncells] or NULL: the OR of every forward step's and every step
 *                   adjoint's NPFEM_CELL_* bits.
 * The library owns the workspace (checkpoints, segment states, gradient buffers; about
 * (2 nsteps/ckpt_every + 2 ckpt_every + 7) x 24 N_total bytes), allocated on the first
 * call and grown when a later call needs more.  Asynchronous on `stream`.  Errors:
 * INVALID_ARG (null pointer, FP32-form batch, nsteps or ckpt_every < 1, tol != 0,
 * collisions on), CUDA, OOM. */
npfem_status npfem_rollout_adjoint(npfem_batch* batch, const double* x0, const double* v0, const double* f_ext,
                                   const int32_t* iters, const npfem_solver_opts* opts, int32_t nsteps,
                                   int32_t ckpt_every, const double* gx_end, const double* gv_end, double* gx0,
                                   double* gv0, double* gf, double* gweights, int32_t* status_out, void* stream);

/* Gradients through the CONVERGED step (FP64 batches): the solver run to convergence
 * (Implementation and architecture section) differentiated by the implicit-function
 * theorem instead of through the unrolled iteration.  The forward step is run here,
 * with the batch's mode, on internal copies of x and v (iters, opts as in npfem_step;
 * opts->tol > 0 and a generous budget make it converge); then, with x* its result,
 * H = grad^2 f(x*) and v* = (x* - x_n)/dt, each cell solves
 *   H lam = gx_next + gv_next / dt
 * by conjugate gradients preconditioned with the prefactored matrix A^-1, and returns
 *   gx = (M/dt^2) lam - gv_next/dt,  gv = (M/dt) lam,  gf = lam,
 *   gw[cell][q] = -lam . d(grad f)/d(w_q) for (w_strain, w_bend, w_area, w_vol).
 * The gradients are exact for the minimiser; for an unconverged x* they are those of
 * the minimiser's linearisation at x*.
 *   cg_tol       stop when |residual| <= cg_tol |gx_next + gv_next/dt| (finite, > 0)
 *   cg_max_iters at most this many CG iterations per cell (>= 1)
 *   status_out   out [ncells] or NULL: the forward step's flags, with 16 ORed in where CG
 *                stopped before cg_tol (budget used, or H not positive along a direction).
 * With Rayleigh damping (c_alpha, c_beta of a type) the dissipation term is part of f: it
 * enters H and the weight derivatives, and since it depends on x_n directly,
 * gx gains C lam / dt.
 * Arrays as in npfem_step_adjoint.  The first call allocates two [3][N_total] FP64 copies
 * and the adjoint workspace.  Asynchronous on `stream`.  Errors: INVALID_ARG (null
 * pointer, FP32-form batch, bad cg_tol / cg_max_iters, collisions on), CUDA, OOM. */
npfem_status npfem_step_adjoint_implicit(npfem_batch* batch, const void* x, const void* v, const void* f_ext,
                                         const int32_t* iters, const npfem_solver_opts* opts,
                                         const double* gx_next, const double* gv_next, double* gx, double* gv,
                                         double* gf, double* gw, double cg_tol, int32_t cg_max_iters,
                                         int32_t* status_out, void* stream);

/* Launch shape of the cells of one type (the autotuner's knobs): warps per CTA
 * (1..4; one warp advances one cell), CTAs per SM (1..16), whether each warp's FP64
 * solve vector lives in shared memory (1) or in the workspace (0), and whether the
 * three coordinates share each triangular sweep (solve_per_coord = 0, vector of
 * 24*(n+1) bytes) or are swept one after another (1, vector of 8*(n+1) bytes; applies
 * to a vector in shared memory only: one in the workspace is always swept whole).
 * The adjoints use the shape's warp slots and solve placement too: the unrolled adjoint
 * runs a CTA of four warps per cell over them (one slot each), the implicit adjoint one
 * warp per cell.  Results do not depend on the shape.  Reallocates that type's workspace; synchronises
 * the device.  Default: 4 warps, 3 CTAs/SM, shared memory when four interleaved
 * vectors fit in 72 KB.  Errors: INVALID_ARG, UNSUPPORTED (vectors exceed shared
 * memory), OOM.  npfem_batch_get_launch fills shape[5] = {warps per CTA, CTAs per SM,
 * solve in shared memory, per-coordinate solve, grid size}. */
npfem_status npfem_batch_set_launch(npfem_batch* batch, int32_t type_index, int32_t warps_per_block,
                                    int32_t blocks_per_sm, int32_t solve_in_shared, int32_t solve_per_coord);
npfem_status npfem_batch_get_launch(const npfem_batch* batch, int32_t type_index, int32_t* shape);

/* Execution mode of npfem_step for a batch.  mode 1 (default, "split"): per cell type
 * one kernel for the prediction and first evaluation, then per iteration one kernel for
 * the FP64 global solves and one for the rest of the iteration (all asynchronous on the
 * stream; needs the iteration bound: opts->iters without an iters array, else
 * opts->max_iters in 1..32; a cell whose count exceeds it stops there and gets status
 * bit 8).  mode 0 ("fused"): one persistent kernel per cell type (any iteration count;
 * also used by split-mode batches when the bound is unknown).  The two modes agree to
 * rounding (their kernels are compiled separately and the compiler may contract
 * multiply-adds differently).  Split launch shapes do not change split-mode results,
 * except that placement 2 applies the factor updates in another (equally exact) order:
 * its results agree with the others to FP64 rounding.
 * npfem_batch_set_split_launch sets, per type, shape[7] = {warps per CTA (1..4), CTAs per
 * SM (1..16) of the iteration kernels; warps per CTA (1..4; placement 2: 2, 4, 6 or 8),
 * CTAs per SM (1..16), placement of the FP64 solve vectors (0: each cell's workspace,
 * 1: shared memory, one per warp, 2: shared memory, one per CTA whose warps sweep the
 * cell together through a level packing of the factor), per-coordinate solve, cells per warp (1..4)
 * of the solve kernel: a warp sweeps that many cells of the type together through the
 * shared factor (placement 2: cells per CTA, 1, or 2 with 2 or 4 warps per CTA: each
 * factor entry updates both cells' vectors, with each cell's updates in the one-cell
 * order)};
 * NPFEM_ERR_INVALID_ARG outside those ranges, NPFEM_ERR_UNSUPPORTED when a CTA's solve
 * vectors exceed shared memory.  npfem_batch_get_split_launch returns those seven values
 * plus the mode in shape[7] (host array of 8). */
npfem_status npfem_batch_set_mode(npfem_batch* batch, int32_t mode);

/* Split mode: cut the cells of type type_index into `groups` (1..4) contiguous groups,
 * each with its own chain of kernels on its own stream, running concurrently: the
 * chains fill each other's wave tails and one group's FP32 iteration kernel overlaps
 * another group's FP64 solve.  Default: 4 groups for types with at least 4096 cells in
 * the batch, 2 from 2048, else 1; in an FP32-form batch of one cell type (no other
 * type's chains to overlap with) 4 from 1024 cells, 2 from 512.  Results do not depend on
 * the grouping.
 * NPFEM_ERR_INVALID_ARG for groups outside 1..4 or a type without cells in the batch. */
npfem_status npfem_batch_set_groups(npfem_batch* batch, int32_t type_index, int32_t groups);

/* Split mode with several chains (cell types or groups): enable != 0 launches every
 * chain's FP64 solves on a stream of their own at the highest stream priority, the rest
 * of the chain at the lowest, ordered by events (so pending solve CTAs take SM slots
 * first as they free up).  Default on in the FP32 form, off in FP64 (whose iteration
 * kernels need the FP64 pipe as much); enable = 0 keeps each chain on one stream.
 * Results do not change.  The streams are created on the next uncaptured step.
 * Synchronises the device. */
npfem_status npfem_batch_set_solve_streams(npfem_batch* batch, int32_t enable);
npfem_status npfem_batch_get_groups(const npfem_batch* batch, int32_t type_index, int32_t* groups);

/* Split mode: iteration kernels of type type_index (the prediction with the first
 * objective evaluation, and the rest of each iteration around the FP64 solve).
 * warps in 1, 2, 4, 8, 16 (default in the FP32 form: 2 for up to 256 vertices, 4 up to 1024, else 8; in the FP64
 * form 0, whose objective is bound by the FP64 pipe rather than by gathers): one CTA of that
 * many warps per cell, the cell's start positions, trial displacement and gradient in
 * shared memory during each objective evaluation (9n values: 23 KB for a 642-vertex FP32
 * cell), triangles and hinges visited by colour classes whose elements share no vertex
 * (Implementation and architecture section: the per-element local step with the gradient
 * assembled per vertex), CTA-wide sums.  warps = 0: one warp per cell with per-element
 * records in the workspace and a per-vertex gather.  The width sets the order of a cell's
 * sums: results of different widths agree to rounding; for a given width they do not
 * depend on any other launch setting.  NPFEM_ERR_INVALID_ARG for warps not among 0, 1, 2,
 * 4, 8, 16 or a type without cells in the batch; NPFEM_ERR_UNSUPPORTED when the shared-memory arrays
 * exceed a CTA or the type needs more than 64 colour classes (the setting is then left as
 * it was; a new batch falls back to warps = 0 in those cases).  npfem_batch_get_iter_width
 * returns the width and, when ctas_per_sm is not null, the CTAs per SM that are resident
 * at that width (0 with warps = 0). */
npfem_status npfem_batch_set_iter_width(npfem_batch* batch, int32_t type_index, int32_t warps);
npfem_status npfem_batch_get_iter_width(const npfem_batch* batch, int32_t type_index, int32_t* warps,
                                        int32_t* ctas_per_sm);
npfem_status npfem_batch_set_split_launch(npfem_batch* batch, int32_t type_index, const int32_t* shape);
npfem_status npfem_batch_get_split_launch(const npfem_batch* batch, int32_t type_index, int32_t* shape);

/* Per-phase telemetry of the batch's steps since creation or the last reset, counted
 * only while npfem_batch_set_phase_counting(batch, 1) is in effect (off by default: the
 * kernels then skip the per-phase atomics): SM clock cycles summed over all warps (the
 * CTA iteration kernels: over CTAs), in the order prediction, objective evaluation,
 * two-loop recursion, global FP64 solve, history update, write-back, and (contained in
 * the objective) the area/volume pass and the gradient assembly (gather, or the colour
 * passes of the CTA kernels).  npfem_batch_phase_cycles synchronises the device;
 * cycles: host array of 8; reset != 0 zeroes the counters after reading. */
npfem_status npfem_batch_set_phase_counting(npfem_batch* batch, int32_t enable);
npfem_status npfem_batch_phase_cycles(npfem_batch* batch, uint64_t* cycles, int32_t reset);

/* Per-kernel timing of split-mode steps with CUDA events recorded on the stream each
 * kernel is launched on (a per-type internal stream when the batch holds several
 * types).  enable != 0 creates the events (once) and makes every later split-mode step
 * record a start/end pair around each of its launches; under stream capture the pairs
 * become event-record nodes that each graph replay re-records.  npfem_batch_kernel_times
 * waits for the last recorded step of cell type type_index and returns, in host arrays
 * of 3, the summed durations in ms and launch counts of {k_begin, k_solve, k_iter}.
 * Errors: NPFEM_ERR_INVALID_ARG when timing was never enabled or the type has no cells;
 * NPFEM_ERR_CUDA when an event cannot be read. */
npfem_status npfem_batch_set_kernel_timing(npfem_batch* batch, int32_t enable);
npfem_status npfem_batch_kernel_times(npfem_batch* batch, int32_t type_index, double* ms, int32_t* launches);
/* The same launches as time spans: for each of {k_begin, k_solve, k_iter}, the length in
 * ms of the union of the launch intervals of the last timed step (concurrent chains of
 * the type -- or, for type_index = -1, of all types -- overlap, so the union is the time
 * during which at least one such kernel was running).  span_ms: host array of 3. */
npfem_status npfem_batch_kernel_spans(npfem_batch* batch, int32_t type_index, double* span_ms);

/* Collisions.  The paper names collision detection and collision forces among the
 * coupled code's work (Performance figure, "Other"), a collision weight (Collision at
 * an obstacle section), and a fluid-free cell-packing application in which npFEM with
 * collisions resolves the overlaps of cells placed at random (Cell Packing section); it
 * gives no formula.  The reading implemented here: at the start of every step, each
 * vertex i of cell a is matched with the nearest vertex j of each other cell b closer
 * than `radius` (equal distances: the smaller j), and the two nearest such cells are
 * kept (equal distances: the smaller b).  Each match is a plane through x_j with normal
 * n_j, b's unit area-weighted outward vertex normal, both from the step's input state
 * and fixed during the step; the step objective gains, per match,
 * (weight/2) max(0, delta - (n_j . x_i - n_j . x_j))^2.  Distances are compared in FP64
 * (squared, evaluated as (dx*dx + dy*dy) + dz*dz).  Cells stay independent within a
 * step, so the step keeps its data-parallel structure. */
typedef struct {
  double radius; /* um: match search radius (also the detection grid's cell edge) */
  double delta;  /* um: contact thickness, >= 0 */
  double weight; /* nN/um: collision weight, >= 0 */
  int32_t walls; /* != 0: the faces of the box [box_lo, box_hi] act on every vertex of the
                    current iterate with (weight/2) max(0, delta - gap)^2 per face, gap the
                    distance inside the box along that face's axis (cell-wall contact) */
  double box_lo[3]; /* um, with walls: box corners, box_lo < box_hi on every axis */
  double box_hi[3];
} npfem_collision_params;

/* Enable collisions for every later npfem_step / npfem_step_host of the batch (params
 * != NULL) or disable them (NULL).  The first enable allocates the detection buffers
 * (about 170 bytes per vertex plus a hash table of 16 bytes per slot, the next power of
 * two >= N_total slots, at least 4096) and uploads the vertex-to-cell map (synchronous).
 * While enabled, each step first runs the detection kernels on its stream (captured
 * into graphs like the rest of the step); npfem_step_host then copies all inputs before
 * the step instead of overlapping chunks; npfem_step_adjoint returns INVALID_ARG
 * (contacts are not differentiated).  Errors: INVALID_ARG (null batch; radius not
 * finite and > 0; delta or weight negative or not finite), UNSUPPORTED (2^30 vertices or
 * more), CUDA / OOM. */
npfem_status npfem_batch_set_collisions(npfem_batch* batch, const npfem_collision_params* params);

/* The contacts found by the last step (device arrays, caller-owned, each NULL to skip),
 * asynchronous on `stream`:
 *   count  [N_total] int32 matches per vertex (0..2);
 *   vertex [N_total][2] int32 global index of the matched vertex j, nearest first, -1 unused;
 *   plane  [N_total][2][4] double: n_j, then n_j . (x_j - x_anchor), x_anchor the first
 *          vertex of the cell of vertex i (the vertex matched) at the step's input (zeros unused).
 * Errors: INVALID_ARG (null batch, collisions never enabled), CUDA. */
npfem_status npfem_batch_contacts(npfem_batch* batch, int32_t* count, int32_t* vertex, double* plane,
                                  void* stream);

/* With kernel timing on (npfem_batch_set_kernel_timing) and collisions on, every step
 * records a CUDA event pair around its detection kernels on the step's stream (event
 * records under stream capture, re-recorded by each replay).  This waits for the last
 * step's pair and returns the time between them in ms.  Errors: INVALID_ARG (null
 * argument; the last step ran without timing or without collisions), CUDA. */
npfem_status npfem_batch_contact_time(npfem_batch* batch, double* ms);

/* Same step with HOST arrays (pageable or pinned): copies x, v, f_ext (and iters,
 * when given) to batch-owned device buffers, runs the step, and copies x, v,
 * residuals, statuses (and opts->iters_done) back; synchronous.  residual_out,
 * status_out and opts->iters_done are host arrays or NULL.  In split mode the batch is cut into chunks of consecutive cells whose
 * copies in and out overlap the other chunks' kernels (pinned host memory lets the
 * copies run asynchronously); results equal those of npfem_step. */
npfem_status npfem_step_host(npfem_batch* batch, void* x, void* v, const void* f_ext,
                             const int32_t* iters, const npfem_solver_opts* opts,
                             double* residual_out, int32_t* status_out, void* stream);

/* Allocation-free step for callers that must not allocate device memory: code
 * running inside a framework whose pool owns all device memory, code called while a
 * stream is being captured, or tools with a device-memory budget fixed at start-up.
 * The paper has no counterpart; this is a library convenience.
 * Steps `ncells` cells of one type laid out back to back (cell i owns vertices
 * [i*n, (i+1)*n) of x, v, f_ext, each [3][ncells*n], same element types and
 * meaning as npfem_step).  It allocates nothing: its workspace is a 32 MiB static
 * device array reserved on every GPU that loads the library, held until exit.
 * Limits: ncells <= 65536, and the type's per-warp workspace must fit four warps
 * in the array (otherwise NPFEM_ERR_UNSUPPORTED with the sizes in the message).
 * Every call looks up the array's device address in the current device's context and
 * sets the kernels' shared-memory limit (neither allocates nor is cached, so calls after
 * a cudaDeviceReset work); the first call on a device also loads the library's kernels
 * there, so make that first call before any stream capture.
 * Every call reuses the same array (the work-queue counter is cleared on each call),
 * so calls whose GPU work overlaps (two streams, or two threads) race and must be
 * serialised by the caller.  Asynchronous on `stream`. */
npfem_status npfem_step_noalloc(const npfem_cell_type* type, npfem_precision prec, int32_t ncells,
                                void* x, void* v, const void* f_ext, const int32_t* iters,
                                const npfem_solver_opts* opts, double* residual_out,
                                int32_t* status_out, void* stream);

/* Message of the last error returned on the calling thread (empty if none). */
npfem_status npfem_last_error_string(char* buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* NPFEM_H */
