/*
 * amr4.h -- C ABI of the GB300-native fourth-order AMR elliptic solver.
 *
 * Method: Zhao & Zhang, "Fourth-order AMR both in space and in time for incompressible
 * Navier-Stokes equations with Dirichlet boundary conditions" (arXiv 2506.02663).
 * The library solves the paper's fourth-order finite-volume elliptic systems -- the
 * pure-Neumann pressure Poisson equation and the Helmholtz systems (I - gamma*nu*k*L) of
 * Eq. (GePUP-IMEX b) -- on a block-structured AMR hierarchy (Sec. 5) by geometric
 * multigrid (Sec. 6.5), with every step in hand-written sm_103a CUDA kernels.
 *
 * Conventions shared by every call
 * --------------------------------
 * Ownership.  The caller owns every field buffer and the stream.  The library owns the
 *   hierarchy metadata (host and device copies), multigrid scratch and bottom-solve
 *   factors; they are freed by the matching destroy call.
 * Memory.  Field pointers are DEVICE pointers (cudaMalloc'd or torch tensors) unless a
 *   call says otherwise.  ``stream`` is a cudaStream_t passed as void* (NULL = legacy
 *   default stream).  Calls are stream-ordered; a call that returns statistics or norms
 *   synchronises its stream before returning.
 * Errors.  Every call returns an amr_status; nothing crosses the ABI as an exception.
 *   Argument and geometry errors are detected on the host before any launch and leave the
 *   outputs untouched.  amr_last_error() returns a thread-local message for the last
 *   failing call of the calling thread.
 * Composite field layout.  A composite field is one contiguous array of doubles (or
 *   floats where a call says so) holding every box ("patch") of every level, levels in
 *   order, boxes in the order given at creation.  Patch p occupies
 *       [offset_p, offset_p + stride_z_p * (n_z + 4))        (3-D)
 *       [offset_p, offset_p + stride_y_p * (n_y + 4))        (2-D)
 *   and cell (i, j, k) of the box (0-based, x fastest) sits at
 *       offset_p + (k+2)*stride_z_p + (j+2)*stride_y_p + (i+2)
 *   i.e. every box is wrapped by the two ghost layers of Sec. 3 (paragraph after
 *   Eq. appProj).  amr_field_layout() returns the offsets and strides.  Values on the
 *   invalid region of a level (Eq. validRegion) are defined as the average of their
 *   children (Eq. AMR_avergingDownToCrse); calls that read a composite field overwrite
 *   them with that average first.
 * Boundary data layout.  Optional ``bc`` arrays hold, for every level l and face
 *   f = 2*d + side (side 0 = low, 1 = high), one value per cell of the domain's face at
 *   level l (the domain's cells with dimension d removed, lowest remaining dimension
 *   fastest), levels in order, faces in order.  Dirichlet data are face averages of the
 *   solution; Neumann data are face averages of its OUTWARD normal derivative
 *   (Eqs. velBCHomoDiri5th, Neumann5).  NULL means homogeneous data.
 *   amr_bc_layout() returns the offsets.
 */
#ifndef AMR4_H
#define AMR4_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AMR_OK = 0,
  AMR_ERR_INVALID_ARG = 1,   /* bad argument, layout or descriptor                      */
  AMR_ERR_NESTING = 2,       /* proper nesting violated (paragraph after Eq. pBlock)     */
  AMR_ERR_REFINEMENT = 3,    /* proper refinement violated (Eq. pBlock)                  */
  AMR_ERR_BOX_TOO_SMALL = 4, /* a box of level >= 1 has fewer than 4 cells in a dimension */
  AMR_ERR_NOT_CONVERGED = 5, /* max_vcycles reached above tolerance (stats still valid)   */
  AMR_ERR_NONFINITE = 6,     /* a residual norm became NaN or Inf                          */
  AMR_ERR_CUDA = 7,          /* a CUDA runtime call failed (message in amr_last_error)    */
  AMR_ERR_OOM = 8            /* device allocation failed                                  */
} amr_status;

typedef enum { AMR_BC_DIRICHLET = 0, AMR_BC_NEUMANN = 1 } amr_bc;
typedef enum { AMR_FP64 = 0, AMR_MIXED = 1 } amr_precision;

/* Hierarchy description (Eqs. grids, AMRHier).
 *   dim       2 or 3
 *   ratio     refinement ratio r (2; 4 is accepted by amr_hierarchy_create and the
 *             index maps, solver calls need 2)
 *   n0        cells of level 0 per dimension (>= 5); level l has n0 * r^l
 *   h0        cell size of level 0 (square cells)
 *   nlevels   number of levels (>= 1)
 *   nboxes    boxes per level (nboxes[0] must be 1: level 0 is the domain)
 *   boxes     for every box of every level in order: lo[0..dim-1], hi[0..dim-1],
 *             inclusive indices in that level's index space
 * Validation order (the first failing check is reported): dim/ratio/n0/level-0 box;
 * then every box of every level >= 1 in order: bounds (INVALID_ARG), >= 4 cells per
 * dimension (BOX_TOO_SMALL), lo and hi+1 divisible by r (REFINEMENT); then pairwise
 * disjointness per level (INVALID_ARG); then nesting for levels >= 2: C_r(box) grown by 3
 * coarse cells (clipped to the domain) inside level l-1 (NESTING); finally the coarsest
 * level-0 multigrid grid must have at most 1024 cells (INVALID_ARG). */
typedef struct {
  int dim;
  int ratio;
  int n0[3];
  double h0;
  int nlevels;
  const int* nboxes;
  const int* boxes;
} amr_hierarchy_desc;

typedef struct amr_hierarchy amr_hierarchy;
typedef struct amr_operator amr_operator;

typedef struct {
  int level;
  int box;          /* index of the box within its level */
  int lo[3], hi[3]; /* inclusive, level index space (unused dims 0) */
  long long offset; /* element offset of the padded patch in a composite field */
  long long stride_y, stride_z;
  long long nelems; /* elements occupied by the padded patch */
} amr_patch_info;

/* Index maps (host arrays owned by the hierarchy, valid until destroy).  They are the
 * bit-exact parity artefacts of Sec. 5.1 / Fig. 1(c):
 *   valid         one int per interior cell of every patch (patch order, x fastest):
 *                 1 valid, 0 invalid (Eq. validRegion)
 *   component     one int per box of every level: connected-component label of the box
 *                 within its level (boxes sharing a face patch of positive measure are
 *                 connected; label = smallest box index of the component)
 *   ghost_code    one int per padded cell of every patch (extents n+4 per dimension, x
 *                 fastest, no pitch padding): 0 interior, 1 physical, 2 copy from a box of
 *                 the same level, 3 AMRCFI, 4 unused (outside the box in >= 2 dims)
 *   ghost_src     same shape: physical -> face id 2d+side; copy -> source box index;
 *                 else -1
 *   ghost_aux     same shape: physical -> ghost layer (1 or 2); copy -> source cell's
 *                 interior linear index in the source box (x fastest); else -1
 *   ncfi          number of AMRCFI ghost cells; for each (ordered by padded-cell index
 *                 over all patches): cfi_cell (padded-cell index over all patches, in the
 *                 ghost_code numbering), cfi_start[dim] (global coarse index of the first
 *                 cell of the 5-cell window per dimension), cfi_pos[dim] (parent coarse
 *                 cell within the window, 0..4), cfi_sub[dim] (fine sub-cell, 0..r-1)
 *   nreflux       number of coarse valid cells with a coarse-fine face (COH-3); for each:
 *                 reflux_cell[3] = (level, box, interior linear index), reflux_faces =
 *                 bit (2d+side) set for every face of the cell that borders the invalid
 *                 region. */
typedef struct {
  long long ncells_interior;
  long long ncells_padded;
  const int* valid;
  const int* component;
  const int* ghost_code;
  const int* ghost_src;
  const int* ghost_aux;
  long long ncfi;
  const long long* cfi_cell;
  const int* cfi_start; /* ncfi * dim */
  const int* cfi_pos;   /* ncfi * dim */
  const int* cfi_sub;   /* ncfi * dim */
  long long nreflux;
  const int* reflux_cell;  /* nreflux * 3 */
  const int* reflux_faces; /* nreflux */
} amr_index_maps;

typedef struct {
  int nu1, nu2;      /* pre/post smoothing sweeps (4, 4: Fig. mg_convergenceRate)        */
  double omega;      /* weighted-Jacobi weight (2/3, Sec. 6.5)                           */
  double rtol, atol; /* stop when ||f - A phi||_inf,valid <= max(rtol*||f||_inf, atol)    */
  int max_vcycles;   /* hard cap on V-cycles (no unbounded device loop exists)            */
  int precision;     /* AMR_FP64, or AMR_MIXED: FP32 V-cycles inside FP64 refinement      */
  int zero_initial;  /* 1: start from phi = 0; 0: use phi as the initial guess            */
  int use_graph;     /* 1: capture the whole solve as one CUDA graph (device-side loop over
                        V-cycles, no host round trip per V-cycle) and replay it              */
  int fuse_coarse;   /* coarse end of the level-0 V-cycle.  0 (default): per-grid launches (in
                        2-D the one-block square coarse kernel where it applies).  1: one
                        shared-memory block from the largest grid that fits (generic per-cell
                        code).  2 (3-D): the grids of at most 32^3 cells as one launch of one
                        thread-block cluster, phases separated by cluster barriers, same
                        per-cell arithmetic as the per-grid kernels.  On GB300 both fused
                        forms are slower than captured per-grid launches.                   */
  int temporal_blocking; /* 1 (default): in forward FP32 V-cycles on 2-D level-0 multigrid grids,
                        each down leg (nu1 sweeps, residual, restriction) and each up leg
                        (prolongation, nu2 sweeps) is one launch over shared-memory tiles
                        with halos (same per-cell arithmetic); 0: one launch per sweep    */
  int cycles_per_refinement; /* mixed precision: FP32 V-cycles per FP64 residual (1..4; 1 by
                        default).  With c > 1 each refinement step runs c correction cycles,
                        the later ones on the FP32 composite residual of the correction so far
                        (in exact arithmetic the same iterate as c steps of one cycle each),
                        and pays for one FP64 residual, update and norm instead of c.  The
                        stopping test runs once per step: vcycles is a multiple of c (at most
                        max_vcycles + c - 1) and res_history holds one entry per step.  The
                        2-D work-list batch keeps one cycle per step; FP64 solves ignore it. */
} amr_solver_params;

typedef struct {
  int vcycles;          /* V-cycles performed                                   */
  double rhs_norm;      /* ||f||_inf over valid cells (after the solvability fix) */
  double final_res;     /* ||f - A phi||_inf over valid cells at exit             */
  double removed_mean;  /* pure Neumann: constant removed from f (Sec. 6.4)       */
  double res_history[64]; /* residual norm before each V-cycle (first 64)         */
} amr_solve_stats;

/* ---- hierarchy ------------------------------------------------------------------ */
amr_status amr_hierarchy_create(const amr_hierarchy_desc* desc, amr_hierarchy** out);
void amr_hierarchy_destroy(amr_hierarchy* h);
/* Number of patches, total elements of a composite field; ``patches`` (nullable) receives
 * npatches entries. */
amr_status amr_field_layout(const amr_hierarchy* h, int* npatches, long long* nelems,
                            amr_patch_info* patches);
/* offsets[l*2*dim + f] = element offset of face f of level l in a bc array;
 * offsets[nlevels*2*dim] = total length.  ``offsets`` needs nlevels*2*dim+1 entries. */
amr_status amr_bc_layout(const amr_hierarchy* h, long long* offsets);
amr_status amr_get_index_maps(const amr_hierarchy* h, amr_index_maps* out);

/* ---- operators -------------------------------------------------------------------- */
/* alpha*I + beta*L with boundary types bc_types[2*dim] (face f = 2d+side); the PPE is
 * alpha = 0, beta = 1 with all faces Neumann; the viscous systems alpha = 1,
 * beta = -gamma*nu*k (Eq. GePUP-IMEX b).  Precomputes the dense bottom-solve inverse
 * and allocates multigrid scratch.  Needs ratio 2. */
amr_status amr_operator_create(amr_hierarchy* h, double alpha, double beta, const int* bc_types,
                               amr_operator** out);
void amr_operator_destroy(amr_operator* op);

/* COH-1 on a composite field: average down (Eq. AMR_avergingDownToCrse), then fill the
 * stored ghost cells: copies from boxes of the same level and AMRCFI from the next coarser
 * level (Sec. 5.2).  Ghost cells outside the physical domain are never stored: every
 * kernel evaluates Eqs. (velBCHomoDiri5th)/(Neumann5) on the fly where a stencil leaves
 * the domain.  Unused corner ghosts are not written.  bc is accepted for symmetry and
 * not read. */
amr_status amr_fill_ghosts(amr_operator* op, double* phi, const double* bc, void* stream);

/* out = alpha*phi + beta*L^comp phi (COH-1..4, refluxing of Eq. cell2face fluxes). */
amr_status amr_apply(amr_operator* op, double* phi, double* out, const double* bc, void* stream);

/* res = f - A^comp phi on every covered cell (meaningful on valid cells);
 * *norm (host, nullable) = ||res||_inf over valid cells (synchronises). */
amr_status amr_residual(amr_operator* op, double* phi, const double* f, double* res,
                        const double* bc, double* norm, void* stream);

/* nsweeps weighted-Jacobi sweeps (true diagonal, homogeneous physical ghosts, zero CF
 * ghosts) of level ``level``'s operator on x for right-hand side b (both composite fields;
 * only that level is touched).  Kernel-level entry point of the smoother (Sec. 6.5). */
amr_status amr_smooth(amr_operator* op, int level, int nsweeps, double omega, double* x,
                      const double* b, void* stream);

/* One composite V-cycle (Sec. 6.5) in FP64 on phi for right-hand side f. */
amr_status amr_vcycle(amr_operator* op, const amr_solver_params* p, double* phi, const double* f,
                      const double* bc, void* stream);

/* V-cycles until the max-norm residual test of Sec. 7 passes.  Pure Neumann: f (const)
 * is corrected into an internal copy (Sec. 6.4) and phi is returned with zero h^D-weighted
 * mean over the valid cells.  stats (host, nullable). */
amr_status amr_solve(amr_operator* op, const amr_solver_params* p, double* phi, const double* f,
                     const double* bc, amr_solve_stats* stats, void* stream);

/* Sec. 6.4 for the composite PPE: f -= m on every valid cell with
 * m * sum_valid h^D = sum_valid h^D f - beta * sum_boundary h^(D-1) g (g = Neumann data in
 * bc, NULL = 0), compensated sums.  *m (host, nullable) receives m.  One component: level
 * 0 is the whole (connected) domain. */
amr_status amr_solvability_fix(amr_operator* op, double* f, const double* bc, double* m, void* stream);

/* phi -= (h^D-weighted mean over valid cells), compensated sums; *mean (nullable). */
amr_status amr_mean_zero(amr_hierarchy* h, double* phi, double* mean, void* stream);

/* Allocation-free variant of amr_mean_zero.  The paper has no counterpart: this exists for
 * callers that must not allocate device memory at the point of the call -- code running
 * while device memory is fully held by another allocator (a framework's caching pool), or
 * inside a timing- or latency-critical loop where cudaMalloc's implicit device-wide
 * synchronisation is not acceptable.  It launches exactly the kernels of amr_mean_zero with
 * the same launch shapes (average-down, the grid-stride compensated sums with at most 512
 * blocks per level, the fixed-order final sum, the shift), so the removed mean and the
 * result are bitwise those of amr_mean_zero; only its reduction scratch differs: a fixed
 * file-scope device array inside the library (8192 block partials plus a few scalars, about
 * 128 KiB per GPU that loads the library, held until the process exits) instead of
 * hierarchy-owned memory.  It calls no cudaMalloc, cudaFree or allocating library routine.
 *   - The hierarchy must already have its device copy (any earlier device call on it, e.g.
 *     amr_operator_create or amr_mean_zero, makes it); otherwise AMR_ERR_INVALID_ARG.
 *   - Hierarchies whose reduction needs more than 8192 blocks (more than 16 levels of at
 *     least 131,072 cells) are rejected with AMR_ERR_INVALID_ARG and a message giving the
 *     count; nothing is launched and phi is unchanged.  amr_mean_zero has the same limit.
 *   - The first call on a device looks up the array's device address with that device
 *     current (cudaGetSymbolAddress); make that first call before any stream capture.  A
 *     first call on a device whose stream is capturing is refused with AMR_ERR_INVALID_ARG.
 *   - Every call shares the one array and it keeps the last call's contents; each call
 *     writes every slot it reads before reading it.  Calls that overlap on the GPU (on
 *     different streams, or from different threads on the same device) race on the array
 *     and must be serialised by the caller.
 *   - *mean (host, nullable) receives the removed mean and then the call synchronises. */
amr_status amr_mean_zero_noalloc(amr_hierarchy* h, double* phi, double* mean, void* stream);

/* G^comp (COH-1,2,4; Eq. discreteOps a): grad[d] = component d.  Ghosts of phi use
 * bc_types (data bc, nullable). */
amr_status amr_gradient(amr_hierarchy* h, const int* bc_types, double* phi, double* const* grad,
                        const double* bc, void* stream);
/* D^comp (COH-1..4 with refluxing of Eq. cell2face face values; Eq. discreteOps b).
 * Ghosts of u[d] use bc_types with data bc[d] (array of dim pointers, or NULL). */
amr_status amr_divergence(amr_hierarchy* h, const int* bc_types, double* const* u, double* out,
                          const double* const* bc, void* stream);

/* Composite projection u = w - G^comp (L^comp)^{-1} D^comp w (Eq. comp_ProjOp): ppe is an
 * all-Neumann operator with alpha = 0, beta = 1; w ghosts use vel_bc_types with data
 * w_bc[d] (nullable); no average-down of u afterwards (Lemma compositeProjection).
 * phi (device, composite field) receives the mean-zero potential. */
amr_status amr_project(amr_operator* ppe, const amr_solver_params* p, const int* vel_bc_types,
                       double* const* w, const double* const* w_bc, double* const* u, double* phi,
                       amr_solve_stats* stats, void* stream);

/* Adjoint (transposed) operator: out = A^T y over the valid cells (homogeneous data);
 * y and out are composite fields whose invalid cells are ignored (out's are set to 0). */
amr_status amr_apply_transpose(amr_operator* op, const double* y, double* out, void* stream);
/* lambda = A^{-T} g over the valid cells (the adjoint solve), by V-cycles on A^T: every
 * level operator replaced by its transpose (interior stencil, physical-ghost coefficients),
 * exact composite transposes (refluxing, AMRCFI, average-down) for the residuals passed
 * between levels, FP64 outer residual (precision as in amr_solve).  Values of g on invalid
 * cells are first handed to their children (transposed average-down), so that a gradient
 * with respect to a composite field whose invalid cells are averages is propagated
 * correctly; ghost cells of g are ignored; lambda's invalid cells are set to 0.
 * Pure-Neumann operator (alpha = 0, every face Neumann): the adjoint of the whole solve map
 * of amr_solve (Sec. 6.4 solvability correction, solve, h^D-weighted mean zero).  With
 * w = h^D on the valid cells it returns the lambda with A^T lambda = g - w (1^T g)/(1^T w)
 * and 1^T lambda = 0 (the null vectors of A are 1 on the right and w on the left);
 * stats->removed_mean receives (1^T g)/(1^T w). */
amr_status amr_solve_transpose(amr_operator* op, const amr_solver_params* p, double* lambda,
                               const double* g, amr_solve_stats* stats, void* stream);

/* out = (G^comp)^T y: the adjoint of amr_gradient's linear part (homogeneous boundary data,
 * ghosts of types bc_types).  y: dim device composite fields; weight on their invalid cells
 * (where G^comp's output is the average of the children, COH-4) is handed to the children
 * first.  out (device composite field) receives values on the valid cells and 0 on the
 * invalid cells; its ghost cells are scratch.  Uses a hierarchy-owned scratch of three
 * fields (allocated on the first call): calls on one hierarchy must not overlap. */
amr_status amr_gradient_transpose(amr_hierarchy* h, const int* bc_types, const double* const* y, double* out,
                                  void* stream);
/* out[d] = the component-d part of (D^comp)^T y (adjoint of amr_divergence's linear part,
 * including the transposed refluxing of the face values of Eq. cell2face).  Same
 * conventions as amr_gradient_transpose. */
amr_status amr_divergence_transpose(amr_hierarchy* h, const int* bc_types, const double* y, double* const* out,
                                    void* stream);
/* out = P^T v: the adjoint of amr_project's linear map w -> u (homogeneous w_bc), as a map
 * on the covered cells of every level of each of the dim components: u_d reads w_d itself
 * on every cell and, on the valid cells, through G^comp (L^comp)^{-1} D^comp.  Hence
 * out_d = v_d - (D^comp)^T lambda with lambda = M^T (G^comp)^T v, M the pure-Neumann solve
 * map (amr_solve_transpose).  lambda (device composite field) receives that adjoint
 * potential.  ppe as for amr_project; p controls the adjoint solve. */
amr_status amr_project_transpose(amr_operator* ppe, const amr_solver_params* p, const int* vel_bc_types,
                                 const double* const* v, double* const* out, double* lambda,
                                 amr_solve_stats* stats, void* stream);

/* Batched solves: n independent problems (each with its own operator; hierarchies may
 * differ, e.g. the uneven sizes of a batch of single-level Helmholtz problems; boundary data
 * homogeneous).  When every problem is a single-level 2-D problem solved in mixed precision
 * with temporally blocked legs (nu1, nu2 in 1..4, no pure-Neumann operator) whose level-0
 * pyramid ends in the square one-block coarse V-cycle (64 -> 4 or 48 -> 6: level-0 sizes
 * 64 * 2^k or 48 * 2^k), the batch runs as one captured CUDA graph (built on the first call,
 * reused while the operators, fields and parameters stay the same): every phase of the
 * refinement loop (the down legs of one depth, the coarse V-cycles, the up legs, the update,
 * the FP64 residual, its norm, the stopping test) is one launch over a descriptor list
 * covering all problems, and a device-side loop runs until every problem has converged,
 * problems that have converged skipping their entries.  When the problems are 3-D, their
 * hierarchies have one geometry (the same boxes on every level) and their operators are one
 * operator (alpha, beta, boundary types; not the pure-Neumann PPE) -- e.g. the Helmholtz
 * systems of the velocity components -- they are solved as one stacked problem: a hierarchy
 * holding one replica of every patch and work list per problem (built on the first call,
 * kept with the first operator), one captured graph in which every phase of the V-cycle and
 * of the refinement loop is one launch over all replicas, a stopping test per replica (a
 * converged replica's phi is no longer updated; statistics and statuses per problem as for
 * separate solves; the fields are copied in and out of the stacked arrays inside the call)
 * when amr_set_stacked_batches(1) is in effect.  Otherwise each problem runs its own
 * captured graph (p->use_graph is forced to 1), launched concurrently on a pool of internal
 * streams forked from ``stream`` and joined back to it; problems that share a hierarchy then
 * run one after another on the same stream because they share its reduction scratch.  The
 * call synchronises ``stream``.
 * stats and status (host arrays of n entries, nullable) receive each problem's statistics
 * and status; the return value is the first non-OK status (AMR_OK if all converged). */
amr_status amr_batch_solve(amr_operator* const* ops, int n, const amr_solver_params* p, double* const* phi,
                           const double* const* f, amr_solve_stats* stats, int* status, void* stream);

/* Host-buffer variant of amr_solve: phi and f are HOST pointers (pinned or pageable);
 * the library copies them to its own device buffers and back inside the call. */
amr_status amr_solve_host(amr_operator* op, const amr_solver_params* p, double* phi_host,
                          const double* f_host, const double* bc_host, amr_solve_stats* stats,
                          void* stream);

/* Host-buffer variant of amr_batch_solve (same batching, statistics and return value):
 * phi_host[k] and f_host[k] are HOST pointers (pinned or pageable) of problem k's composite
 * fields.  Every f (and phi unless p->zero_initial) is copied into device buffers owned by
 * the problem's operator (allocated on the first host-buffer call, freed with the
 * operator), the batch is solved, and every phi is copied back before the call returns.
 * An operator may appear only once in a call (AMR_ERR_INVALID_ARG otherwise). */
amr_status amr_batch_solve_host(amr_operator* const* ops, int n, const amr_solver_params* p, double* const* phi_host,
                                const double* const* f_host, amr_solve_stats* stats, int* status, void* stream);

/* ---- coarse-fine interface conditions of a subcycled level solve ------------------- */
/* In the subcycled method each refined level l advances with its own time step and reads its
 * coarse-fine interface data from level l-1 at four equispaced coarse times (Sec. 6.3, steps
 * CIC-2 and CIC-3).  These calls are the data-parallel part of that: the interface ghosts at
 * an intermediate time and the corrected interface face averages.  All need 1 <= level <
 * nlevels on an unstacked hierarchy of refinement ratio 2 (AMR_ERR_INVALID_ARG otherwise). */

/* CF ghost cells of `level` at the time t* of Eq. (timeInterp): coarse[i] (i = 0..3; device
 * composite fields, only level-1 read) hold the data at t_{-i} = t^{l-1} - i k (so coarse[0]
 * is the latest), k > 0 is the coarse time step and eta = t* - t_{-1} (usually 0 <= eta <=
 * k).  The printed matrix's columns take the four times in increasing order (its entries are
 * the cubic Lagrange weights of eta = -2k, -k, 0, k), the reverse of the printed vector, so
 * printed column j is applied to coarse[3-j]; eta = 0 gives exactly coarse[1] and eta = k
 * coarse[0].  The printed second row is the eta-derivative of the first, so `rate` receives
 * d(phi)/dt at t* (multiply by k for the k d(phi)/dt of the equation's left side).  Every
 * level-`level` ghost cell that AMRCFI fills (Sec. 5.2) receives, in `value`, the AMRCFI
 * value of the interpolated coarse data, and in `rate` (nullable) that of its time
 * derivative; no other cell of either field is written.  AMRCFI windows may include coarse
 * cells covered by `level`: coarse[i] must hold their average-down there, as after
 * amr_fill_ghosts.  Fails on null fields, k <= 0 or a non-finite k or eta. */
amr_status amr_cic_ghosts(amr_hierarchy* h, int level, const double* const* coarse, double k, double eta,
                          double* value, double* rate, void* stream);

/* The coarse-fine interface faces of `level` (faces between a cell of the level's boxes and a
 * CF ghost cell; one per first-layer CF ghost) and the level's connected components (Sec.
 * 5.1; numbered in ascending order of their smallest box index in the level's box list).
 * Host-only, works without a GPU.  Faces are grouped by component.  Two-call pattern: any
 * output may be NULL.  nfaces / ncomponents: counts; cell (nfaces x dim ints): global index,
 * at the level, of the interior cell next to each face; face (nfaces): 2 d + side (side 1:
 * the cell's high face along dimension d, so the outward normal is +e_d; 0: -e_d);
 * component (nfaces): the face's component. */
amr_status amr_cic_faces(const amr_hierarchy* h, int level, int* nfaces, int* ncomponents, int* cell, int* face,
                         int* component);

/* Normal face averages n . <w> on the interface faces of `level`, corrected per connected
 * component (Sec. 6.4, Eq. correctingFaceAvg).  w[d] (d < dim; device composite fields):
 * the velocity components, with the level's ghost cells filled (CF ghosts at the wanted time,
 * e.g. by amr_cic_ghosts; ghosts inside sibling boxes copied, e.g. by amr_fill_ghosts).  Each
 * face average is Eq. (cell2face) along the normal over the two interior cells and the two
 * ghost layers.  phys (device, ncomponents doubles, nullable = zeros): for each component,
 * the sum of the face averages n . <u^b> over its faces on the physical boundary.  Then for
 * every component c one shift delta_c is added to all its interface faces, so that
 * -delta_c |faces of c| = (sum of its uncorrected interface averages) + phys[c], i.e. the
 * corrected interface sum plus phys[c] is zero.  faces (device, nfaces doubles; NULL allowed
 * when the level has no interface face): the corrected averages in amr_cic_faces order;
 * delta (device, ncomponents doubles, nullable): the shifts (0 for a component with no
 * interface face).  Every sum is a fixed-order tree (two passes over chunks of each
 * component's faces), so results are deterministic. */
amr_status amr_cic_face_averages(amr_hierarchy* h, int level, const double* const* w, const double* phys,
                                 double* faces, double* delta, void* stream);

/* The level problem of Def. GePUP-E-OneLevel on a connected component of `level` that is a
 * single box: level l solved alone on that box, with the interface conditions as boundary
 * data on the box faces that lie on the coarse-fine interface.  Such a component is a
 * one-level problem whose domain is the box (n0 = hi - lo + 1, h0 = the level's cell size),
 * so amr_hierarchy_create, amr_operator_create and amr_solve solve it; these two calls give
 * its geometry and its interface data.  Components of several boxes are rejected with
 * AMR_ERR_INVALID_ARG (their level problem is not a box problem).
 *
 * amr_cic_component_box (host-only): lo[dim], hi[dim] (nullable) the box in the level's
 * index space; interface_faces[2*dim] (nullable) 1 where face f = 2d+side of the box lies on
 * the coarse-fine interface, 0 where it lies on the physical boundary. */
amr_status amr_cic_component_box(const amr_hierarchy* h, int level, int component, int* lo, int* hi,
                                 int* interface_faces);

/* Face averages <x> (Eq. cell2face along the face normal, over the two interior cells and the
 * two ghost layers) of the composite field x (device; the level's ghosts filled, CF ghosts at
 * the wanted time, e.g. by amr_cic_ghosts) on every interface face of a single-box component,
 * written into bc (device) in the boundary-data layout of the component's one-level box
 * problem (amr_bc_layout of that hierarchy: faces f = 2d+side in order, each over the box's
 * cells with dimension d removed, lowest remaining dimension fastest): the Dirichlet data
 * w = w^I on the interface (Eq. GePUP-localized a).  Slots of faces on the physical boundary
 * are not written. */
amr_status amr_cic_interface_bc(amr_hierarchy* h, int level, int component, const double* x, double* bc,
                                void* stream);

/* ---- regridding ----------------------------------------------------------------------- */
/* New level boxes from tagged cells (Sec. 5.4, RDM-2 and RDM-3), host-only.  Level
 * nlevels-1 is built from the tags of level nlevels-2 by the clustering algorithm of Berger
 * and Rigoutsos; then for l = nlevels-3 .. 0 the tags of level l are united with the boxes of
 * the new level l+2 coarsened twice and grown by ceil(3 / ratio) cells (clipped to the
 * domain) and clustered into the new level l+1 -- the growth makes every new level contain
 * the three-cell margin that AMRCFI windows need around the next finer one (the paper grows
 * by one cell with ratio 4, which is the same margin), and the clustered boxes are refined
 * by `ratio`.  Clustering of the tagged cells T of a region (the recursion partitions the
 * level's domain into disjoint regions at least min_width cells wide): the bounding box of T,
 * widened inside the region to min_width cells; accepted when |T| >= efficiency x its cells;
 * otherwise cut in two (both parts at least min_width wide) at a hole of a signature (tags
 * per slice) closest to the middle of its dimension, else at the inflection point (second
 * differences of the signature of strictly opposite signs) with the largest jump, else at
 * the middle of the longest dimension that can be cut; ties go to the cut closest to its
 * dimension's middle, then the longer dimension, the lower dimension, the lower position;
 * a box that cannot be cut is accepted.  The result passes amr_hierarchy_create's checks.
 *   ntags[l], tags[l] (l = 0 .. nlevels-2; host): ntags[l] cells of level l, dim ints each
 *     (global indices in level l's index space; repeats allowed).
 *   new_nlevels: levels of the new hierarchy (a level with no box ends it);
 *   nboxes (nlevels ints, nullable): boxes per new level (nboxes[0] = 1, 0 past the end);
 *   boxes (nullable): the amr_hierarchy_desc box list (the level-0 domain box first, then
 *     every new level's boxes: lo[0..dim-1], hi[0..dim-1]), at most max_boxes boxes;
 *     AMR_ERR_INVALID_ARG when more are needed (call with boxes = NULL for the counts). */
/* Data migration after regridding (Sec. 5.4, last paragraph): the composite field old_x of
 * old_h onto new_x of new_h (device fields; same dimension, ratio and level-0 domain; old_x
 * and new_x distinct; ratio 2).  Levels in order: every cell of a box of new level l that lies in a
 * box of old level l takes the old value of that cell (level 0 is copied whole); every other
 * cell takes the AMRCFI value (Sec. 5.2) from new level l-1, which is complete by then, so
 * the interpolation source is old data throughout (copied, or itself interpolated from old
 * data).  Ghost cells of new_x are not written.  The plan (copy blocks, AMRCFI windows) is
 * built on the host at each call and its device copy freed before returning; the call
 * synchronises `stream`.  AMR_ERR_NESTING if an AMRCFI window leaves new level l-1. */
amr_status amr_migrate(amr_hierarchy* old_h, const double* old_x, amr_hierarchy* new_h, double* new_x,
                       void* stream);

/* The migration plan of one new level (host-only, for inspection and tests; two-call
 * pattern, every output nullable): nblocks copy blocks as (new patch, old patch, lo[dim],
 * hi[dim]) in blocks (2 + 2*dim ints each, level index space); ncells interpolated cells:
 * cells (dim ints each, global index), starts (dim ints each, the window's first coarse
 * cell), dst (the cell's element offset in new_x), src (the element offset in new_x of the
 * window's first cell when the window lies in one coarse patch, else -1-k: the window's
 * 5^dim offsets are side[k*5^dim ...]); nside / side: the side tables. */
amr_status amr_migrate_plan(const amr_hierarchy* old_h, const amr_hierarchy* new_h, int level, int* nblocks,
                            int* blocks, long long* ncells, int* cells, int* starts, long long* dst, long long* src,
                            long long* nside, long long* side);

typedef struct {
  double efficiency; /* 0 < efficiency <= 1 */
  int min_width;     /* smallest box width, in cells of the clustered level; >= ceil(4 / ratio) */
} amr_regrid_params;

amr_status amr_regrid(int dim, int ratio, const int* n0, int nlevels, const int* ntags, const int* const* tags,
                      const amr_regrid_params* p, int* new_nlevels, int* nboxes, int* boxes, int max_boxes);

void amr_default_params(amr_solver_params* p);
const char* amr_last_error(void);
/* Number of CUDA kernels this library has launched in the process so far (a host-side
 * counter; a replayed CUDA graph counts its kernel nodes). */
long long amr_kernel_launches(void);
/* Bench instrumentation.  amr_profile_enable(1) clears the record and makes the library
 * bracket every launch of the instrumented kernel classes with CUDA events on the
 * launching stream (0 stops recording).  amr_profile_read() synchronises on the recorded
 * events and returns, for one class, the number of launches, the summed event intervals
 * (ms) and the summed algorithmic bytes.  Classes: 0 weighted-Jacobi sweeps, 1 level
 * residual / apply (FP32; FP64 applications), 2 restriction and average-down, 3
 * prolongation, 4 temporally blocked down legs (f read, x and the coarse f written once),
 * 5 temporally blocked up legs (x, f and the coarse correction read once, x written once),
 * 6 one-block coarse V-cycles (f read, x written once), 7 FP64 level residuals (the
 * refinement loop's residual: x, f read, r written). */
amr_status amr_profile_enable(int on);
amr_status amr_profile_read(int kernel_class, long long* launches, double* total_ms, double* total_bytes);
/* The same sums over the launches of one class whose grid has between min_cells and
 * max_cells cells (inclusive; level operators, sweeps and residuals record their grid's cell
 * count, other classes record 0). */
amr_status amr_profile_read_range(int kernel_class, double min_cells, double max_cells, long long* launches,
                                  double* total_ms, double* total_bytes);
/* Tile shape of the tiled level-operator kernels (not in the paper: a tuning and testing
 * control).  rows = 0 (the default) uses the autotuner's choice per grid; rows = 1, 2 or 4
 * forces that many cells per thread along y in the 2-D kernel, rows = 2 or 4 in the 3-D
 * z-chunked kernel (a 3-D grid whose y extent is not a multiple of 8 rows takes 2; rows = 1
 * counts as 2 there).  Process-wide; AMR_ERR_INVALID_ARG for any other value. */
amr_status amr_set_tile_rows(int rows);
/* FP64 residual of 3-D single-patch levels whose x / y extents are multiples of 32 x 16 (the
 * refinement loop's residual and amr_residual).  on = 1 (the default): every value of phi
 * the stencil reads is rounded once to a 64-bit fixed-point frame whose unit is 2^-52 times
 * the largest interior |phi| rounded down to a power of two (at most half a unit in the last
 * place of that value, the size of one FP64 rounding of it); the sum 16 s1 - s2 - 90 phi of
 * Eq. (discreteOps) is then exact in int64, and r = f - alpha phi - beta/(12 h^2) * sum is
 * formed in FP64.  Physical ghost values are fixed combinations of interior values and
 * always fit; a stored ghost value (coarse-fine, copy) of 4 * 2^53 units or more, or a
 * non-finite value, makes the plain FP64 kernel recompute the level.  Not in the paper: on
 * this GPU FP64 arithmetic runs at a small fraction of the integer rate.  on = 0: the plain
 * FP64 kernel always.  Process-wide; AMR_ERR_INVALID_ARG for any other value. */
amr_status amr_set_fx_residual(int on);
/* 3-D level operator of single-patch levels whose x extent is a multiple of 64 cells and whose
 * y extent is a multiple of 16 (not in the paper: a kernel choice for this GPU).  The
 * weighted-Jacobi sweeps, residuals and operator applications of such levels can run in a
 * kernel whose planes of x and f are streamed into shared memory by tensor-map TMA copies
 * (a producer thread, a warp that writes the physical ghost values into the staged planes,
 * consumer warps; a ring of slots with mbarriers), or in the z-chunked register-prefetch
 * kernel; both evaluate the same operations per cell.  on = 1 (the default): the tile
 * autotuner times both on every such grid and keeps the faster; on = 2: the bulk-copy kernel
 * wherever eligible; on = 0: never.  Process-wide; AMR_ERR_INVALID_ARG for any other value. */
amr_status amr_set_bulk_sweep(int on);
/* The bulk-copy 3-D kernel bounds every wait on its shared-memory pipeline; a wait that runs
 * out sets a device flag (the kernel then stops without writing its remaining cells).  This
 * call reads and clears the flag: AMR_ERR_CUDA if it was set since the last check, else
 * AMR_OK.  Solves check it when they finish (amr_solve and amr_batch_solve return
 * AMR_ERR_CUDA). */
amr_status amr_check_kernel_flags(void);
/* Stacked solves of 3-D batches that share one geometry and one operator in amr_batch_solve
 * (not in the paper: a launch-count choice).  on = 1: stacked (one launch per phase over all
 * problems); on = 0 (the default): one captured solve per problem, launched concurrently --
 * on GB300 the concurrent graphs overlap one problem's latency-bound coarse phases with
 * another's bandwidth-bound fine phases and measure faster.  Process-wide;
 * AMR_ERR_INVALID_ARG for any other value. */
amr_status amr_set_stacked_batches(int on);

#ifdef __cplusplus
}
#endif
#endif /* AMR4_H */
