/*
 * gmg.h - C ABI of the GB300 octree geometric-multigrid Poisson solver with
 * level-set Dirichlet boundaries (method of Teunissen & Schiavello,
 * arXiv 2205.09411).
 *
 * The library solves  Laplacian(phi) = g  (Sec. 1, Eq. (poisson) with a
 * constant coefficient) on a quadtree/octree of N^D-cell blocks (Sec. 2.1).
 * Irregular Dirichlet boundaries are the zero contour of a level-set
 * function (Sec. 3.1); their distances to cell centres come from line
 * searches (Sec. 3.2) and enter per-block stored cut-cell stencils
 * (Sec. 3.3, Sec. 3.6.2).  The solver is a FAS multigrid V-cycle with
 * red-black Gauss-Seidel smoothing, mean restriction, (bi/tri)linear
 * prolongation and an exact coarse-level solve (Sec. 2.2, Sec. 3.4, 3.5).
 *
 * Conventions for every function:
 *  - return value: GMG_OK (0) or a negative GMG_ERR_* code; the message of
 *    the last error of the calling thread is gmg_last_error().
 *  - "host" pointers are ordinary CPU memory owned by the caller; the
 *    library copies what it needs before returning.  "device" pointers are
 *    CUDA global memory of the current device, borrowed for the call only.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream); device
 *    work is enqueued on it and the call returns without waiting, except
 *    where a function says it synchronises.
 *  - leaf-cell order: leaf blocks by increasing level, inside a level by
 *    increasing Morton code of the block's integer coordinates (x lowest
 *    bit); inside a block, cells x-fastest then y then z.
 *  - right-hand-side slots: a tree holds nrhs (gmg_set_num_rhs, default 1)
 *    independent copies of its level fields, one per right-hand side, that
 *    share the tables, stencils and coarse inverse.  Every kernel runs the
 *    (block, slot) pairs of a level in one launch.  Arrays that hold leaf
 *    values of several slots are slot-major: slot r's leaf cells start at
 *    r * n_leaf_cells.
 *  - forests: gmg_forest_create merges many set-up trees (independent
 *    problems) into one gmg_tree; a "unit" is one (slot, tree) pair, unit
 *    r * n_trees + i.  Per-unit arrays (residuals, statistics, activity
 *    masks) hold nrhs * n_trees entries; a single tree has one tree.
 *  - a gmg_tree owns all the device memory it uses: either one workspace
 *    the caller binds (gmg_tree_bind with a device pointer) or one the
 *    library allocates itself (gmg_tree_bind with NULL).  It stays valid
 *    until gmg_tree_destroy.  A tree is not thread-safe.
 */
#ifndef GMG_H
#define GMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GMG_OK 0
#define GMG_ERR_INVALID_ARG (-1)   /* a size, pointer or option is out of range   */
#define GMG_ERR_OOM (-2)           /* workspace too small or allocation refused    */
#define GMG_ERR_CUDA (-3)          /* a CUDA runtime call failed                   */
#define GMG_ERR_NOT_CONVERGED (-4) /* the tolerance was not met in max_cycles      */
#define GMG_ERR_NONFINITE (-5)     /* a residual norm became NaN/Inf or diverged   */
#define GMG_ERR_STATE (-6)         /* call out of order (e.g. solve before bind)   */
#define GMG_ERR_TIMEOUT (-7)       /* a bounded device-side wait ran out           */

/* domain wall boundary conditions: Dirichlet ghost 2 phi_w - phi_i, Neumann ghost phi_i */
#define GMG_WALL_DIRICHLET 0
#define GMG_WALL_NEUMANN 1 /* zero normal derivative */

/* built-in level-set functions f(x); f < 0 inside the object (Sec. 3.1) */
#define GMG_LSF_NONE 0
#define GMG_LSF_SPHERE 1    /* p[0..2] centre c, p[3] radius R: |x - c| - R, Eq. (lsf-example) */
#define GMG_LSF_CAPSULE 2   /* p[0..2] a, p[3..5] b, p[6] r: distance to segment ab minus r   */
#define GMG_LSF_ELLIPSOID 3 /* p[0..2] c, p[3..11] rotation Q (row-major), p[12..14] semi-axes s:
                               min(s) * (|diag(s)^-1 Q^T (x - c)| - 1)                         */
#define GMG_LSF_CALLBACK 4  /* the host function `fn` */
#define GMG_LSF_SHAPE 5     /* the sharp shapes of Sec. 4.3: p[0] = 0 spheroid, 1 rhombus, 2 heart,
                               3 astroid in the coordinates (p, q) = (4 (x - 1/2), 4 (y - 1/2)),
                               or with p[1] = 1 revolved: (4 (sqrt(x^2 + y^2) - 1/2), 4 (z - 1/2)) */
#define GMG_LSF_GRID 6      /* samples of f on a uniform grid, interpolated (bi/tri)linearly:
                               p[0..2] sample counts (>= 2 on each used axis), p[3..5] position of
                               sample 0, p[6..8] spacing (> 0); `user` points to the samples
                               (double, x fastest), caller-owned, alive while the tree may set up
                               or re-mesh; points outside the sampled box take the nearest face */

/* solver arithmetic */
#define GMG_FP64 0  /* FAS V-cycles in FP64                                            */
#define GMG_MIXED 1 /* FP64 defect correction around FP32 V-cycles; the fine residual,
                       the solution update and the coarsest-level solve stay in FP64  */
#define GMG_MIXED_BF16 2 /* GMG_MIXED with the FP32 correction's state (e) on the finest
                       level stored as BF16: 2 bytes a cell instead of 4 in the sweeps,
                       restriction, prolongation and accumulation of that level; the
                       arithmetic stays FP32, b stays FP32, and every result written
                       to the level is rounded to BF16 (nearest, ties to even).  The
                       BF16 values live in that level's part of the second FP32 buffer
                       of the workspace (no extra memory).  A tree whose finest level
                       runs inside the coarse cooperative or cluster kernels, or whose
                       block side has no compiled kernel (3D: 4, 8, 16; 2D: 8, 16,
                       32), runs GMG_MIXED instead.  The BF16 rounding limits what one
                       correction can reduce (a few 1e-3 relative), so a step can
                       reduce the residual less than a GMG_MIXED step; the solve still
                       ends at the requested FP64 residual, checked in FP64.  No
                       counterpart in the paper (Sec. 2.2 gives the smoother and
                       transfers in one precision). */

/* where a caller's array lives.  A GMG_HOST array in page-locked memory
 * mapped into the device's address space (cudaHostAlloc, cudaHostRegister,
 * pinned PyTorch tensors) is read or written by the library's kernels
 * directly over the CPU-GPU link; pageable host memory is staged through
 * device memory with cudaMemcpyAsync.  Same values either way.  As with any
 * asynchronous copy from page-locked memory, a page-locked input must stay
 * unchanged until the stream has passed the call (calls that return host
 * results synchronise the stream before they return). */
#define GMG_HOST 0
#define GMG_DEVICE 1

typedef struct gmg_tree gmg_tree;

/* host callback: value at point x[3] (unused coordinates are 0) */
typedef double (*gmg_fn)(const double *x, void *user);
/* host callback: refine block bix[3] of `level` (1 = root level)? nonzero = yes */
typedef int (*gmg_refine_fn)(int level, const int *bix, void *user);

typedef struct {
  int dim;               /* 2 or 3                                                      */
  int block_n;           /* cells per block side N: even, 4 <= N <= 16 (3D), <= 32 (2D)  */
  int coarse_blocks[3];  /* root blocks per side (level 1)                              */
  double lo[3];          /* domain corner                                               */
  double h_root;         /* cell size on level 1 (cubic cells)                          */
  int max_level;         /* finest level allowed, 1..20                                 */
  int max_coarse_cells;  /* coarsest-level size for the direct solve; 0 = 64 (2D) / 512 (3D) */
  gmg_refine_fn refine;  /* NULL: refine every block up to max_level (uniform tree)     */
  void *refine_user;
} gmg_domain;

typedef struct {
  int kind;     /* GMG_LSF_*                        */
  double p[16]; /* parameters of the built-in kinds */
  gmg_fn fn;    /* GMG_LSF_CALLBACK: f(x, user)     */
  void *user;
} gmg_lsf;

typedef struct {
  int n_down;         /* GSRB sweeps before restriction (Sec. 2.2; default 2)          */
  int n_up;           /* GSRB sweeps after prolongation (default 2)                    */
  double eps_tol;     /* line-search relative tolerance (Sec. 3.2; default 1e-8)       */
  double mask_factor; /* L = mask_factor sqrt(D) dx in Eq. (boundary-mask) (1.5)        */
  double w_min;       /* unresolved-root threshold of Sec. 3.6.3 (0 = off)             */
} gmg_params;

typedef struct { /* per slot */
  int cycles;     /* V-cycles run (FP64) or defect-correction steps (mixed)    */
  double rel_l2;  /* final ||b - A phi||_2 / ||b||_2 over leaf cells           */
  double linf;    /* final max |b - A phi|                                      */
  double bnorm;   /* ||b||_2                                                   */
} gmg_stats;

/* Fills *p with the defaults of Sec. 2.2, 3.2 and 3.6.1. */
void gmg_default_params(gmg_params *p);

/* Builds the block tree (Sec. 2.1) on the host: root blocks at level 1,
 * refinement decided by domain->refine level by level, then closed under
 * 2:1 balance across faces, edges and corners; levels below 1 coarsen inside
 * the root blocks until the coarsest level has at most max_coarse_cells
 * cells (the coarse-grid solve of Sec. 3.5 is exact on that level).
 * params may be NULL (defaults).  No device memory is touched.
 * Errors: INVALID_ARG for sizes out of range. */
int gmg_tree_create(const gmg_domain *domain, const gmg_params *params, gmg_tree **out);
void gmg_tree_destroy(gmg_tree *tree);

/* Tree shape: level range, number of leaf cells, number of blocks. */
int gmg_tree_info(const gmg_tree *tree, int *lmin, int *lmax, long long *n_leaf_cells, long long *n_blocks);
/* Level shape: number of blocks, cells per block side, cell size. */
int gmg_level_info(const gmg_tree *tree, int level, int *n_blocks, int *block_n, double *h);
/* Blocks of one level in canonical order: bix[3*i..], has_children[i] (host arrays). */
int gmg_level_blocks(const gmg_tree *tree, int level, int *bix, int *has_children);
/* Cell centres of the leaf cells (host array of n_leaf_cells * dim doubles). */
int gmg_leaf_centers(const gmg_tree *tree, double *xyz);

/* Domain-wall conditions (2*dim entries, order -x,+x,-y,+y,-z,+z).  Dirichlet
 * values come from fn(x_face, user) when fn != NULL, else from values[]. */
int gmg_set_walls(gmg_tree *tree, const int *types, const double *values, gmg_fn fn, void *user);

/* Boundary detection and stencils (Sec. 3.2, 3.3, 3.6): on every level the
 * mask of Eq. (boundary-mask), line searches toward the 2D neighbour
 * centres, the unresolved-root search of Sec. 3.6.3 (if w_min > 0), the
 * cut-cell coefficients of Eq. (lpl-1d-lsf) with the coefficients of
 * boundary neighbours moved to the right-hand side (value phib(x0, user) at
 * the root x0, or phib_const when phib == NULL), the Dirichlet wall terms,
 * and the coarsest-level inverse.  Runs before gmg_tree_bind (results are
 * uploaded by gmg_tree_bind).  With a built-in sphere, capsule or ellipsoid
 * and a CUDA device present (option GMG_OPT_DEVICE_SETUP, default on) the
 * mask, line searches and unresolved-root search run as device kernels on
 * the current device (temporary device memory, freed before the call
 * returns; the call synchronises); callbacks, sampled level sets and sharp
 * shapes run on the host.  Both give the same values bit for bit.  The
 * stencils and terms are assembled on the host.
 * Errors: STATE if already bound, CUDA (device set-up). */
int gmg_store_stencils(gmg_tree *tree, const gmg_lsf *lsf, gmg_fn phib, void *phib_user, double phib_const);
/* 1 when the tree's last gmg_store_stencils ran its boundary detection on
 * the device, else 0. */
int gmg_setup_on_device(const gmg_tree *tree);

/* A new boundary value phi_b (phib(x0, user), or phib_const when phib ==
 * NULL) on the stored boundary: phi_b at every located root and the moved
 * coefficients' right-hand-side terms are recomputed from the stored
 * distances, without new line searches (the stencils do not depend on
 * phi_b).  Gives the boundary terms a full gmg_store_stencils with the new
 * value gives.  After gmg_store_stencils, before gmg_tree_bind (a single
 * tree; forests take trees set up this way).  Errors: STATE otherwise. */
int gmg_set_boundary_value(gmg_tree *tree, gmg_fn phib, void *phib_user, double phib_const);

/* Forest of independent problems (the batched form of the method: many
 * trees, each with its own level set, boundary values, refinement and size,
 * in every launch).  `trees` are n_trees set-up trees (gmg_tree_create +
 * gmg_set_walls + gmg_store_stencils, not bound), each with exactly one root
 * block, and all with the same dimension, block size, root cell size,
 * coarsest level, sweep counts and wall types (wall values, level sets and
 * depths may differ).  The forest copies what it needs: the trees may be
 * destroyed afterwards.  Level l of the forest holds the level-l blocks of
 * every tree; the coarsest level holds one block per tree with that tree's
 * direct-solve inverse.  Leaf cells are tree-major: tree i's leaves, in its
 * own leaf order, start at the offset gmg_forest_tree_info returns.  Norms,
 * convergence tests and freezing are per (slot, tree) unit, so each tree's
 * result is that of its own solve.  Errors: INVALID_ARG (shapes differ, a
 * tree has several roots), STATE (a tree not set up or already bound). */
int gmg_forest_create(gmg_tree *const *trees, int n_trees, gmg_tree **out);
int gmg_num_trees(const gmg_tree *tree);
int gmg_forest_tree_info(const gmg_tree *forest, int tree, long long *leaf_offset, long long *n_leaf_cells);

/* Re-meshing (Sec. 4.5: boundary detection is done for newly added cells;
 * removing refinement costs nothing): a new tree on the same domain, level
 * set, boundary values, walls and parameters as `old`, refined by `refine`
 * up to max_level, with its set-up done.  Blocks that exist in `old` (same
 * level and coordinates) take old's set-up (it depends only on the block's
 * own cells); only new blocks run the mask, line searches and stencils.
 * The result equals a set-up from scratch.  `old` must have been set up with
 * built-in or still valid callbacks; the new tree is not bound.
 * gmg_setup_counts tells how many blocks were set up and how many reused.
 * Errors: STATE (old not set up), INVALID_ARG (a forest). */
int gmg_tree_remesh(const gmg_tree *old, gmg_refine_fn refine, void *refine_user, int max_level, gmg_tree **out);
int gmg_setup_counts(const gmg_tree *tree, long long *computed, long long *reused);
/* Initial guess of a re-meshed tree from the previous tree's solution, for
 * every slot: blocks that exist in both copy their values, new blocks take
 * the value of the parent cell containing each cell, covered cells are then
 * restricted.  Both trees bound, same slot count.  Synchronises. */
int gmg_transfer_solution(const gmg_tree *old, gmg_tree *tree, void *stream);

/* Number of right-hand-side slots (1 .. 65536) the workspace holds; call
 * before gmg_tree_bind (default 1).  Errors: STATE after bind. */
int gmg_set_num_rhs(gmg_tree *tree, int nrhs);
int gmg_num_rhs(const gmg_tree *tree);

/* Number of bytes of device workspace the tree needs (after
 * gmg_store_stencils): tables, FP64 and FP32 level fields, stencil pools,
 * coarse inverse, reduction scratch.  256-byte alignment is enough. */
int gmg_workspace_bytes(const gmg_tree *tree, size_t *bytes);
/* Binds the device workspace: `device_ptr` (caller-owned, at least
 * gmg_workspace_bytes, 256-byte aligned; it must outlive the tree) or NULL
 * (the library allocates it with cudaMalloc and frees it at destroy), and
 * uploads tables and stencils.  Synchronises the device.
 * Errors: STATE before gmg_store_stencils, OOM, CUDA. */
int gmg_tree_bind(gmg_tree *tree, void *device_ptr, size_t bytes);

/* Right-hand sides g on the leaf cells (leaf-cell order, FP64, host or
 * device by `where`; nrhs x n_leaf_cells values, slot-major): sets
 * b = g - (moved boundary terms) - (Dirichlet wall terms) and phi = 0 on
 * every level (zero initial guess) of every slot. */
int gmg_set_rhs(gmg_tree *tree, const double *g, int where, void *stream);
/* The same for slots slot0 .. slot0 + nslots - 1 only (g: nslots x
 * n_leaf_cells); the other slots are untouched, so a slot can take a new
 * right-hand side while the others are mid-solve.  Errors: INVALID_ARG for a
 * slot range outside 0 .. nrhs - 1. */
int gmg_set_rhs_slots(gmg_tree *tree, int slot0, int nslots, const double *g, int where, void *stream);
/* Initial guess on the leaf cells of every slot (nrhs x n_leaf_cells;
 * covered cells get the mean of their children). */
int gmg_set_solution(gmg_tree *tree, const double *phi, int where, void *stream);
/* Copies phi on the leaf cells of every slot (nrhs x n_leaf_cells), or of
 * slots slot0 .. slot0 + nslots - 1, to `phi` (host: synchronises the
 * stream). */
int gmg_get_solution(gmg_tree *tree, double *phi, int where, void *stream);
int gmg_get_solution_slots(gmg_tree *tree, int slot0, int nslots, double *phi, int where, void *stream);

/* n_cycles FAS V-cycles in FP64 on every slot (Sec. 2.2: N_down sweeps,
 * restriction of phi and of the residual, coarse right-hand side
 * A phi + R r, exact coarse solve, (bi/tri)linear prolongation of the
 * correction, N_up sweeps). */
int gmg_vcycle(gmg_tree *tree, int n_cycles, void *stream);
/* n_cycles FMG cycles in FP64 on every slot (Sec. 2.2 "Multigrid cycle":
 * V-cycles from the coarsest grid up to the finest).  FAS form: residuals
 * and FAS right-hand sides are carried from the finest level to the
 * coarsest without smoothing, the coarsest level is solved exactly, then
 * for each finer level the coarse correction is prolonged to it and one
 * V-cycle (N_down / N_up sweeps) is done with that level on top. */
int gmg_fmg(gmg_tree *tree, int n_cycles, void *stream);
/* Composite residual ||b - A phi||_2 over leaf cells, relative to ||b||_2,
 * and max |b - A phi|, per unit (host arrays of nrhs * n_trees doubles, or
 * NULL).  Synchronises the stream. */
int gmg_residual(gmg_tree *tree, double *rel_l2, double *linf, void *stream);
/* The same composite residual as gmg_residual, for callers that cannot
 * allocate device memory: code that runs inside another runtime's memory
 * pool, allocation-free real-time loops, or plug-ins that may only use the
 * buffers they are handed.  The paper has no counterpart; this is a service
 * of the library.  `out` is a caller-owned device array of two doubles that
 * receives ||b - A phi||_2 / ||b||_2 (||r||_2 when b = 0) and max |b - A phi|;
 * the work is enqueued on `stream` and the call does not synchronise.  It
 * calls no cudaMalloc, cudaFree or allocating library routine: the per-block
 * partial sums live in one static device array of the library (3 MiB, held
 * on every device that loads the library until the process exits), which
 * limits the tree to 131072 blocks (larger trees: GMG_ERR_INVALID_ARG).
 * The first call on a device sets that device up: it looks up the device
 * addresses of that array and of a constant activity flag
 * (cudaGetSymbolAddress) and sets the kernels' shared-memory attributes, so
 * make it before any stream capture.  The call writes no state of the tree
 * (solves of the same tree on other streams are not disturbed).  All calls
 * share the array: calls that overlap on the GPU (several streams or host
 * threads at once) race and must be serialised by the caller.
 * With several right-hand-side slots it evaluates slot 0 (over all trees of
 * a forest together).
 * Errors: INVALID_ARG, STATE (tree not bound), CUDA. */
int gmg_residual_noalloc(gmg_tree *tree, double *out, void *stream);
/* Solves every unit (slot, tree) to ||b - A phi||_2 <= rel_tol ||b||_2 from
 * its current phi with GMG_FP64 V-cycles or GMG_MIXED / GMG_MIXED_BF16 defect
 * correction.  A
 * unit that reaches the tolerance is frozen: later cycles skip its blocks,
 * so its result does not depend on the other units.  stats: NULL or an
 * array of nrhs * n_trees entries.  Synchronises once per cycle (the
 * convergence test).
 * Errors: NOT_CONVERGED after max_cycles, NONFINITE on NaN or growth. */
int gmg_solve(gmg_tree *tree, int precision, double rel_tol, int max_cycles, gmg_stats *stats, void *stream);
/* gmg_solve with the residual history: the same loop, stopping and failure
 * rules, and device work per step, run through gmg_iterate.  history:
 * (max_cycles + 1) x (nrhs * n_trees) doubles, caller-owned, step-major:
 * history[k * units + u] is unit u's relative L2 residual after step k
 * (step 0: the first residual; a unit keeps its value once it has
 * converged), NaN after the last step.  stats as in gmg_solve.  Cite: the
 * residual-per-cycle curves of Sec. 4.  Synchronises once per step.
 * Errors: as gmg_solve (INVALID_ARG, STATE if not bound, NOT_CONVERGED,
 * NONFINITE); the history holds the steps run. */
int gmg_solve_history(gmg_tree *tree, int precision, double rel_tol, int max_cycles, double *history,
                      gmg_stats *stats, void *stream);
/* One step of the solve loop on the units with active[u] != 0 (host array
 * of nrhs * n_trees ints; the other units are left untouched): residual_only != 0 runs
 * the composite residual only (the first step of a new right-hand side; in
 * GMG_MIXED and GMG_MIXED_BF16 it also prepares the FP32 defect), else one
 * V-cycle (FP64) or one defect-correction step (GMG_MIXED, GMG_MIXED_BF16)
 * followed by the residual.  Writes
 * every unit's relative L2 and max residual into rel_l2 / linf (host arrays
 * of nrhs * n_trees doubles, or NULL; a unit not stepped keeps its last
 * values).
 * This is the unit a serving loop interleaves with gmg_set_rhs_slots.
 * Synchronises the stream. */
int gmg_iterate(gmg_tree *tree, int precision, const int *active, int residual_only, double *rel_l2, double *linf,
                void *stream);
/* gmg_iterate in two halves, so that steps of several trees (each on its
 * own stream) run on the device at the same time: _begin enqueues the step
 * (it waits only for this tree's previous work on `stream`), _end waits for
 * it and reads the norms.  A tree holds at most one step in flight.
 * Errors: STATE for _begin with a step in flight or _end without one. */
int gmg_iterate_begin(gmg_tree *tree, int precision, const int *active, int residual_only, void *stream);
int gmg_iterate_end(gmg_tree *tree, double *rel_l2, double *linf);

/* Field E = -grad(phi) on the upper faces of every leaf cell (Sec. 4.4: the
 * components of grad(phi) on a staggered grid, taking the stored boundary
 * distances into account): for axis k of leaf cell i, the face i + 1/2 e_k.
 * Where the irregular boundary lies between i and its +k neighbour at
 * relative distance d < 1 the gradient is (phi_b - phi_i) / (d dx); at a
 * Dirichlet domain wall 2 (phi_w - phi_i) / dx, at a Neumann wall 0;
 * elsewhere (phi_neighbour - phi_i) / dx with the operator's ghost value
 * (same-level neighbour or refinement-boundary ghost).  Cells whose centre
 * lies inside the object get E = 0.  out: nrhs x n_leaf_cells x dim
 * doubles (leaf-cell order, components x fastest), host or device by
 * `where` (host: synchronises the stream). */
int gmg_efield(gmg_tree *tree, double *out, int where, void *stream);

/* Inspection (tests, tools): phi (which = 0) or b (which = 1) of every cell
 * of a level in canonical block order, FP64 host array; distances d
 * (nb * N^D * 2D) and mask flags (nb * N^D) of a level. */
int gmg_get_level(gmg_tree *tree, int level, int which, double *out, void *stream);
int gmg_get_distances(const gmg_tree *tree, int level, double *out);
int gmg_get_mask(const gmg_tree *tree, int level, int *out);
int gmg_num_cut_blocks(const gmg_tree *tree, int level);
/* Cut lists of a level (host, after gmg_store_stencils): for block i of the
 * level in canonical order, counts[2i] and counts[2i+1] receive how many of
 * its cells of colour 0 ((x+y+z) even) and colour 1 have a stencil that
 * differs from the regular one (some d < 1, Sec. 3.3); the kernels keep those
 * cells and their coefficients in per-colour lists.  counts: 2 * (blocks of
 * the level) ints, caller-owned. */
int gmg_cut_counts(const gmg_tree *tree, int level, int *counts);
/* Right-hand-side boundary terms of a level (host, after gmg_store_stencils):
 * nb * N^D values in canonical block order (0 for blocks without any), the
 * term subtracted from the source g of each leaf cell. */
int gmg_get_boundary_terms(const gmg_tree *tree, int level, double *out);

/* Number of kernels the last gmg_vcycle / gmg_solve call enqueued. */
long long gmg_last_launch_count(const gmg_tree *tree);

/* Kernel timing: while enabled, every kernel the tree enqueues is bracketed
 * by CUDA events on its stream.  gmg_profile_read synchronises, aggregates
 * the recorded launches per (kernel kind, precision, level) into the caller's
 * arrays (up to `cap` entries: kind, prec 0 = FP64 / 1 = FP32 / 2 = FP32
 * arithmetic on BF16 storage (GMG_MIXED_BF16's finest level), level,
 * launches, total milliseconds), clears the record and returns the number of
 * entries (or a negative error).  Kinds: 0 smooth, 1 residual+restrict,
 * 2 FAS right-hand side, 3 coarse solve, 4 prolongation, 5 restriction of
 * phi, 6 residual norm, 7 norm reduction, 8 mixed-path accumulation,
 * 9 right-hand side / copies, 10 bottom of the cycle on a thread-block
 * cluster (GMG_OPT_CLUSTER_TAIL), 11 down leg and 12 up leg of a level in one
 * cooperative launch (GMG_OPT_LEVEL_LEGS). */
int gmg_profile_enable(gmg_tree *tree, int enable);
int gmg_profile_read(gmg_tree *tree, int cap, int *kind, int *prec, int *level, long long *launches, double *ms);

/* Execution options (defaults in brackets): GMG_OPT_GRAPHS [1] replays the
 * solve phases as captured CUDA graphs; GMG_OPT_COARSE_COOP [1] runs the
 * levels with at most 160 blocks and the coarse solve in one cooperative
 * launch with grid barriers; GMG_OPT_SPIN_LIMIT [2^24] bounds the polls of
 * such a barrier (about 100 ns each) before it records GMG_ERR_TIMEOUT.
 * Results are identical with every setting. */
#define GMG_OPT_GRAPHS 1
#define GMG_OPT_COARSE_COOP 2
#define GMG_OPT_SPIN_LIMIT 3
#define GMG_OPT_FUSED_SWEEPS 4 /* [0] FP32 levels without refinement boundaries: all N_down (N_up)
                                  half-sweeps of a visit in one pass over a tile with a halo */
#define GMG_OPT_CTA_THREADS 5  /* [0] threads per CTA of the smoothing, residual, restriction and
                                  FAS kernels: 64, 128 or 256; 0 = 64 for blocks of at most 512
                                  cells, 256 otherwise */
#define GMG_OPT_COOP_MAX_BLOCKS 6 /* [160] levels with at most this many blocks (from the coarsest
                                     up to the last such level) join the cooperative launch */
#define GMG_OPT_INNER_CYCLES 7   /* [1] FP32 V-cycles per defect-correction step of GMG_MIXED
                                    (1 .. 8): more cycles per FP64 residual, fewer steps */
#define GMG_OPT_FMG_STEPS 9      /* [0] each step of gmg_solve / gmg_iterate is an FMG cycle (FP64,
                                    or the FP32 inner cycles of GMG_MIXED) instead of a V-cycle */
#define GMG_OPT_SLOTS_PER_CTA 8  /* [1] with several slots, the half-sweeps of 8^3 / 16^3 blocks
                                    stage and update 1, 2 or 4 slots of a block per CTA (the
                                    block's tables and index arithmetic shared); same results */
#define GMG_OPT_PDL 10           /* [1] the per-level kernels of a solve step are launched with
                                    programmatic dependent launch: each is dispatched as its
                                    predecessor's CTAs exit and waits for it on the device before
                                    reading its results; same results */
#define GMG_OPT_CLUSTER_TAIL 11  /* [1] the bottom of the V-cycle (the levels holding one block per
                                    root, and the level of each root's 2^D children when it is
                                    complete) on a cluster of CTAs per (root, slot) (4 in 2D; 8 or
                                    16 in 3D, GMG_OPT_CLUSTER_PARTS), each CTA holding one part of
                                    every such level in shared memory and writing its neighbours'
                                    ghost cells through distributed shared memory: 0 off (one CTA
                                    per (root, slot) inside the cooperative launch), 1 when every
                                    unit's cluster is resident at once, 2 whenever the tree
                                    qualifies (parts of even side, within one CTA's shared
                                    memory); same arithmetic */
#define GMG_OPT_DEVICE_SETUP 12  /* [1] gmg_store_stencils with a built-in sphere, capsule or ellipsoid
                                    level set runs the boundary mask, the line searches and the
                                    unresolved-root search on the device when a CUDA device is
                                    present (the same values bit for bit); 0 on the host.  Set it
                                    before gmg_store_stencils. */
#define GMG_OPT_CLUSTER_PARTS 13 /* [0] CTAs of the 3D cluster of GMG_OPT_CLUSTER_TAIL: 8 (octants of
                                    N/2 cells a side), 16 (parts of N/2 x N/2 x N/4; non-portable
                                    cluster size, split levels' sides multiples of 8), or 0: 16
                                    when the tree and the device allow it, else 8; same arithmetic */
#define GMG_OPT_LEVEL_LEGS 14    /* [0] a level whose (block, slot) CTAs fit on the GPU at once (256
                                    threads, four per SM: the 512 blocks of a 128^3 tree in 16^3
                                    blocks) runs its down leg (sweeps, residual and restriction) and
                                    its up leg (prolongation, sweeps) as one cooperative launch each,
                                    with a grid barrier between the phases; same results bit for bit
                                    (half the launches, the same solve time on the 128^3 sphere) */
int gmg_set_option(gmg_tree *tree, int option, long long value);

/* Sweep schedule: N_down / N_up red-black sweeps on one level (default: the
 * parameters' n_down / n_up on every level; the coarsest level is solved
 * exactly and ignores them).  A schedule that differs from level to level
 * is a tuning choice outside the paper's uniform N_down / N_up: it changes
 * the V-cycle (and its convergence rate), not the discretisation or the
 * solution it converges to.  Before or after gmg_tree_bind.
 * Errors: INVALID_ARG for a level out of range or counts outside 0..64. */
int gmg_set_level_sweeps(gmg_tree *tree, int level, int n_down, int n_up);
int gmg_get_level_sweeps(const gmg_tree *tree, int level, int *n_down, int *n_up);

/* Failure-detection self test: launches a cooperative kernel whose grid
 * barrier waits for one CTA more than exist, so its bounded wait must run
 * out.  Synchronises the stream; returns GMG_ERR_TIMEOUT when the wait ended
 * as designed (the context stays usable), GMG_OK if it did not. */
int gmg_selftest_barrier_timeout(gmg_tree *tree, long long spin_limit, void *stream);

/* Self test of the integer-operation conversions that the FP64 residual and
 * the FP64 update of the mixed path use (double -> float rounded to nearest
 * even, float -> double): converts the n doubles x and the n floats f (device
 * arrays) both ways and by the hardware, and writes to mismatches[0] and
 * mismatches[1] (device array of 2, overwritten) how many results differ bit
 * for bit.  Synchronises the stream.  Errors: INVALID_ARG for null arrays or
 * n < 0; CUDA on a failed launch. */
int gmg_selftest_conversions(const double *x, const float *f, long long n, unsigned long long *mismatches,
                             void *stream);

const char *gmg_error_string(int code);
const char *gmg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
