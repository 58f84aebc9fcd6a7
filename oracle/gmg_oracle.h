/*
 * Serial FP64 oracle for the octree geometric-multigrid Poisson solver with
 * level-set Dirichlet boundaries (Teunissen & Schiavello, "Geometric multigrid
 * method for solving Poisson's equation on octree grids with irregular
 * boundaries", arXiv 2205.09411).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, obviously
 * correct reference against which the CUDA library is checked.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg load it; the
 * CUDA library shares no code, header, table or helper with it.
 *
 * Every function below follows one passage of the paper:
 *   mesh of N^D-cell blocks, 2:1 balance ............ Sec. 2.1
 *   5/7-point Laplacian, residual ................... Sec. 2.2, Eq. (lpl-1d), Eq. (residual)
 *   red-black Gauss-Seidel .......................... Sec. 2.2 "Smoother"
 *   restriction (mean) / prolongation (linear) ...... Sec. 2.2, Sec. 3.4
 *   FAS V-cycle, N_down = N_up = 2 .................. Sec. 2.2 "Multigrid cycle"
 *   refinement-boundary ghost cells ................. Sec. 2.2 "Ghost cells"
 *   level-set function .............................. Sec. 3.1, Eq. (lsf-example)
 *   relative distance, bisection, golden section .... Sec. 3.2, Eq. (relative-distance)
 *   cut-cell Laplacian, boundary term to the RHS .... Sec. 3.3, Eqs. (lpl-1d-lsf), (lpl-2d-lsf)
 *   coarse-grid direct solve ........................ Sec. 3.5 (replaces the paper's Hypre solve)
 *   boundary-detection mask ......................... Sec. 3.6.1, Eq. (boundary-mask)
 *   stored stencils and moved-coefficient sums ...... Sec. 3.6.2
 *   unresolved roots on coarse grids ................ Sec. 3.6.3
 *
 * Where the paper is silent or ambiguous the oracle takes the readings listed
 * at the top of gmg_oracle.c.
 *
 * Parity pins: see the comment above each exported function; the only
 * function without an independent pin is the per-V-cycle convergence rate
 * (parity unpinned: the paper prints per-FMG ranges only).
 */
#ifndef GMG_ORACLE_H
#define GMG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef double (*ot_fn)(const double *x, void *user);
typedef int (*ot_refine_fn)(int level, const int *bix, void *user);

/* level-set function kinds (Sec. 3.1; shapes of Sec. 4) */
enum {
  OT_LSF_NONE = 0,      /* no irregular boundary                                  */
  OT_LSF_SPHERE = 1,    /* p[0..2] centre, p[3] radius: |x-c| - R, Eq. (lsf-example) */
  OT_LSF_CAPSULE = 2,   /* p[0..2] a, p[3..5] b, p[6] r: dist(x, segment ab) - r   */
  OT_LSF_ELLIPSOID = 3, /* p[0..2] c, p[3..11] Q row-major, p[12..14] semi-axes     */
  OT_LSF_CALLBACK = 4,  /* user function                                          */
  OT_LSF_SHAPE = 5,     /* Sec. 4.3 shapes: p[0] 0 spheroid, 1 rhombus, 2 heart, 3 astroid;
                           p[1] = 1: revolved about the z axis (3D)                */
  OT_LSF_GRID = 6       /* samples on a uniform grid (user: doubles, x fastest), the
                           (bi/tri)linear interpolant; p[0..2] counts, p[3..5] sample 0,
                           p[6..8] spacing; outside the box: the nearest face      */
};

typedef struct {
  int kind;
  double p[16];
  ot_fn fn;
  void *user;
} ot_lsf;

enum { OT_WALL_DIRICHLET = 0, OT_WALL_NEUMANN = 1 };

typedef struct ot_tree ot_tree;

/* Build the block tree (Sec. 2.1): cb[d] root blocks of N^D cells at level 1,
 * cell size h1 on level 1; refine(level, bix) decides which blocks get 2^D
 * children up to max_level (refine == NULL refines every block: a uniform
 * tree); then the tree is closed under 2:1 balance over
 * faces, edges and corners.  Levels below 1 coarsen inside the root blocks
 * while the level holds more than max_coarse_cells cells. */
ot_tree *ot_create(int dim, int N, const int *cb, const double *lo, double h1,
                   int max_level, ot_refine_fn refine, void *ruser,
                   int max_coarse_cells);
void ot_destroy(ot_tree *T);

void ot_levels(const ot_tree *T, int *lmin, int *lmax);
int ot_level_nblocks(const ot_tree *T, int level);
int ot_level_n(const ot_tree *T, int level);
double ot_level_h(const ot_tree *T, int level);
/* canonical order: blocks of a level sorted by Morton code of their coordinates */
void ot_level_blocks(const ot_tree *T, int level, int *bix /* nb*3 */, int *has_children);
int64_t ot_num_leaf_cells(const ot_tree *T);
/* leaf cells: leaf blocks by (level, Morton), cells x-fastest inside a block */
void ot_leaf_centers(const ot_tree *T, double *xyz /* nleaf*dim */);
void ot_leaf_levels(const ot_tree *T, int *lev);

void ot_set_params(ot_tree *T, int n_down, int n_up, double eps_tol,
                   double mask_factor, double w_min);
void ot_set_walls(ot_tree *T, const int *type /* 2*dim */, const double *value,
                  ot_fn fn, void *user);
void ot_set_lsf(ot_tree *T, const ot_lsf *lsf);
/* Sec. 3.2, 3.3, 3.6: mask, line searches, cut stencils, boundary terms and
 * the coarse-level matrix.  phib_fn may be NULL (then phib_const is used). */
int ot_store_stencils(ot_tree *T, ot_fn phib_fn, void *user, double phib_const);
int ot_num_cut_blocks(const ot_tree *T, int level);

/* b = g - (moved boundary terms) - (Dirichlet wall terms) on leaf cells */
void ot_set_rhs(ot_tree *T, const double *g);
void ot_set_solution(ot_tree *T, const double *phi);
void ot_get_solution(const ot_tree *T, double *phi);
void ot_get_level(const ot_tree *T, int level, int which /*0 phi,1 b*/, double *out);
void ot_vcycle(ot_tree *T, int n);
/* n FMG cycles (Sec. 2.2 "Multigrid cycle"; reading FMG).  Pin: after two
 * cycles from phi = 0 the error against the analytic sphere solution is
 * that of the converged discrete solution (Sec. 4.1: the discretisation
 * error dominates after two FMG iterations). */
void ot_fmg(ot_tree *T, int n);
/* E = -grad(phi) on the upper face of every leaf cell (Sec. 4.4), leaf
 * cells x D.  Pin: -a exactly for phi = a.x + c. */
void ot_efield(ot_tree *T, double *out);
/* composite residual over leaf cells: returns ||r||_2; linf, bnorm optional */
double ot_residual(ot_tree *T, double *linf, double *bnorm, double *r_out);
int ot_solve(ot_tree *T, double rel_tol, int max_cycles, double *hist);

/* --- pieces exposed for the pins ------------------------------------- */
double ot_line_search(ot_fn f, void *user, int dim, const double *a,
                      const double *b, double eps_tol);
double ot_lsf_eval(const ot_lsf *lsf, int dim, const double *x);
/* per-level distances: nb*n^D*2D, canonical order (1 for uncut cells) */
void ot_get_d(const ot_tree *T, int level, double *out);
/* per-level mask flags nb*n^D */
void ot_get_mask(const ot_tree *T, int level, int *out);
/* full operator incl. boundary terms: out = A phi + bterm on leaf cells,
 * phi given on leaf cells (covered cells restricted first) */
void ot_apply_composite(ot_tree *T, const double *phi, double *out, int with_bterm);
/* dense composite matrix on leaf cells (column j = A e_j) and the rhs b */
int ot_composite_matrix(ot_tree *T, double *A, double *b);
/* prolong a correction given on level l-1 (canonical) into level l (zero
 * initial) and return level l values */
void ot_prolong_test(ot_tree *T, int level, const double *coarse, double *fine);
/* restrict level l values into level l-1 covered cells, return level l-1 */
void ot_restrict_test(ot_tree *T, int level, const double *fine, double *coarse);
/* one red (color 0) or black (1) half-sweep on a level (Sec. 2.2) */
void ot_halfsweep(ot_tree *T, int level, int color);
/* r = b - A phi on every cell of a level (canonical order) */
void ot_level_residual(ot_tree *T, int level, double *out);
/* overwrite phi (which 0) or b (which 1) of a level (canonical order) */
void ot_set_level(ot_tree *T, int level, int which, const double *in);
/* dense LU solve with partial pivoting (coarse-grid solver) */
int ot_lu_solve(int n, const double *A, const double *b, double *x);

#ifdef __cplusplus
}
#endif
#endif
