/*
 * Serial FP64 oracle for the octree geometric-multigrid Poisson solver with
 * level-set Dirichlet boundaries (arXiv 2205.09411).  TEST INFRASTRUCTURE
 * ONLY: it exists so that the CUDA library can be checked against a plain,
 * slow, obviously correct implementation written from the paper.  It shares
 * no code with the CUDA library.  Build: gcc -O2 -ffp-contract=off -shared.
 *
 * Readings taken where the paper is silent, ambiguous or garbled:
 *  S   GSRB update: the printed 1D update has "+dx^2 g", which contradicts
 *      Eq. (lpl-1d); the update used is phi_i = (b_i - sum_j c_ij phi_j)/c_ii.
 *  SW  one smoothing step = ghost fill, red half-sweep, ghost fill, black
 *      half-sweep; red = even (i+j[+k]) in global cell indices of the level;
 *      ghost values are those filled before the half-sweep.
 *  UP  on the way up a level is smoothed N_up times after receiving its
 *      correction (so the finest level is post-smoothed).
 *  G   refinement-boundary ghost: g = f/3 + 2/3 * c_hat, f the adjacent fine
 *      cell, c_hat the coarse cell containing the ghost centre shifted by
 *      unlimited central tangential slopes (+-1/4 coarse cell).  Exact for
 *      linear phi; averaged fine and coarse fluxes then agree for linear phi.
 *  W   domain walls: Dirichlet ghost = 2 phi_w - phi_i, Neumann-0 ghost =
 *      phi_i.  The operator is kept linear (homogeneous ghosts -phi_i /
 *      +phi_i) and the inhomogeneous part 2 c phi_w goes to the right-hand
 *      side, like the moved cut-cell coefficients of Sec. 3.3.  Edge/corner
 *      ghosts outside the domain compose the per-axis reflections.
 *  IN  every cell is an unknown, also inside the object.
 *  D0  d is clamped to [eps_tol, 1].
 *  BS  bisection on t in [0, t_hi] along a->b, halving while the bracket is
 *      at least eps_tol wide; the bracket midpoint is returned.
 *  GS  golden-section minimisation of f(a) f(a + t(b-a)) on [0,1] while the
 *      interval is at least eps_tol wide; every new point with
 *      f(a) f(x) <= 0 ends the search and bisection runs on [0, t_x].
 *  M   mask gradient: central differences with step dx; descent gradient:
 *      step w_min; at most floor(dx/w_min) steps; "neighbour closest to x" =
 *      axis of the largest |x_k - a_k|, lowest axis on ties; applied only if
 *      that neighbour lies inside the domain.  No line search is made toward
 *      a neighbour centre outside the domain (the wall rule applies there).
 *  BV  both the moved-coefficient sum and the boundary term sum c*phi_b(x0)
 *      are stored, x0 being the located root.
 *  C   coarse level: exact solve (LU, partial pivoting) on a level made by
 *      coarsening inside the root blocks until it holds at most
 *      max_coarse_cells cells.
 *  P   prolongation edge/corner coarse values come from diagonal neighbours
 *      on the same level (all exist under the face/edge/corner 2:1 balance)
 *      or from the wall reflections.
 *  R   stop on ||b - A phi||_2 / ||b||_2 over leaf cells.
 *  V   a V-cycle ends by restricting phi into covered cells, so that the
 *      composite operator sees covered values equal to the mean of their
 *      children (no effect on the iterates of a uniform tree).
 *  FMG an FMG cycle carries residuals and FAS right-hand sides from the
 *      finest level to the coarsest without smoothing, solves the coarsest
 *      level, then for each finer level prolongs the coarse correction and
 *      does one V-cycle with that level on top (which ends with reading V
 *      up to that level).
 */
#include "gmg_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define LOFF 32 /* level l is stored at index l + LOFF */
#define NLEV 64

typedef struct {
  int level, ix[3], n;
  int parent, pofs[3];
  int child[8], has_children;
  double *phi, *b, *old, *r, *tmp, *gh;
  int cut;
  double *st;  /* n^D x (2D+1): diag, (-x,+x), (-y,+y), (-z,+z) */
  double *bnd; /* sum of moved c * phi_b */
  double *smv; /* sum of moved c */
  double *dd;  /* n^D x 2D distances (cut blocks only) */
  double *bterm;
  unsigned char *mask;
} OB;

struct ot_tree {
  int D, N, cb[3], max_level, lmin, lmax, max_coarse;
  double lo[3], h1;
  int nb, cap;
  OB *B;
  int lev_cnt[NLEV], lev_cap[NLEV];
  int *lev_list[NLEV];
  int *lev_map[NLEV];
  /* parameters (Sec. 2.2, 3.2, 3.6) */
  int n_down, n_up;
  double eps_tol, mask_factor, w_min;
  int wall_type[6];
  double wall_val[6];
  ot_fn wall_fn;
  void *wall_user;
  ot_lsf lsf;
  int have_lsf;
  /* boundary value on the object (gmg_store_stencils' phi_b) */
  ot_fn phib_fn;
  void *phib_user;
  double phib_const;
  /* coarse level LU factors */
  int nc;
  double *lu;
  int *piv;
  int stencils_ready;
};

/* ------------------------------------------------------------------ */
/* level geometry (Sec. 2.1)                                           */
/* ------------------------------------------------------------------ */
static int lvl_n(const ot_tree *T, int l) { return l >= 1 ? T->N : (T->N >> (1 - l)); }
static double lvl_h(const ot_tree *T, int l) { return ldexp(T->h1, 1 - l); }
static void lvl_bext(const ot_tree *T, int l, int e[3]) {
  for (int d = 0; d < 3; d++)
    e[d] = d < T->D ? (l >= 1 ? T->cb[d] << (l - 1) : T->cb[d]) : 1;
}
static void lvl_cext(const ot_tree *T, int l, int e[3]) {
  lvl_bext(T, l, e);
  for (int d = 0; d < T->D; d++) e[d] *= lvl_n(T, l);
}
static int ncell(const ot_tree *T, int n) { return T->D == 3 ? n * n * n : n * n; }
static int nghost(const ot_tree *T, int n) { return T->D == 3 ? (n + 2) * (n + 2) * (n + 2) : (n + 2) * (n + 2); }
static int cidx(int n, const int p[3]) { return p[0] + n * (p[1] + n * p[2]); }
static int gidx(const ot_tree *T, int n, const int p[3]) {
  int m = n + 2;
  return (p[0] + 1) + m * ((p[1] + 1) + (T->D == 3 ? m * (p[2] + 1) : 0));
}

static int map_find(const ot_tree *T, int l, const int bix[3]) {
  int e[3];
  lvl_bext(T, l, e);
  for (int d = 0; d < 3; d++)
    if (bix[d] < 0 || bix[d] >= e[d]) return -1;
  int *m = T->lev_map[l + LOFF];
  if (!m) return -1;
  return m[bix[0] + e[0] * (bix[1] + e[1] * bix[2])];
}

static void lev_ensure_map(ot_tree *T, int l) {
  if (T->lev_map[l + LOFF]) return;
  int e[3];
  lvl_bext(T, l, e);
  size_t sz = (size_t)e[0] * e[1] * e[2];
  int *m = (int *)malloc(sz * sizeof(int));
  for (size_t i = 0; i < sz; i++) m[i] = -1;
  T->lev_map[l + LOFF] = m;
}

static int new_block(ot_tree *T, int l, const int bix[3], int parent, const int pofs[3]) {
  if (T->nb == T->cap) {
    T->cap = T->cap ? 2 * T->cap : 64;
    T->B = (OB *)realloc(T->B, (size_t)T->cap * sizeof(OB));
  }
  int id = T->nb++;
  OB *B = &T->B[id];
  memset(B, 0, sizeof(OB));
  B->level = l;
  for (int d = 0; d < 3; d++) {
    B->ix[d] = bix[d];
    B->pofs[d] = pofs[d];
  }
  B->n = lvl_n(T, l);
  B->parent = parent;
  for (int c = 0; c < 8; c++) B->child[c] = -1;
  int li = l + LOFF;
  if (T->lev_cnt[li] == T->lev_cap[li]) {
    T->lev_cap[li] = T->lev_cap[li] ? 2 * T->lev_cap[li] : 16;
    T->lev_list[li] = (int *)realloc(T->lev_list[li], (size_t)T->lev_cap[li] * sizeof(int));
  }
  T->lev_list[li][T->lev_cnt[li]++] = id;
  lev_ensure_map(T, l);
  int e[3];
  lvl_bext(T, l, e);
  T->lev_map[li][bix[0] + e[0] * (bix[1] + e[1] * bix[2])] = id;
  return id;
}

/* Sec. 2.1: refining a block creates its 2^D children (half the spacing). */
static void refine_block(ot_tree *T, int id) {
  if (T->B[id].has_children) return;
  int D = T->D, nch = 1 << D;
  for (int o = 0; o < nch; o++) {
    OB *P = &T->B[id];
    int bix[3] = {0, 0, 0}, pofs[3] = {0, 0, 0};
    for (int d = 0; d < D; d++) {
      int bit = (o >> d) & 1;
      bix[d] = 2 * P->ix[d] + bit;
      pofs[d] = bit * (P->n / 2);
    }
    int l = P->level + 1;
    int c = new_block(T, l, bix, id, pofs);
    T->B[id].child[o] = c; /* T->B may have moved */
  }
  T->B[id].has_children = 1;
}

/* make block (l, bix) exist, refining coarser blocks as needed */
static void ensure_block(ot_tree *T, int l, const int bix[3]) {
  if (map_find(T, l, bix) >= 0) return;
  int pb[3] = {bix[0] >> 1, bix[1] >> 1, bix[2] >> 1};
  ensure_block(T, l - 1, pb);
  refine_block(T, map_find(T, l - 1, pb));
}

static uint64_t morton(const int b[3], int D) {
  uint64_t m = 0;
  for (int bit = 0; bit < 21; bit++)
    for (int d = 0; d < D; d++) m |= (uint64_t)((b[d] >> bit) & 1) << (bit * D + d);
  return m;
}

static const ot_tree *sort_T;
static int cmp_morton(const void *a, const void *b) {
  const OB *A = &sort_T->B[*(const int *)a], *B = &sort_T->B[*(const int *)b];
  uint64_t ma = morton(A->ix, sort_T->D), mb = morton(B->ix, sort_T->D);
  return ma < mb ? -1 : (ma > mb ? 1 : 0);
}

ot_tree *ot_create(int dim, int N, const int *cb, const double *lo, double h1, int max_level,
                   ot_refine_fn refine, void *ruser, int max_coarse_cells) {
  if (dim < 2 || dim > 3 || N < 2 || (N & 1) || max_level < 1 || max_level > 20) return NULL;
  ot_tree *T = (ot_tree *)calloc(1, sizeof(ot_tree));
  T->D = dim;
  T->N = N;
  for (int d = 0; d < 3; d++) {
    T->cb[d] = d < dim ? cb[d] : 1;
    T->lo[d] = d < dim ? lo[d] : 0.0;
  }
  T->h1 = h1;
  T->max_level = max_level;
  T->max_coarse = max_coarse_cells;
  T->n_down = 2;
  T->n_up = 2;
  T->eps_tol = 1e-8;
  T->mask_factor = 1.5;
  T->w_min = 0.0;
  for (int w = 0; w < 6; w++) T->wall_type[w] = OT_WALL_DIRICHLET;

  /* level 1: the root grid */
  int e[3];
  lvl_bext(T, 1, e);
  int zero[3] = {0, 0, 0};
  for (int z = 0; z < e[2]; z++)
    for (int y = 0; y < e[1]; y++)
      for (int x = 0; x < e[0]; x++) {
        int bix[3] = {x, y, z};
        new_block(T, 1, bix, -1, zero);
      }
  /* refinement decided level by level by the callback */
  for (int l = 1; l < max_level; l++) {
    int cnt = T->lev_cnt[l + LOFF];
    for (int i = 0; i < cnt; i++) {
      int id = T->lev_list[l + LOFF][i];
      int bix[3] = {T->B[id].ix[0], T->B[id].ix[1], T->B[id].ix[2]};
      if (!refine || refine(l, bix, ruser)) refine_block(T, id);
    }
  }
  /* 2:1 balance over faces, edges and corners (Sec. 2.1): every block at
   * level l needs the level l-1 blocks covering all its neighbour regions */
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int l = max_level; l >= 2; l--) {
      int cnt = T->lev_cnt[l + LOFF];
      lvl_bext(T, l, e);
      for (int i = 0; i < cnt; i++) {
        int id = T->lev_list[l + LOFF][i];
        int z0 = dim == 3 ? -1 : 0, z1 = dim == 3 ? 1 : 0;
        for (int dz = z0; dz <= z1; dz++)
          for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
              int q[3] = {T->B[id].ix[0] + dx, T->B[id].ix[1] + dy, T->B[id].ix[2] + dz};
              if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= e[0] || q[1] >= e[1] || q[2] >= e[2]) continue;
              int p[3] = {q[0] >> 1, q[1] >> 1, q[2] >> 1};
              if (map_find(T, l - 1, p) < 0) {
                ensure_block(T, l - 1, p);
                changed = 1;
              }
            }
      }
    }
  }
  T->lmax = 1;
  for (int l = 1; l <= max_level; l++)
    if (T->lev_cnt[l + LOFF] > 0) T->lmax = l;
  /* coarse levels inside the root blocks (reading C) */
  T->lmin = 1;
  for (;;) {
    int l = T->lmin, n = lvl_n(T, l);
    long cells = (long)T->lev_cnt[l + LOFF] * ncell(T, n);
    if (cells <= max_coarse_cells || (n & 1) || n / 2 < 2) break;
    int cnt = T->lev_cnt[l + LOFF];
    for (int i = 0; i < cnt; i++) {
      int id = T->lev_list[l + LOFF][i];
      int bix[3] = {T->B[id].ix[0], T->B[id].ix[1], T->B[id].ix[2]};
      int pid = new_block(T, l - 1, bix, -1, zero);
      T->B[id].parent = pid;
      for (int d = 0; d < 3; d++) T->B[id].pofs[d] = 0;
      T->B[pid].child[0] = id;
      T->B[pid].has_children = 1;
    }
    T->lmin = l - 1;
  }
  /* canonical order and storage */
  sort_T = T;
  for (int l = T->lmin; l <= T->lmax; l++)
    qsort(T->lev_list[l + LOFF], (size_t)T->lev_cnt[l + LOFF], sizeof(int), cmp_morton);
  for (int i = 0; i < T->nb; i++) {
    OB *B = &T->B[i];
    int nc = ncell(T, B->n);
    B->phi = (double *)calloc((size_t)nc, sizeof(double));
    B->b = (double *)calloc((size_t)nc, sizeof(double));
    B->old = (double *)calloc((size_t)nc, sizeof(double));
    B->r = (double *)calloc((size_t)nc, sizeof(double));
    B->tmp = (double *)calloc((size_t)nc, sizeof(double));
    B->gh = (double *)calloc((size_t)nghost(T, B->n), sizeof(double));
  }
  return T;
}

static void free_stencil(OB *B) {
  free(B->st);
  free(B->bnd);
  free(B->smv);
  free(B->dd);
  free(B->bterm);
  free(B->mask);
  B->st = B->bnd = B->smv = B->dd = B->bterm = NULL;
  B->mask = NULL;
  B->cut = 0;
}

void ot_destroy(ot_tree *T) {
  if (!T) return;
  for (int i = 0; i < T->nb; i++) {
    OB *B = &T->B[i];
    free(B->phi);
    free(B->b);
    free(B->old);
    free(B->r);
    free(B->tmp);
    free(B->gh);
    free_stencil(B);
  }
  for (int l = 0; l < NLEV; l++) {
    free(T->lev_list[l]);
    free(T->lev_map[l]);
  }
  free(T->B);
  free(T->lu);
  free(T->piv);
  free(T);
}

void ot_levels(const ot_tree *T, int *lmin, int *lmax) {
  *lmin = T->lmin;
  *lmax = T->lmax;
}
int ot_level_nblocks(const ot_tree *T, int level) {
  if (level < T->lmin || level > T->lmax) return 0;
  return T->lev_cnt[level + LOFF];
}
int ot_level_n(const ot_tree *T, int level) { return lvl_n(T, level); }
double ot_level_h(const ot_tree *T, int level) { return lvl_h(T, level); }
void ot_level_blocks(const ot_tree *T, int level, int *bix, int *has_children) {
  int cnt = ot_level_nblocks(T, level);
  for (int i = 0; i < cnt; i++) {
    const OB *B = &T->B[T->lev_list[level + LOFF][i]];
    for (int d = 0; d < 3; d++) bix[3 * i + d] = B->ix[d];
    if (has_children) has_children[i] = B->has_children;
  }
}

#define FOR_LEAF_BLOCKS(T, l, i, B)                                   \
  for (int l = (T)->lmin; l <= (T)->lmax; l++)                        \
    for (int i = 0; i < (T)->lev_cnt[l + LOFF]; i++)                  \
      for (OB *B = &(T)->B[(T)->lev_list[l + LOFF][i]]; B; B = NULL)  \
        if (!B->has_children)

#define FOR_CELLS(T, n, p)                                            \
  for (int p##z = 0; p##z < ((T)->D == 3 ? (n) : 1); p##z++)          \
    for (int p##y = 0; p##y < (n); p##y++)                            \
      for (int p##x = 0; p##x < (n); p##x++)                          \
        for (int p[3] = {p##x, p##y, p##z}, p##once = 1; p##once; p##once = 0)

int64_t ot_num_leaf_cells(const ot_tree *T) {
  int64_t s = 0;
  FOR_LEAF_BLOCKS(T, l, i, B) s += ncell(T, B->n);
  return s;
}

static void cell_center(const ot_tree *T, const OB *B, const int p[3], double x[3]) {
  double h = lvl_h(T, B->level);
  for (int d = 0; d < 3; d++) {
    if (d < T->D)
      x[d] = T->lo[d] + ((double)(B->ix[d] * B->n + p[d]) + 0.5) * h;
    else
      x[d] = 0.0;
  }
}

void ot_leaf_centers(const ot_tree *T, double *xyz) {
  int64_t k = 0;
  FOR_LEAF_BLOCKS(T, l, i, B) {
    FOR_CELLS(T, B->n, p) {
      double x[3];
      cell_center(T, B, p, x);
      for (int d = 0; d < T->D; d++) xyz[k * T->D + d] = x[d];
      k++;
    }
  }
}

void ot_leaf_levels(const ot_tree *T, int *lev) {
  int64_t k = 0;
  FOR_LEAF_BLOCKS(T, l, i, B) {
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc; c++) lev[k++] = B->level;
  }
}

void ot_set_params(ot_tree *T, int n_down, int n_up, double eps_tol, double mask_factor, double w_min) {
  T->n_down = n_down;
  T->n_up = n_up;
  T->eps_tol = eps_tol;
  T->mask_factor = mask_factor;
  T->w_min = w_min;
}

void ot_set_walls(ot_tree *T, const int *type, const double *value, ot_fn fn, void *user) {
  for (int w = 0; w < 2 * T->D; w++) {
    T->wall_type[w] = type[w];
    T->wall_val[w] = value ? value[w] : 0.0;
  }
  T->wall_fn = fn;
  T->wall_user = user;
}

void ot_set_lsf(ot_tree *T, const ot_lsf *lsf) {
  T->lsf = *lsf;
  T->have_lsf = lsf->kind != OT_LSF_NONE;
}

/* ------------------------------------------------------------------ */
/* level-set functions (Sec. 3.1, Eq. (lsf-example))                   */
/* ------------------------------------------------------------------ */
double ot_lsf_eval(const ot_lsf *L, int D, const double *x) {
  const double *p = L->p;
  switch (L->kind) {
  case OT_LSF_SPHERE: {
    double s = 0.0;
    for (int d = 0; d < D; d++) {
      double t = x[d] - p[d];
      s = s + t * t;
    }
    return sqrt(s) - p[3];
  }
  case OT_LSF_CAPSULE: {
    /* distance to the segment a->b minus the radius */
    double ab[3], ax[3], num = 0.0, den = 0.0;
    for (int d = 0; d < D; d++) {
      ab[d] = p[3 + d] - p[d];
      ax[d] = x[d] - p[d];
      num = num + ax[d] * ab[d];
      den = den + ab[d] * ab[d];
    }
    double t = num / den;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double s = 0.0;
    for (int d = 0; d < D; d++) {
      double q = x[d] - (p[d] + t * ab[d]);
      s = s + q * q;
    }
    return sqrt(s) - p[6];
  }
  case OT_LSF_ELLIPSOID: {
    /* a_min (|S^-1 Q^T (x - c)| - 1), Q a rotation, S the semi-axes */
    double s = 0.0, amin = p[12];
    for (int i = 0; i < D; i++) {
      double y = 0.0;
      for (int j = 0; j < D; j++) y = y + p[3 + 3 * j + i] * (x[j] - p[j]);
      double q = y / p[12 + i];
      s = s + q * q;
      if (p[12 + i] < amin) amin = p[12 + i];
    }
    return amin * (sqrt(s) - 1.0);
  }
  case OT_LSF_SHAPE: {
    /* Eqs. (spheroid)-(astroid) of Sec. 4.3 in (p, q) = 4 (x - 1/2, y - 1/2),
     * or 4 (r - 1/2, z - 1/2) with r = sqrt(x^2 + y^2) (reading SH) */
    double P, Q;
    if (p[1] != 0.0) {
      P = 4.0 * (sqrt(x[0] * x[0] + x[1] * x[1]) - 0.5);
      Q = 4.0 * (x[2] - 0.5);
    } else {
      P = 4.0 * (x[0] - 0.5);
      Q = 4.0 * (x[1] - 0.5);
    }
    if (p[0] == 0.0) return sqrt(8.0 * P * P + Q * Q) - 1.0;
    if (p[0] == 1.0) return 8.0 * fabs(P) + fabs(Q) - 1.5;
    if (p[0] == 2.0) {
      double w = Q - cbrt(P * P);
      return P * P + w * w - 1.0;
    }
    return cbrt(P * P) / 0.8 + cbrt(Q * Q) / 1.5 - 0.8;
  }
  case OT_LSF_CALLBACK:
    return L->fn(x, L->user);
  case OT_LSF_GRID: {
    /* multilinear interpolant of gridded samples: locate the grid cell of x
     * (clamped to the sampled box), then sum the 2^D corner samples with
     * weights prod_d (w_d or 1 - w_d), corners in order with the x bit
     * fastest */
    const double *v = (const double *)L->user;
    int lo[3] = {0, 0, 0};
    double w[3] = {0.0, 0.0, 0.0};
    long long stride[3];
    stride[0] = 1;
    stride[1] = (long long)p[0];
    stride[2] = (long long)p[0] * (long long)p[1];
    for (int d = 0; d < D; d++) {
      const int n = (int)p[d];
      double t = (x[d] - p[3 + d]) / p[6 + d];
      if (t < 0.0) t = 0.0;
      if (t > n - 1.0) t = n - 1.0;
      int i = (int)floor(t);
      if (i > n - 2) i = n - 2;
      lo[d] = i;
      w[d] = t - i;
    }
    double f = 0.0;
    for (int corner = 0; corner < (1 << D); corner++) {
      double weight = 1.0;
      long long at = 0;
      for (int d = 0; d < D; d++) {
        const int up = (corner >> d) & 1;
        weight = weight * (up ? w[d] : 1.0 - w[d]);
        at = at + (long long)(lo[d] + up) * stride[d];
      }
      f = f + weight * v[at];
    }
    return f;
  }
  default:
    return 1.0;
  }
}

typedef struct {
  const ot_lsf *L;
  int D;
} lsf_ctx;
static double lsf_cb(const double *x, void *u) {
  const lsf_ctx *c = (const lsf_ctx *)u;
  return ot_lsf_eval(c->L, c->D, x);
}

/* ------------------------------------------------------------------ */
/* line search (Sec. 3.2, Eq. (relative-distance), readings BS, GS)   */
/* ------------------------------------------------------------------ */
static void seg_point(int D, const double *a, const double *b, double t, double *x) {
  for (int d = 0; d < 3; d++) x[d] = d < D ? a[d] + t * (b[d] - a[d]) : 0.0;
}

/* bisection for the root on t in [0, t_hi], with f(a) f(x(t_hi)) <= 0 */
static double bisect(ot_fn f, void *u, int D, const double *a, const double *b, double fa, double t_hi,
                     double eps) {
  double lo = 0.0, hi = t_hi, x[3];
  while (hi - lo >= eps) {
    double mid = 0.5 * (lo + hi);
    seg_point(D, a, b, mid, x);
    if (fa * f(x, u) <= 0.0)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

/* relative distance d in (0, 1] from a toward b; 1 when no root is found */
double ot_line_search(ot_fn f, void *u, int D, const double *a, const double *b, double eps) {
  double x[3], fa, fb;
  seg_point(D, a, b, 0.0, x);
  fa = f(a, u);
  fb = f(b, u);
  double t;
  if (fa * fb <= 0.0) {
    t = bisect(f, u, D, a, b, fa, 1.0, eps);
  } else {
    /* golden-section search for the minimum of f(a) f(x) on the segment */
    const double gr = (sqrt(5.0) - 1.0) / 2.0;
    double lo = 0.0, hi = 1.0;
    double t1 = hi - gr * (hi - lo), t2 = lo + gr * (hi - lo);
    seg_point(D, a, b, t1, x);
    double h1 = fa * f(x, u);
    if (h1 <= 0.0) {
      t = bisect(f, u, D, a, b, fa, t1, eps);
      goto done;
    }
    seg_point(D, a, b, t2, x);
    double h2 = fa * f(x, u);
    if (h2 <= 0.0) {
      t = bisect(f, u, D, a, b, fa, t2, eps);
      goto done;
    }
    while (hi - lo >= eps) {
      if (h1 < h2) {
        hi = t2;
        t2 = t1;
        h2 = h1;
        t1 = hi - gr * (hi - lo);
        seg_point(D, a, b, t1, x);
        h1 = fa * f(x, u);
        if (h1 <= 0.0) {
          t = bisect(f, u, D, a, b, fa, t1, eps);
          goto done;
        }
      } else {
        lo = t1;
        t1 = t2;
        h1 = h2;
        t2 = lo + gr * (hi - lo);
        seg_point(D, a, b, t2, x);
        h2 = fa * f(x, u);
        if (h2 <= 0.0) {
          t = bisect(f, u, D, a, b, fa, t2, eps);
          goto done;
        }
      }
    }
    return 1.0; /* no bracket found: no boundary */
  }
done:
  if (t < eps) t = eps; /* reading D0 */
  if (t > 1.0) t = 1.0;
  return t;
}

/* ------------------------------------------------------------------ */
/* boundary detection, distances, stencils (Sec. 3.3, 3.6)             */
/* ------------------------------------------------------------------ */
static int inside_domain(const ot_tree *T, int l, const int G[3]) {
  int e[3];
  lvl_cext(T, l, e);
  for (int d = 0; d < T->D; d++)
    if (G[d] < 0 || G[d] >= e[d]) return 0;
  return 1;
}

/* Sec. 3.6.3: gradient descent toward f = 0 from a cell centre a whose
 * mask is set but whose line searches found no root. */
static void unresolved(const ot_tree *T, lsf_ctx *ctx, const OB *B, const int p[3], const double *a, double fa,
                       double h, double *dd) {
  int D = T->D;
  double w = T->w_min;
  int nsteps = (int)floor(h / w);
  double x[3] = {a[0], a[1], a[2]};
  for (int s = 0; s < nsteps; s++) {
    double g[3] = {0, 0, 0}, gn = 0.0;
    for (int k = 0; k < D; k++) {
      double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
      xp[k] = x[k] + w;
      xm[k] = x[k] - w;
      g[k] = (lsf_cb(xp, ctx) - lsf_cb(xm, ctx)) / (2.0 * w);
      gn = gn + g[k] * g[k];
    }
    gn = sqrt(gn);
    if (!(gn > 0.0)) return;
    double sgn = fa > 0.0 ? -1.0 : 1.0; /* move toward f = 0 */
    for (int k = 0; k < D; k++) x[k] = x[k] + w * (sgn * g[k] / gn);
    double fx = lsf_cb(x, ctx);
    if (fa * fx <= 0.0) {
      double t = bisect(lsf_cb, ctx, D, a, x, fa, 1.0, T->eps_tol);
      double dist = 0.0;
      for (int k = 0; k < D; k++) dist = dist + (x[k] - a[k]) * (x[k] - a[k]);
      dist = t * sqrt(dist);
      double dv = dist / h;
      if (dv < T->eps_tol) dv = T->eps_tol;
      if (dv > 1.0) dv = 1.0;
      int ax = 0;
      double best = fabs(x[0] - a[0]);
      for (int k = 1; k < D; k++)
        if (fabs(x[k] - a[k]) > best) {
          best = fabs(x[k] - a[k]);
          ax = k;
        }
      int side = x[ax] - a[ax] > 0.0 ? 1 : 0;
      int G[3];
      for (int d = 0; d < 3; d++) G[d] = d < D ? B->ix[d] * B->n + p[d] : 0;
      G[ax] += side ? 1 : -1;
      if (inside_domain(T, B->level, G)) dd[2 * ax + side] = dv;
      return;
    }
  }
}

static double phib_at(ot_fn fn, void *u, double c, const double *x) { return fn ? fn(x, u) : c; }

static double wall_value_at(const ot_tree *T, int w, const double *x) {
  return T->wall_fn ? T->wall_fn(x, T->wall_user) : T->wall_val[w];
}

static int lu_factor(int n, double *A, int *piv);
static void lu_apply(int n, const double *LU, const int *piv, const double *b, double *x);

static void build_coarse_matrix(ot_tree *T);

int ot_store_stencils(ot_tree *T, ot_fn phib_fn, void *user, double phib_const) {
  int D = T->D;
  T->phib_fn = phib_fn;
  T->phib_user = user;
  T->phib_const = phib_const;
  lsf_ctx ctx = {&T->lsf, D};
  for (int l = T->lmin; l <= T->lmax; l++) {
    double h = lvl_h(T, l);
    double L = T->mask_factor * sqrt((double)D) * h;
    for (int i = 0; i < T->lev_cnt[l + LOFF]; i++) {
      OB *B = &T->B[T->lev_list[l + LOFF][i]];
      free_stencil(B);
      int n = B->n, nc = ncell(T, n);
      B->mask = (unsigned char *)calloc((size_t)nc, 1);
      double *dd = (double *)malloc((size_t)nc * 2 * D * sizeof(double));
      for (int c = 0; c < nc * 2 * D; c++) dd[c] = 1.0;
      int cut = 0;
      if (T->have_lsf) {
        FOR_CELLS(T, n, p) {
          int c = cidx(n, p);
          double a[3];
          cell_center(T, B, p, a);
          double fa = lsf_cb(a, &ctx);
          /* Eq. (boundary-mask): |f| < L |grad f|, central differences */
          double gn = 0.0;
          for (int k = 0; k < D; k++) {
            double xp[3] = {a[0], a[1], a[2]}, xm[3] = {a[0], a[1], a[2]};
            xp[k] = a[k] + h;
            xm[k] = a[k] - h;
            double g = (lsf_cb(xp, &ctx) - lsf_cb(xm, &ctx)) / (2.0 * h);
            gn = gn + g * g;
          }
          gn = sqrt(gn);
          int mask = fabs(fa) < L * gn;
          B->mask[c] = (unsigned char)mask;
          if (!mask) continue;
          double *dc = dd + (size_t)c * 2 * D;
          int found = 0;
          for (int k = 0; k < D; k++)
            for (int s = 0; s < 2; s++) {
              int G[3];
              for (int d = 0; d < 3; d++) G[d] = d < D ? B->ix[d] * n + p[d] : 0;
              G[k] += s ? 1 : -1;
              if (!inside_domain(T, l, G)) continue;
              double bpt[3] = {a[0], a[1], a[2]};
              bpt[k] = s ? a[k] + h : a[k] - h;
              dc[2 * k + s] = ot_line_search(lsf_cb, &ctx, D, a, bpt, T->eps_tol);
              if (dc[2 * k + s] < 1.0) found = 1;
            }
          if (!found && T->w_min > 0.0 && h > T->w_min) unresolved(T, &ctx, B, p, a, fa, h, dc);
          for (int k = 0; k < 2 * D; k++)
            if (dc[k] < 1.0) cut = 1;
        }
      }
      B->cut = cut;
      if (cut) {
        B->dd = dd;
        B->st = (double *)calloc((size_t)nc * (2 * D + 1), sizeof(double));
        B->bnd = (double *)calloc((size_t)nc, sizeof(double));
        B->smv = (double *)calloc((size_t)nc, sizeof(double));
        double inv_h2 = 1.0 / (h * h);
        FOR_CELLS(T, n, p) {
          int c = cidx(n, p);
          double a[3];
          cell_center(T, B, p, a);
          const double *dc = dd + (size_t)c * 2 * D;
          double *st = B->st + (size_t)c * (2 * D + 1);
          double diag = 0.0, bnd = 0.0, smv = 0.0;
          /* Eq. (lpl-1d-lsf) per dimension, Eq. (lpl-2d-lsf) */
          for (int k = 0; k < D; k++) {
            double dm = dc[2 * k], dp = dc[2 * k + 1];
            double cm = 2.0 * inv_h2 / ((dp + dm) * dm);
            double cp = 2.0 * inv_h2 / ((dp + dm) * dp);
            diag = diag - (cm + cp);
            if (dm < 1.0) { /* boundary between i-1 and i: phi_b to the RHS */
              double x0[3] = {a[0], a[1], a[2]};
              x0[k] = a[k] - dm * h;
              bnd = bnd + cm * phib_at(phib_fn, user, phib_const, x0);
              smv = smv + cm;
              cm = 0.0;
            }
            if (dp < 1.0) {
              double x0[3] = {a[0], a[1], a[2]};
              x0[k] = a[k] + dp * h;
              bnd = bnd + cp * phib_at(phib_fn, user, phib_const, x0);
              smv = smv + cp;
              cp = 0.0;
            }
            st[1 + 2 * k] = cm;
            st[2 + 2 * k] = cp;
          }
          st[0] = diag;
          B->bnd[c] = bnd;
          B->smv[c] = smv;
        }
      } else {
        free(dd);
      }
      /* boundary terms of the right-hand side: moved coefficients and
       * Dirichlet walls (reading W) */
      B->bterm = (double *)calloc((size_t)nc, sizeof(double));
      FOR_CELLS(T, n, p) {
        int c = cidx(n, p);
        double t = B->cut ? B->bnd[c] : 0.0;
        double a[3];
        cell_center(T, B, p, a);
        for (int k = 0; k < D; k++)
          for (int s = 0; s < 2; s++) {
            int G[3];
            for (int d = 0; d < 3; d++) G[d] = d < D ? B->ix[d] * n + p[d] : 0;
            G[k] += s ? 1 : -1;
            if (inside_domain(T, l, G)) continue;
            int w = 2 * k + s;
            if (T->wall_type[w] != OT_WALL_DIRICHLET) continue;
            double coef = B->cut ? B->st[(size_t)c * (2 * D + 1) + 1 + 2 * k + s] : 1.0 / (h * h);
            double xf[3] = {a[0], a[1], a[2]};
            xf[k] = s ? a[k] + 0.5 * h : a[k] - 0.5 * h;
            t = t + coef * (2.0 * wall_value_at(T, w, xf));
          }
        B->bterm[c] = t;
      }
    }
  }
  build_coarse_matrix(T);
  T->stencils_ready = 1;
  return 0;
}

int ot_num_cut_blocks(const ot_tree *T, int level) {
  int s = 0;
  for (int i = 0; i < ot_level_nblocks(T, level); i++) s += T->B[T->lev_list[level + LOFF][i]].cut;
  return s;
}

void ot_get_d(const ot_tree *T, int level, double *out) {
  int D = T->D;
  size_t k = 0;
  for (int i = 0; i < ot_level_nblocks(T, level); i++) {
    const OB *B = &T->B[T->lev_list[level + LOFF][i]];
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc * 2 * D; c++) out[k++] = B->cut ? B->dd[c] : 1.0;
  }
}

void ot_get_mask(const ot_tree *T, int level, int *out) {
  size_t k = 0;
  for (int i = 0; i < ot_level_nblocks(T, level); i++) {
    const OB *B = &T->B[T->lev_list[level + LOFF][i]];
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc; c++) out[k++] = B->mask ? B->mask[c] : 0;
  }
}

/* ------------------------------------------------------------------ */
/* ghost cells (Sec. 2.2 "Ghost cells", readings G, W, P)              */
/* ------------------------------------------------------------------ */
enum { F_PHI = 0, F_CORR = 1 };

static double field(const OB *B, int which, int c) {
  return which == F_PHI ? B->phi[c] : B->phi[c] - B->old[c];
}

/* value at global cell G of level l inside the domain; *ok = 0 if the
 * level has no block there */
static double value_in(const ot_tree *T, int l, const int G[3], int which, int *ok) {
  int n = lvl_n(T, l), bix[3], p[3];
  for (int d = 0; d < 3; d++) {
    bix[d] = d < T->D ? G[d] / n : 0;
    p[d] = d < T->D ? G[d] - bix[d] * n : 0;
  }
  int id = map_find(T, l, bix);
  if (id < 0) {
    *ok = 0;
    return NAN;
  }
  *ok = 1;
  return field(&T->B[id], which, cidx(n, p));
}

/* value at G, reflecting across domain walls (homogeneous wall ghosts) */
static double value_walls(const ot_tree *T, int l, const int Gin[3], int which, int *ok) {
  int e[3], G[3] = {Gin[0], Gin[1], Gin[2]};
  lvl_cext(T, l, e);
  double sign = 1.0;
  for (int d = 0; d < T->D; d++) {
    if (G[d] < 0) {
      G[d] = -1 - G[d];
      sign *= T->wall_type[2 * d] == OT_WALL_DIRICHLET ? -1.0 : 1.0;
    } else if (G[d] >= e[d]) {
      G[d] = 2 * e[d] - 1 - G[d];
      sign *= T->wall_type[2 * d + 1] == OT_WALL_DIRICHLET ? -1.0 : 1.0;
    }
  }
  double v = value_in(T, l, G, which, ok);
  return sign * v;
}

/* reading G: ghost of fine block B at face axis a across a refinement
 * boundary, from the adjacent fine cell and the coarse level */
static double refine_ghost(const ot_tree *T, const OB *B, const int p[3], const int G[3], int a, int which) {
  int n = B->n, q[3] = {p[0], p[1], p[2]};
  q[a] = p[a] < 0 ? 0 : n - 1;
  double f = field(B, which, cidx(n, q));
  int Gc[3] = {G[0] >> 1, G[1] >> 1, G[2] >> 1}, ok;
  if (T->D == 2) Gc[2] = 0;
  double c = value_in(T, B->level - 1, Gc, which, &ok);
  if (!ok) return NAN;
  double chat = c;
  for (int t = 0; t < T->D; t++) {
    if (t == a) continue;
    double o = (G[t] & 1) ? 0.25 : -0.25;
    int Gp[3] = {Gc[0], Gc[1], Gc[2]}, Gm[3] = {Gc[0], Gc[1], Gc[2]};
    Gp[t] += 1;
    Gm[t] -= 1;
    int okp, okm;
    double cp = value_walls(T, B->level - 1, Gp, which, &okp);
    double cm = value_walls(T, B->level - 1, Gm, which, &okm);
    if (!okp || !okm) return NAN;
    chat = chat + o * (0.5 * (cp - cm));
  }
  return f / 3.0 + 2.0 * chat / 3.0;
}

static double ghost_value(const ot_tree *T, const OB *B, const int p[3], int which) {
  int n = B->n, G[3], e[3], nout = 0, outdom = 0, a = 0;
  lvl_cext(T, B->level, e);
  for (int d = 0; d < 3; d++) {
    G[d] = d < T->D ? B->ix[d] * n + p[d] : 0;
    if (d < T->D && (p[d] < 0 || p[d] >= n)) {
      nout++;
      a = d;
    }
    if (d < T->D && (G[d] < 0 || G[d] >= e[d])) outdom = 1;
  }
  int ok;
  if (!outdom) {
    double v = value_in(T, B->level, G, which, &ok);
    if (ok) return v;
    if (nout == 1) return refine_ghost(T, B, p, G, a, which);
    return NAN;
  }
  double v = value_walls(T, B->level, G, which, &ok);
  return ok ? v : NAN;
}

static void fill_ghosts(ot_tree *T, int l, int which, int corners) {
  int D = T->D;
  for (int i = 0; i < T->lev_cnt[l + LOFF]; i++) {
    OB *B = &T->B[T->lev_list[l + LOFF][i]];
    int n = B->n;
    int z0 = D == 3 ? -1 : 0, z1 = D == 3 ? n : 0;
    for (int z = z0; z <= z1; z++)
      for (int y = -1; y <= n; y++)
        for (int x = -1; x <= n; x++) {
          int p[3] = {x, y, z}, nout = 0;
          for (int d = 0; d < D; d++)
            if (p[d] < 0 || p[d] >= n) nout++;
          double v;
          if (nout == 0)
            v = field(B, which, cidx(n, p));
          else if (nout >= 2 && !corners)
            v = NAN;
          else
            v = ghost_value(T, B, p, which);
          B->gh[gidx(T, n, p)] = v;
        }
  }
}

/* ------------------------------------------------------------------ */
/* operator (Eq. (lpl-1d), Eq. (lpl-2d-lsf)), smoother, residual       */
/* ------------------------------------------------------------------ */
/* off-diagonal part sum_j c_ij phi_j (ghosts from B->gh) and the diagonal */
static double op_offdiag(const ot_tree *T, const OB *B, const int p[3], double *diag) {
  int D = T->D, n = B->n;
  double s = 0.0;
  if (!B->cut) {
    double h = lvl_h(T, B->level), inv_h2 = 1.0 / (h * h);
    for (int k = 0; k < D; k++) {
      int pm[3] = {p[0], p[1], p[2]}, pp[3] = {p[0], p[1], p[2]};
      pm[k]--;
      pp[k]++;
      s = s + (B->gh[gidx(T, n, pm)] + B->gh[gidx(T, n, pp)]) * inv_h2;
    }
    *diag = -2.0 * D * inv_h2;
  } else {
    const double *st = B->st + (size_t)cidx(n, p) * (2 * D + 1);
    for (int k = 0; k < D; k++) {
      int pm[3] = {p[0], p[1], p[2]}, pp[3] = {p[0], p[1], p[2]};
      pm[k]--;
      pp[k]++;
      if (st[1 + 2 * k] != 0.0) s = s + st[1 + 2 * k] * B->gh[gidx(T, n, pm)];
      if (st[2 + 2 * k] != 0.0) s = s + st[2 + 2 * k] * B->gh[gidx(T, n, pp)];
    }
    *diag = st[0];
  }
  return s;
}

static int color_of(const OB *B, const int p[3], int D) {
  int s = 0;
  for (int d = 0; d < D; d++) s += B->ix[d] * B->n + p[d];
  return s & 1;
}

/* one half-sweep of red-black Gauss-Seidel (Sec. 2.2, reading S, SW) */
static void gsrb(ot_tree *T, int l, int color) {
  fill_ghosts(T, l, F_PHI, 0);
  for (int i = 0; i < T->lev_cnt[l + LOFF]; i++) {
    OB *B = &T->B[T->lev_list[l + LOFF][i]];
    FOR_CELLS(T, B->n, p) {
      if (color_of(B, p, T->D) != color) continue;
      double diag, s = op_offdiag(T, B, p, &diag);
      int c = cidx(B->n, p);
      B->phi[c] = (B->b[c] - s) / diag;
    }
  }
}

/* Eq. (residual): r = b - A phi on all blocks of level l */
static void residual_level(ot_tree *T, int l) {
  fill_ghosts(T, l, F_PHI, 0);
  for (int i = 0; i < T->lev_cnt[l + LOFF]; i++) {
    OB *B = &T->B[T->lev_list[l + LOFF][i]];
    FOR_CELLS(T, B->n, p) {
      double diag, s = op_offdiag(T, B, p, &diag);
      int c = cidx(B->n, p);
      B->r[c] = B->b[c] - (diag * B->phi[c] + s);
    }
  }
}

/* restriction: mean of the 2^D children (Sec. 2.2) */
static void restrict_level(ot_tree *T, int l, int with_r) {
  int D = T->D;
  double w = 1.0 / (double)(1 << D);
  for (int i = 0; i < T->lev_cnt[l + LOFF]; i++) {
    OB *B = &T->B[T->lev_list[l + LOFF][i]];
    OB *P = &T->B[B->parent];
    int h = B->n / 2;
    FOR_CELLS(T, h, q) {
      double sp = 0.0, sr = 0.0;
      for (int dz = 0; dz < (D == 3 ? 2 : 1); dz++)
        for (int dy = 0; dy < 2; dy++)
          for (int dx = 0; dx < 2; dx++) {
            int c[3] = {2 * q[0] + dx, 2 * q[1] + dy, 2 * q[2] + dz};
            sp = sp + B->phi[cidx(B->n, c)];
            sr = sr + B->r[cidx(B->n, c)];
          }
      int pc[3] = {B->pofs[0] + q[0], B->pofs[1] + q[1], D == 3 ? B->pofs[2] + q[2] : 0};
      P->phi[cidx(P->n, pc)] = sp * w;
      if (with_r) P->tmp[cidx(P->n, pc)] = sr * w;
    }
  }
}

/* FAS coarse right-hand side b = A phi + R r on covered cells (Sec. 2.2) */
static void fas_rhs(ot_tree *T, int l) {
  fill_ghosts(T, l, F_PHI, 0);
  for (int i = 0; i < T->lev_cnt[l + LOFF]; i++) {
    OB *B = &T->B[T->lev_list[l + LOFF][i]];
    int nc = ncell(T, B->n);
    if (B->has_children) {
      FOR_CELLS(T, B->n, p) {
        double diag, s = op_offdiag(T, B, p, &diag);
        int c = cidx(B->n, p);
        B->b[c] = (diag * B->phi[c] + s) + B->tmp[c];
      }
    }
    memcpy(B->old, B->phi, (size_t)nc * sizeof(double));
  }
}

/* (bi/tri)linear prolongation of the coarse correction (Sec. 2.2, 3.4) */
static void prolong(ot_tree *T, int l) {
  int D = T->D;
  fill_ghosts(T, l - 1, F_CORR, 1);
  for (int i = 0; i < T->lev_cnt[l + LOFF]; i++) {
    OB *B = &T->B[T->lev_list[l + LOFF][i]];
    const OB *P = &T->B[B->parent];
    FOR_CELLS(T, B->n, p) {
      int q[3], o[3];
      for (int d = 0; d < 3; d++) {
        q[d] = d < D ? B->pofs[d] + p[d] / 2 : 0;
        o[d] = (p[d] & 1) ? 1 : -1;
      }
      double v = 0.0;
      for (int sz = 0; sz < (D == 3 ? 2 : 1); sz++)
        for (int sy = 0; sy < 2; sy++)
          for (int sx = 0; sx < 2; sx++) {
            int s[3] = {sx, sy, sz};
            double wgt = 1.0;
            int qq[3] = {q[0], q[1], q[2]};
            for (int d = 0; d < D; d++) {
              wgt *= s[d] ? 0.25 : 0.75;
              qq[d] += s[d] * o[d];
            }
            v = v + wgt * P->gh[gidx(T, P->n, qq)];
          }
      B->phi[cidx(B->n, p)] += v;
    }
  }
}

/* ------------------------------------------------------------------ */
/* coarse-grid solve (Sec. 3.5, reading C)                             */
/* ------------------------------------------------------------------ */
static int lu_factor(int n, double *A, int *piv) {
  for (int k = 0; k < n; k++) {
    int pr = k;
    double best = fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; i++)
      if (fabs(A[(size_t)i * n + k]) > best) {
        best = fabs(A[(size_t)i * n + k]);
        pr = i;
      }
    piv[k] = pr;
    if (best == 0.0) return -1;
    if (pr != k)
      for (int j = 0; j < n; j++) {
        double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)pr * n + j];
        A[(size_t)pr * n + j] = t;
      }
    for (int i = k + 1; i < n; i++) {
      double m = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      A[(size_t)i * n + k] = m;
      for (int j = k + 1; j < n; j++) A[(size_t)i * n + j] -= m * A[(size_t)k * n + j];
    }
  }
  return 0;
}

static void lu_apply(int n, const double *LU, const int *piv, const double *b, double *x) {
  for (int i = 0; i < n; i++) x[i] = b[i];
  for (int k = 0; k < n; k++)
    if (piv[k] != k) {
      double t = x[k];
      x[k] = x[piv[k]];
      x[piv[k]] = t;
    }
  for (int i = 0; i < n; i++)
    for (int j = 0; j < i; j++) x[i] -= LU[(size_t)i * n + j] * x[j];
  for (int i = n - 1; i >= 0; i--) {
    for (int j = i + 1; j < n; j++) x[i] -= LU[(size_t)i * n + j] * x[j];
    x[i] /= LU[(size_t)i * n + i];
  }
}

int ot_lu_solve(int n, const double *A, const double *b, double *x) {
  double *LU = (double *)malloc((size_t)n * n * sizeof(double));
  int *piv = (int *)malloc((size_t)n * sizeof(int));
  memcpy(LU, A, (size_t)n * n * sizeof(double));
  int rc = lu_factor(n, LU, piv);
  if (rc == 0) lu_apply(n, LU, piv, b, x);
  free(LU);
  free(piv);
  return rc;
}

/* the coarsest level is uniform: row per cell (canonical order) with the
 * homogeneous wall ghosts folded into the diagonal */
static void build_coarse_matrix(ot_tree *T) {
  int l = T->lmin, D = T->D, n = lvl_n(T, l), nc1 = ncell(T, n);
  int nbk = T->lev_cnt[l + LOFF];
  int N = nbk * nc1;
  free(T->lu);
  free(T->piv);
  T->nc = N;
  T->lu = (double *)calloc((size_t)N * N, sizeof(double));
  T->piv = (int *)malloc((size_t)N * sizeof(int));
  /* position of each block in canonical order */
  int *pos = (int *)malloc((size_t)T->nb * sizeof(int));
  for (int i = 0; i < nbk; i++) pos[T->lev_list[l + LOFF][i]] = i;
  double h = lvl_h(T, l), inv_h2 = 1.0 / (h * h);
  int e[3];
  lvl_cext(T, l, e);
  for (int i = 0; i < nbk; i++) {
    const OB *B = &T->B[T->lev_list[l + LOFF][i]];
    FOR_CELLS(T, n, p) {
      int row = i * nc1 + cidx(n, p);
      double *Ar = T->lu + (size_t)row * N;
      const double *st = B->cut ? B->st + (size_t)cidx(n, p) * (2 * D + 1) : NULL;
      Ar[row] += st ? st[0] : -2.0 * D * inv_h2;
      for (int k = 0; k < D; k++)
        for (int s = 0; s < 2; s++) {
          double coef = st ? st[1 + 2 * k + s] : inv_h2;
          int G[3];
          for (int d = 0; d < 3; d++) G[d] = d < D ? B->ix[d] * n + p[d] : 0;
          G[k] += s ? 1 : -1;
          if (G[k] < 0 || G[k] >= e[k]) {
            double sign = T->wall_type[2 * k + s] == OT_WALL_DIRICHLET ? -1.0 : 1.0;
            Ar[row] += sign * coef;
          } else {
            int bix[3], q[3];
            for (int d = 0; d < 3; d++) {
              bix[d] = d < D ? G[d] / n : 0;
              q[d] = d < D ? G[d] - bix[d] * n : 0;
            }
            int col = pos[map_find(T, l, bix)] * nc1 + cidx(n, q);
            Ar[col] += coef;
          }
        }
    }
  }
  free(pos);
  if (lu_factor(N, T->lu, T->piv) != 0) fprintf(stderr, "oracle: singular coarse matrix\n");
}

static void coarse_solve(ot_tree *T) {
  int l = T->lmin, n = lvl_n(T, l), nc1 = ncell(T, n), nbk = T->lev_cnt[l + LOFF];
  double *b = (double *)calloc((size_t)T->nc, sizeof(double));
  double *x = (double *)calloc((size_t)T->nc, sizeof(double));
  for (int i = 0; i < nbk; i++) memcpy(b + (size_t)i * nc1, T->B[T->lev_list[l + LOFF][i]].b, nc1 * sizeof(double));
  lu_apply(T->nc, T->lu, T->piv, b, x);
  for (int i = 0; i < nbk; i++) memcpy(T->B[T->lev_list[l + LOFF][i]].phi, x + (size_t)i * nc1, nc1 * sizeof(double));
  free(b);
  free(x);
}

/* ------------------------------------------------------------------ */
/* V-cycle (Sec. 2.2 "Multigrid cycle", FAS; readings UP, V)           */
/* ------------------------------------------------------------------ */
static void restrict_all_phi(ot_tree *T) {
  for (int l = T->lmax; l >= 2; l--) restrict_level(T, l, 0);
}

/* one V-cycle on the levels lmin .. top (top = lmax: the solver's V-cycle) */
static void vcycle_top(ot_tree *T, int top) {
  for (int l = top; l > T->lmin; l--) {
    for (int s = 0; s < T->n_down; s++) {
      gsrb(T, l, 0);
      gsrb(T, l, 1);
    }
    residual_level(T, l);
    restrict_level(T, l, 1);
    fas_rhs(T, l - 1);
  }
  coarse_solve(T);
  for (int l = T->lmin + 1; l <= top; l++) {
    prolong(T, l);
    for (int s = 0; s < T->n_up; s++) {
      gsrb(T, l, 0);
      gsrb(T, l, 1);
    }
  }
  for (int l = top; l >= 2; l--) restrict_level(T, l, 0); /* reading V */
}

static void vcycle_once(ot_tree *T) { vcycle_top(T, T->lmax); }

/* FMG cycle (Sec. 2.2 "Multigrid cycle": V-cycles from the coarsest grid
   up to the finest), in FAS form (reading FMG): residuals and FAS right-hand
   sides are carried from the finest level down to the coarsest without
   smoothing, the coarsest level is solved, and then for each finer level in
   turn the coarse correction is prolonged to it and one V-cycle is done
   with that level on top. */
void ot_fmg(ot_tree *T, int n) {
  for (int it = 0; it < n; it++) {
    for (int l = T->lmax; l > T->lmin; l--) {
      residual_level(T, l);
      restrict_level(T, l, 1);
      fas_rhs(T, l - 1);
    }
    coarse_solve(T);
    for (int l = T->lmin + 1; l <= T->lmax; l++) {
      prolong(T, l);
      vcycle_top(T, l);
    }
  }
}

void ot_vcycle(ot_tree *T, int n) {
  for (int i = 0; i < n; i++) vcycle_once(T);
}

/* E = -grad(phi) on the upper face of every leaf cell (Sec. 4.4: gradients
 * on a staggered grid that take the stored boundary distances into
 * account): (phi_b - phi)/(d dx) across the object's boundary, 2 (phi_w -
 * phi)/dx at a Dirichlet domain wall, 0 at a Neumann wall, the difference
 * to the neighbour's (ghost) value otherwise; 0 in cells whose centre lies
 * inside the object.  out: leaf cells x D.  Pin: exact (-a) for a linear
 * phi = a.x + c with matching boundary and wall values. */
void ot_efield(ot_tree *T, double *out) {
  int D = T->D;
  for (int l = T->lmin; l <= T->lmax; l++) fill_ghosts(T, l, F_PHI, 0);
  int64_t k = 0;
  FOR_LEAF_BLOCKS(T, l, i, B) {
    int n = B->n, e[3];
    double h = lvl_h(T, l);
    lvl_cext(T, l, e);
    FOR_CELLS(T, n, p) {
      int c = cidx(n, p);
      double a[3], phi = B->phi[c];
      cell_center(T, B, p, a);
      int inside = T->have_lsf && ot_lsf_eval(&T->lsf, D, a) < 0.0;
      for (int ax = 0; ax < D; ax++) {
        double g, d = (B->cut && B->dd) ? B->dd[(size_t)c * 2 * D + 2 * ax + 1] : 1.0;
        int G[3];
        for (int q = 0; q < 3; q++) G[q] = q < D ? B->ix[q] * n + p[q] : 0;
        G[ax] += 1;
        if (inside) {
          g = 0.0;
        } else if (d < 1.0) {
          double x0[3] = {a[0], a[1], a[2]};
          x0[ax] = a[ax] + d * h;
          g = (phib_at(T->phib_fn, T->phib_user, T->phib_const, x0) - phi) / (d * h);
        } else if (G[ax] >= e[ax]) {
          if (T->wall_type[2 * ax + 1] == OT_WALL_DIRICHLET) {
            double xf[3] = {a[0], a[1], a[2]};
            xf[ax] = a[ax] + 0.5 * h;
            g = 2.0 * (wall_value_at(T, 2 * ax + 1, xf) - phi) / h;
          } else {
            g = 0.0;
          }
        } else {
          int q[3] = {p[0], p[1], p[2]};
          q[ax] += 1;
          g = (B->gh[gidx(T, n, q)] - phi) / h;
        }
        out[k * D + ax] = -g;
      }
      k++;
    }
  }
}

void ot_set_rhs(ot_tree *T, const double *g) {
  int64_t k = 0;
  FOR_LEAF_BLOCKS(T, l, i, B) {
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc; c++, k++) B->b[c] = g[k] - (B->bterm ? B->bterm[c] : 0.0);
  }
}

void ot_set_solution(ot_tree *T, const double *phi) {
  int64_t k = 0;
  FOR_LEAF_BLOCKS(T, l, i, B) {
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc; c++) B->phi[c] = phi[k++];
  }
  restrict_all_phi(T);
}

void ot_get_solution(const ot_tree *T, double *phi) {
  int64_t k = 0;
  FOR_LEAF_BLOCKS(T, l, i, B) {
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc; c++) phi[k++] = B->phi[c];
  }
}

void ot_get_level(const ot_tree *T, int level, int which, double *out) {
  size_t k = 0;
  for (int i = 0; i < ot_level_nblocks(T, level); i++) {
    const OB *B = &T->B[T->lev_list[level + LOFF][i]];
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc; c++) out[k++] = which == 0 ? B->phi[c] : B->b[c];
  }
}

/* composite residual over leaf cells (reading R) */
double ot_residual(ot_tree *T, double *linf, double *bnorm, double *r_out) {
  double s2 = 0.0, mx = 0.0, b2 = 0.0;
  int64_t k = 0;
  for (int l = T->lmin; l <= T->lmax; l++) {
    fill_ghosts(T, l, F_PHI, 0);
    for (int i = 0; i < T->lev_cnt[l + LOFF]; i++) {
      OB *B = &T->B[T->lev_list[l + LOFF][i]];
      if (B->has_children) continue;
      FOR_CELLS(T, B->n, p) {
        double diag, s = op_offdiag(T, B, p, &diag);
        int c = cidx(B->n, p);
        double r = B->b[c] - (diag * B->phi[c] + s);
        s2 += r * r;
        b2 += B->b[c] * B->b[c];
        if (fabs(r) > mx) mx = fabs(r);
        if (r_out) r_out[k] = r;
        k++;
      }
    }
  }
  if (linf) *linf = mx;
  if (bnorm) *bnorm = sqrt(b2);
  return sqrt(s2);
}

int ot_solve(ot_tree *T, double rel_tol, int max_cycles, double *hist) {
  double bn, r = ot_residual(T, NULL, &bn, NULL);
  if (bn == 0.0) bn = 1.0;
  if (r / bn <= rel_tol) return 0;
  for (int k = 0; k < max_cycles; k++) {
    vcycle_once(T);
    r = ot_residual(T, NULL, NULL, NULL);
    if (hist) hist[k] = r / bn;
    if (r / bn <= rel_tol) return k + 1;
  }
  return -max_cycles;
}

/* A phi (+ boundary terms) on leaf cells for leaf values phi */
void ot_apply_composite(ot_tree *T, const double *phi, double *out, int with_bterm) {
  ot_set_solution(T, phi);
  int64_t k = 0;
  for (int l = T->lmin; l <= T->lmax; l++) {
    fill_ghosts(T, l, F_PHI, 0);
    for (int i = 0; i < T->lev_cnt[l + LOFF]; i++) {
      OB *B = &T->B[T->lev_list[l + LOFF][i]];
      if (B->has_children) continue;
      FOR_CELLS(T, B->n, p) {
        double diag, s = op_offdiag(T, B, p, &diag);
        int c = cidx(B->n, p);
        double v = diag * B->phi[c] + s;
        if (with_bterm && B->bterm) v += B->bterm[c];
        out[k++] = v;
      }
    }
  }
}

int ot_composite_matrix(ot_tree *T, double *A, double *b) {
  int64_t n = ot_num_leaf_cells(T);
  double *e = (double *)calloc((size_t)n, sizeof(double));
  double *col = (double *)malloc((size_t)n * sizeof(double));
  double *save = (double *)malloc((size_t)n * sizeof(double));
  ot_get_solution(T, save);
  for (int64_t j = 0; j < n; j++) {
    e[j] = 1.0;
    ot_apply_composite(T, e, col, 0);
    for (int64_t i = 0; i < n; i++) A[i * n + j] = col[i];
    e[j] = 0.0;
  }
  int64_t k = 0;
  FOR_LEAF_BLOCKS(T, l, i, B) {
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc; c++) b[k++] = B->b[c];
  }
  ot_set_solution(T, save);
  free(e);
  free(col);
  free(save);
  return 0;
}

void ot_halfsweep(ot_tree *T, int level, int color) { gsrb(T, level, color); }

void ot_level_residual(ot_tree *T, int level, double *out) {
  residual_level(T, level);
  size_t k = 0;
  for (int i = 0; i < ot_level_nblocks(T, level); i++) {
    const OB *B = &T->B[T->lev_list[level + LOFF][i]];
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc; c++) out[k++] = B->r[c];
  }
}

void ot_set_level(ot_tree *T, int level, int which, const double *in) {
  size_t k = 0;
  for (int i = 0; i < ot_level_nblocks(T, level); i++) {
    OB *B = &T->B[T->lev_list[level + LOFF][i]];
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc; c++, k++) {
      if (which == 0)
        B->phi[c] = in[k];
      else
        B->b[c] = in[k];
    }
  }
}

void ot_prolong_test(ot_tree *T, int level, const double *coarse, double *fine) {
  size_t k = 0;
  for (int i = 0; i < ot_level_nblocks(T, level - 1); i++) {
    OB *B = &T->B[T->lev_list[level - 1 + LOFF][i]];
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc; c++, k++) {
      B->phi[c] = coarse[k];
      B->old[c] = 0.0;
    }
  }
  for (int i = 0; i < ot_level_nblocks(T, level); i++) {
    OB *B = &T->B[T->lev_list[level + LOFF][i]];
    memset(B->phi, 0, (size_t)ncell(T, B->n) * sizeof(double));
  }
  prolong(T, level);
  ot_get_level(T, level, 0, fine);
}

void ot_restrict_test(ot_tree *T, int level, const double *fine, double *coarse) {
  size_t k = 0;
  for (int i = 0; i < ot_level_nblocks(T, level); i++) {
    OB *B = &T->B[T->lev_list[level + LOFF][i]];
    int nc = ncell(T, B->n);
    for (int c = 0; c < nc; c++, k++) {
      B->phi[c] = fine[k];
      B->r[c] = 0.0;
    }
  }
  restrict_level(T, level, 0);
  ot_get_level(T, level - 1, 0, coarse);
}
