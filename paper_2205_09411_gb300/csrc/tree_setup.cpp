// Host side of the library: block-tree construction (Sec. 2.1) and the
// boundary set-up (Sec. 3.2, 3.3, 3.6): mask, line searches, unresolved-root
// search, cut-cell stencils, right-hand-side boundary terms and the inverse
// of the coarsest-level operator (Sec. 3.5).  Compiled with
// -ffp-contract=off: the level-set arithmetic is plain IEEE.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <unordered_map>

#include "gmg_internal.h"
#include "lsf.cuh"

namespace gmg {

namespace {

struct TB {  // block under construction
  int level, ix[3], parent, pofs[3], child[8], has_children;
};

struct Builder {
  int D, N, cb[3], max_level;
  std::vector<TB> blocks;
  std::unordered_map<long long, int> maps[kMaxLevels];  // level + 20 -> (key -> id)
  std::vector<int> lists[kMaxLevels];

  static long long key(const int *b) { return ((long long)b[2] << 42) | ((long long)b[1] << 21) | (long long)b[0]; }
  int lidx(int l) const { return l + 20; }
  int n_of(int l) const { return l >= 1 ? N : (N >> (1 - l)); }
  void bext(int l, int *e) const {
    for (int d = 0; d < 3; d++) e[d] = d < D ? (l >= 1 ? cb[d] << (l - 1) : cb[d]) : 1;
  }
  int find(int l, const int *b) const {
    int e[3];
    bext(l, e);
    for (int d = 0; d < 3; d++)
      if (b[d] < 0 || b[d] >= e[d]) return -1;
    auto it = maps[lidx(l)].find(key(b));
    return it == maps[lidx(l)].end() ? -1 : it->second;
  }
  int add(int l, const int *b, int parent, const int *pofs) {
    TB t;
    t.level = l;
    for (int d = 0; d < 3; d++) {
      t.ix[d] = b[d];
      t.pofs[d] = pofs[d];
    }
    t.parent = parent;
    for (int c = 0; c < 8; c++) t.child[c] = -1;
    t.has_children = 0;
    int id = (int)blocks.size();
    blocks.push_back(t);
    maps[lidx(l)][key(b)] = id;
    lists[lidx(l)].push_back(id);
    return id;
  }
  void refine(int id) {
    if (blocks[id].has_children) return;
    for (int o = 0; o < (1 << D); o++) {
      int b[3] = {0, 0, 0}, pofs[3] = {0, 0, 0};
      for (int d = 0; d < D; d++) {
        int bit = (o >> d) & 1;
        b[d] = 2 * blocks[id].ix[d] + bit;
        pofs[d] = bit * (N / 2);
      }
      int c = add(blocks[id].level + 1, b, id, pofs);
      blocks[id].child[o] = c;
    }
    blocks[id].has_children = 1;
  }
  void ensure(int l, const int *b) {
    if (find(l, b) >= 0) return;
    int p[3] = {b[0] >> 1, b[1] >> 1, b[2] >> 1};
    ensure(l - 1, p);
    refine(find(l - 1, p));
  }
};

unsigned long long morton(const int *b, int D) {
  unsigned long long m = 0;
  for (int bit = 0; bit < 21; bit++)
    for (int d = 0; d < D; d++) m |= (unsigned long long)((b[d] >> bit) & 1) << (bit * D + d);
  return m;
}

}  // namespace

int build_tree(gmg_tree *T, const gmg_domain *dom) {
  int D = dom->dim, N = dom->block_n;
  if (D < 2 || D > 3) return set_error("dim must be 2 or 3"), GMG_ERR_INVALID_ARG;
  if (N < 4 || (N & 1) || N > (D == 3 ? 16 : 32))
    return set_error("block_n must be even, 4 <= N <= 16 (3D) or 32 (2D)"), GMG_ERR_INVALID_ARG;
  if (dom->max_level < 1 || dom->max_level > 20) return set_error("max_level must be in 1..20"), GMG_ERR_INVALID_ARG;
  if (!(dom->h_root > 0.0)) return set_error("h_root must be positive"), GMG_ERR_INVALID_ARG;
  Builder B;
  B.D = D;
  B.N = N;
  B.max_level = dom->max_level;
  for (int d = 0; d < 3; d++) {
    B.cb[d] = d < D ? dom->coarse_blocks[d] : 1;
    if (B.cb[d] < 1 || B.cb[d] > 4096) return set_error("coarse_blocks out of range"), GMG_ERR_INVALID_ARG;
  }
  int e[3], zero[3] = {0, 0, 0};
  B.bext(1, e);
  for (int z = 0; z < e[2]; z++)
    for (int y = 0; y < e[1]; y++)
      for (int x = 0; x < e[0]; x++) {
        int b[3] = {x, y, z};
        B.add(1, b, -1, zero);
      }
  // refinement asked level by level
  for (int l = 1; l < dom->max_level; l++) {
    size_t cnt = B.lists[B.lidx(l)].size();
    for (size_t i = 0; i < cnt; i++) {
      int id = B.lists[B.lidx(l)][i];
      int b[3] = {B.blocks[id].ix[0], B.blocks[id].ix[1], B.blocks[id].ix[2]};
      if (!dom->refine || dom->refine(l, b, dom->refine_user)) B.refine(id);
    }
  }
  // 2:1 balance closure over faces, edges and corners
  bool changed = true;
  while (changed) {
    changed = false;
    for (int l = dom->max_level; l >= 2; l--) {
      B.bext(l, e);
      for (size_t i = 0; i < B.lists[B.lidx(l)].size(); i++) {
        int id = B.lists[B.lidx(l)][i];
        for (int dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); dz++)
          for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
              int q[3] = {B.blocks[id].ix[0] + dx, B.blocks[id].ix[1] + dy, B.blocks[id].ix[2] + dz};
              bool in = true;
              for (int d = 0; d < 3; d++) in = in && q[d] >= 0 && q[d] < e[d];
              if (!in) continue;
              int p[3] = {q[0] >> 1, q[1] >> 1, q[2] >> 1};
              if (B.find(l - 1, p) < 0) {
                B.ensure(l - 1, p);
                changed = true;
              }
            }
      }
    }
  }
  int lmax = 1;
  for (int l = 1; l <= dom->max_level; l++)
    if (!B.lists[B.lidx(l)].empty()) lmax = l;
  // coarse levels inside the root blocks
  int max_coarse = dom->max_coarse_cells > 0 ? dom->max_coarse_cells : (D == 2 ? 64 : 512);
  int lmin = 1;
  for (;;) {
    int n = B.n_of(lmin);
    long long cells = (long long)B.lists[B.lidx(lmin)].size() * (D == 3 ? n * n * n : n * n);
    if (cells <= max_coarse || (n & 1) || n / 2 < 2) break;
    std::vector<int> cur = B.lists[B.lidx(lmin)];
    for (int id : cur) {
      int b[3] = {B.blocks[id].ix[0], B.blocks[id].ix[1], B.blocks[id].ix[2]};
      int pid = B.add(lmin - 1, b, -1, zero);
      B.blocks[id].parent = pid;
      for (int d = 0; d < 3; d++) B.blocks[id].pofs[d] = 0;
      B.blocks[pid].child[0] = id;
      B.blocks[pid].has_children = 1;
    }
    lmin--;
  }
  if (lmax - lmin + 1 > kMaxLevels - 1) return set_error("too many levels"), GMG_ERR_INVALID_ARG;

  // canonical order: levels ascending, Morton inside a level
  std::vector<int> order;
  std::vector<int> newid(B.blocks.size(), -1);
  T->levels.clear();
  for (int l = lmin; l <= lmax; l++) {
    std::vector<int> v = B.lists[B.lidx(l)];
    std::sort(v.begin(), v.end(), [&](int a, int b) { return morton(B.blocks[a].ix, D) < morton(B.blocks[b].ix, D); });
    LevelInfo L;
    L.l = l;
    L.n = B.n_of(l);
    L.ncell = D == 3 ? L.n * L.n * L.n : L.n * L.n;
    L.first = (int)order.size();
    L.count = (int)v.size();
    L.h = std::ldexp(dom->h_root, 1 - l);
    B.bext(l, L.bext);
    for (int id : v) {
      newid[id] = (int)order.size();
      order.push_back(id);
    }
    T->levels.push_back(L);
  }
  long long off = 0;
  for (auto &L : T->levels) {
    L.off = off;
    off += (long long)L.count * L.ncell;
  }
  T->total_cells = off;
  T->D = D;
  T->N = N;
  T->max_level = dom->max_level;
  T->lmin = lmin;
  T->lmax = lmax;
  T->max_coarse = max_coarse;
  T->h1 = dom->h_root;
  for (int d = 0; d < 3; d++) {
    T->cb[d] = B.cb[d];
    T->lo[d] = d < D ? dom->lo[d] : 0.0;
  }
  int nb = (int)order.size();
  T->blocks.resize(nb);
  T->nbr_h.assign((size_t)nb * kNbr, -2);
  T->parent_h.assign(nb, -1);
  T->pofs_h.assign(nb, 0);
  T->flags_h.assign(nb, 0);
  T->leaf_ids_h.clear();
  T->n_leaf_cells = 0;
  for (int i = 0; i < nb; i++) {
    const TB &s = B.blocks[order[i]];
    HostBlock &h = T->blocks[i];
    h.level = s.level;
    for (int d = 0; d < 3; d++) {
      h.ix[d] = s.ix[d];
      h.pofs[d] = s.pofs[d];
    }
    h.parent = s.parent >= 0 ? newid[s.parent] : -1;
    for (int c = 0; c < 8; c++) h.child[c] = s.child[c] >= 0 ? newid[s.child[c]] : -1;
    h.has_children = s.has_children;
    T->parent_h[i] = h.parent;
    T->pofs_h[i] = h.pofs[0] | (h.pofs[1] << 10) | (h.pofs[2] << 20);
    int fl = h.has_children ? kHasChildren : 0;
    B.bext(h.level, e);
    for (int d = 0; d < D; d++) {
      if (h.ix[d] == 0) fl |= wall_bit(d, 0);
      if (h.ix[d] == e[d] - 1) fl |= wall_bit(d, 1);
    }
    T->flags_h[i] = fl;
    for (int dz = -1; dz <= 1; dz++)
      for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
          int slot = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
          if (D == 2 && dz != 0) continue;
          int q[3] = {h.ix[0] + dx, h.ix[1] + dy, h.ix[2] + dz};
          bool in = true;
          for (int d = 0; d < 3; d++) in = in && q[d] >= 0 && q[d] < e[d];
          if (!in) {
            T->nbr_h[(size_t)i * kNbr + slot] = -2;
            continue;
          }
          int f = B.find(h.level, q);
          T->nbr_h[(size_t)i * kNbr + slot] = f >= 0 ? newid[f] : -1;
        }
    if (!h.has_children) {
      T->leaf_ids_h.push_back(i);
      T->n_leaf_cells += T->lev(h.level).ncell;
    }
  }
  T->adaptive = false;
  for (int id : T->leaf_ids_h)
    if (T->blocks[id].level != lmax) T->adaptive = true;
  return GMG_OK;
}

// ---------------------------------------------------------------------------
// boundary set-up

namespace {

// Level set sampled on a uniform grid (GMG_LSF_GRID): (bi/tri)linear
// interpolation between the 2^D samples around x; coordinates outside the
// sampled box are clamped to it.  p[0..2] counts, p[3..5] position of
// sample 0, p[6..8] spacing; samples x fastest.
double grid_lsf(const double *p, const double *v, int D, const double *x) {
  int i0[3] = {0, 0, 0};
  double w[3] = {0.0, 0.0, 0.0};
  const long long stride[3] = {1, (long long)p[0], (long long)p[0] * (long long)p[1]};
  for (int d = 0; d < D; d++) {
    const int n = (int)p[d];
    double t = (x[d] - p[3 + d]) / p[6 + d];
    t = std::min(std::max(t, 0.0), (double)(n - 1));
    const int i = std::min((int)std::floor(t), n - 2);
    i0[d] = i;
    w[d] = t - i;
  }
  double s = 0.0;
  for (int corner = 0; corner < (1 << D); corner++) {
    double wt = 1.0;
    long long idx = 0;
    for (int d = 0; d < D; d++) {
      const int b = (corner >> d) & 1;
      wt *= b ? w[d] : 1.0 - w[d];
      idx += (long long)(i0[d] + b) * stride[d];
    }
    s += wt * v[idx];
  }
  return s;
}

struct HostLsf {
  const gmg_lsf *L;
  LsfSpec spec;
  int D;
  double operator()(const double *x) const {
    if (L->kind == GMG_LSF_CALLBACK) {
      double xx[3] = {x[0], D > 1 ? x[1] : 0.0, D > 2 ? x[2] : 0.0};
      return L->fn(xx, L->user);
    }
    if (L->kind == GMG_LSF_GRID) return grid_lsf(L->p, static_cast<const double *>(L->user), D, x);
    return lsf_builtin(spec, D, x);
  }
};

void cell_center(const gmg_tree *T, const HostBlock &B, const LevelInfo &L, const int *p, double *x) {
  for (int d = 0; d < 3; d++)
    x[d] = d < T->D ? T->lo[d] + ((double)(B.ix[d] * L.n + p[d]) + 0.5) * L.h : 0.0;
}

bool in_domain(const LevelInfo &L, int D, const int *G) {
  for (int d = 0; d < D; d++)
    if (G[d] < 0 || G[d] >= L.bext[d] * L.n) return false;
  return true;
}

// Sec. 3.6.3: gradient descent from a (mask set, no root found) toward f = 0
// with step w_min, at most floor(dx / w_min) steps; a sign change gives a
// virtual boundary toward the axis neighbour closest to the end point.
void unresolved_search(const gmg_tree *T, const HostLsf &f, const HostBlock &B, const LevelInfo &L, const int *p,
                       const double *a, double fa, double *dd) {
  int D = T->D;
  double w = T->prm.w_min, h = L.h;
  int nsteps = (int)std::floor(h / w);
  double x[3] = {a[0], a[1], a[2]};
  for (int s = 0; s < nsteps; s++) {
    double g[3] = {0, 0, 0}, gn = 0.0;
    for (int k = 0; k < D; k++) {
      double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
      xp[k] = x[k] + w;
      xm[k] = x[k] - w;
      g[k] = (f(xp) - f(xm)) / (2.0 * w);
      gn = gn + g[k] * g[k];
    }
    gn = std::sqrt(gn);
    if (!(gn > 0.0)) return;
    double sgn = fa > 0.0 ? -1.0 : 1.0;
    for (int k = 0; k < D; k++) x[k] = x[k] + w * (sgn * g[k] / gn);
    double fx = f(x);
    if (fa * fx <= 0.0) {
      double t = bisect_root(f, D, a, x, fa, 1.0, T->prm.eps_tol);
      double dist = 0.0;
      for (int k = 0; k < D; k++) dist = dist + (x[k] - a[k]) * (x[k] - a[k]);
      dist = t * std::sqrt(dist);
      double dv = dist / h;
      dv = dv < T->prm.eps_tol ? T->prm.eps_tol : (dv > 1.0 ? 1.0 : dv);
      int ax = 0;
      double best = std::fabs(x[0] - a[0]);
      for (int k = 1; k < D; k++)
        if (std::fabs(x[k] - a[k]) > best) {
          best = std::fabs(x[k] - a[k]);
          ax = k;
        }
      int side = x[ax] - a[ax] > 0.0 ? 1 : 0;
      int G[3];
      for (int d = 0; d < 3; d++) G[d] = d < D ? B.ix[d] * L.n + p[d] : 0;
      G[ax] += side ? 1 : -1;
      if (in_domain(L, D, G)) dd[2 * ax + side] = dv;
      return;
    }
  }
}

// dense LU with partial pivoting, then the explicit inverse (column solves)
bool invert(int n, std::vector<double> &A, std::vector<double> &inv) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; k++) {
    int pr = k;
    double best = std::fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; i++) {
      double v = std::fabs(A[(size_t)i * n + k]);
      if (v > best) {
        best = v;
        pr = i;
      }
    }
    if (best == 0.0) return false;
    piv[k] = pr;
    if (pr != k)
      for (int j = 0; j < n; j++) std::swap(A[(size_t)k * n + j], A[(size_t)pr * n + j]);
    double inv_p = 1.0 / A[(size_t)k * n + k];
    for (int i = k + 1; i < n; i++) {
      double m = A[(size_t)i * n + k] * inv_p;
      A[(size_t)i * n + k] = m;
      if (m != 0.0)
        for (int j = k + 1; j < n; j++) A[(size_t)i * n + j] -= m * A[(size_t)k * n + j];
    }
  }
  inv.assign((size_t)n * n, 0.0);
  std::vector<double> x(n);
  for (int c = 0; c < n; c++) {
    std::fill(x.begin(), x.end(), 0.0);
    x[c] = 1.0;
    for (int k = 0; k < n; k++) std::swap(x[k], x[piv[k]]);
    for (int i = 0; i < n; i++) {
      double s = x[i];
      for (int j = 0; j < i; j++) s -= A[(size_t)i * n + j] * x[j];
      x[i] = s;
    }
    for (int i = n - 1; i >= 0; i--) {
      double s = x[i];
      for (int j = i + 1; j < n; j++) s -= A[(size_t)i * n + j] * x[j];
      x[i] = s / A[(size_t)i * n + i];
    }
    for (int i = 0; i < n; i++) inv[(size_t)i * n + c] = x[i];
  }
  return true;
}

// Eq. (lpl-1d-lsf) per dimension for every cell of block B from its distances
// dd[nc x 2D]: the stencil st[(2D+1) x nc], the boundary value phi_b(x0) at
// each located root pb[nc x 2D] (0 where d = 1) and the right-hand-side term
// bt[nc] (moved coefficients times phi_b, plus the Dirichlet wall terms).
// The full set-up and gmg_set_boundary_value share it.
void block_terms(const gmg_tree *T, const HostBlock &B, const LevelInfo &L, const double *dd, bool cut, gmg_fn phib,
                 void *phib_user, double phib_const, std::vector<double> &st, std::vector<double> &bt,
                 std::vector<double> &pb) {
  const int D = T->D, S = 2 * D + 1, n = L.n, nc = L.ncell;
  const double h = L.h;
  pb.assign((size_t)nc * 2 * D, 0.0);
  st.assign((size_t)S * nc, 0.0);
  bt.assign(nc, 0.0);
  const double inv_h2 = 1.0 / (h * h);
  for (int c = 0; c < nc; c++) {
    int p[3] = {c % n, (c / n) % n, D == 3 ? c / (n * n) : 0};
    double a[3];
    cell_center(T, B, L, p, a);
    const double *dc = &dd[(size_t)c * 2 * D];
    double diag = 0.0, bnd = 0.0;
    double coef[6];
    for (int k = 0; k < D; k++) {
      double dm = dc[2 * k], dp = dc[2 * k + 1];
      double cm = 2.0 * inv_h2 / ((dp + dm) * dm);
      double cp = 2.0 * inv_h2 / ((dp + dm) * dp);
      diag = diag - (cm + cp);
      if (dm < 1.0) {
        double x0[3] = {a[0], a[1], a[2]};
        x0[k] = a[k] - dm * h;
        pb[(size_t)c * 2 * D + 2 * k] = phib ? phib(x0, phib_user) : phib_const;
        bnd = bnd + cm * pb[(size_t)c * 2 * D + 2 * k];
        cm = 0.0;
      }
      if (dp < 1.0) {
        double x0[3] = {a[0], a[1], a[2]};
        x0[k] = a[k] + dp * h;
        pb[(size_t)c * 2 * D + 2 * k + 1] = phib ? phib(x0, phib_user) : phib_const;
        bnd = bnd + cp * pb[(size_t)c * 2 * D + 2 * k + 1];
        cp = 0.0;
      }
      coef[2 * k] = cm;
      coef[2 * k + 1] = cp;
    }
    st[c] = diag;
    for (int k = 0; k < 2 * D; k++) st[(size_t)(1 + k) * nc + c] = coef[k];
    // Dirichlet wall terms (ghost 2 phi_w - phi_i): coefficient * 2 phi_w
    double t = cut ? bnd : 0.0;
    for (int k = 0; k < D; k++)
      for (int s = 0; s < 2; s++) {
        int G[3];
        for (int d = 0; d < 3; d++) G[d] = d < D ? B.ix[d] * n + p[d] : 0;
        G[k] += s ? 1 : -1;
        if (in_domain(L, D, G)) continue;
        int w = 2 * k + s;
        if (T->wall_type[w] != GMG_WALL_DIRICHLET) continue;
        double cw = cut ? coef[2 * k + s] : inv_h2;
        double xf[3] = {a[0], a[1], a[2]};
        xf[k] = s ? a[k] + 0.5 * h : a[k] - 0.5 * h;
        double v = T->wall_fn ? T->wall_fn(xf, T->wall_user) : T->wall_val[w];
        t = t + cw * (2.0 * v);
      }
    bt[c] = t;
  }
}

// The right-hand-side terms of a block no boundary crosses: only the
// Dirichlet wall terms of the cells beside a domain wall, with the regular
// coefficient 1 / dx^2 (block_terms' values for such a block, in its order).
// Returns false when every term is zero.
bool wall_terms(const gmg_tree *T, const HostBlock &B, const LevelInfo &L, std::vector<double> &bt) {
  const int D = T->D, n = L.n, nc = L.ncell;
  const double h = L.h, inv_h2 = 1.0 / (h * h);
  bool touches = false;
  for (int k = 0; k < D && !touches; k++)
    touches = (T->wall_type[2 * k] == GMG_WALL_DIRICHLET && B.ix[k] == 0) ||
              (T->wall_type[2 * k + 1] == GMG_WALL_DIRICHLET && B.ix[k] + 1 >= L.bext[k]);
  if (!touches) return false;
  bt.assign(nc, 0.0);
  bool any = false;
  for (int c = 0; c < nc; c++) {
    int p[3] = {c % n, (c / n) % n, D == 3 ? c / (n * n) : 0};
    bool shell = false;  // beside one of the block's faces (others have no wall term)
    for (int k = 0; k < D; k++) shell = shell || p[k] == 0 || p[k] == n - 1;
    if (!shell) continue;
    double t = 0.0;
    for (int k = 0; k < D; k++)
      for (int s = 0; s < 2; s++) {
        int G[3];
        for (int d = 0; d < 3; d++) G[d] = d < D ? B.ix[d] * n + p[d] : 0;
        G[k] += s ? 1 : -1;
        if (in_domain(L, D, G)) continue;
        int w = 2 * k + s;
        if (T->wall_type[w] != GMG_WALL_DIRICHLET) continue;
        double a[3];
        cell_center(T, B, L, p, a);
        double xf[3] = {a[0], a[1], a[2]};
        xf[k] = s ? a[k] + 0.5 * h : a[k] - 0.5 * h;
        double v = T->wall_fn ? T->wall_fn(xf, T->wall_user) : T->wall_val[w];
        t = t + inv_h2 * (2.0 * v);
      }
    bt[c] = t;
    any = any || t != 0.0;
  }
  return any;
}

}  // namespace

int host_setup(gmg_tree *T, const gmg_lsf *lsf, gmg_fn phib, void *phib_user, double phib_const,
               const gmg_tree *reuse) {
  const int D = T->D, S = 2 * D + 1;
  gmg_lsf none{};
  none.kind = GMG_LSF_NONE;
  if (!lsf) lsf = &none;
  if (lsf->kind < GMG_LSF_NONE || lsf->kind > GMG_LSF_GRID || (lsf->kind == GMG_LSF_CALLBACK && !lsf->fn))
    return set_error("invalid level-set specification"), GMG_ERR_INVALID_ARG;
  if (lsf->kind == GMG_LSF_GRID) {
    bool ok = lsf->user != nullptr;
    for (int d = 0; d < D; d++) ok = ok && lsf->p[d] >= 2.0 && lsf->p[6 + d] > 0.0;
    if (!ok) return set_error("grid level set: samples, counts >= 2 and spacings > 0 needed"), GMG_ERR_INVALID_ARG;
  }
  T->lsf_spec = *lsf;
  T->phib_fn = phib;
  T->phib_user = phib_user;
  T->phib_const = phib_const;
  HostLsf f{lsf, LsfSpec{}, D};
  f.spec.kind = lsf->kind;
  std::memcpy(f.spec.p, lsf->p, sizeof(f.spec.p));
  const bool have = lsf->kind != GMG_LSF_NONE;
  const int nb = (int)T->blocks.size();
  T->st_base_h.assign(nb, -1);
  T->bt_base_h.assign(nb, -1);
  T->wallv_base_h.assign(nb, -1);
  T->wallv_h.clear();
  T->bphib_h.clear();
  T->dist_base_h.assign(nb, -1);
  T->mask_base_h.assign(nb, -1);
  T->stencil_h.clear();
  T->spec_h.clear();
  T->bterm_h.clear();
  T->dist_h.clear();
  T->mask_h.clear();
  // Per-block work (mask, line searches, stencils, boundary terms) runs in
  // parallel threads when no host callback is involved (callbacks may not be
  // thread-safe); the results are then concatenated in block order, so the
  // stores are the same whatever the thread count.
  struct BlockOut {
    std::vector<uint8_t> mask;   // bit 0: Eq. (boundary-mask); bit 1: cell centre inside the object
    std::vector<double> dd, st, bt, pb, wv;
    bool cut = false, anybt = false;
  };
  std::vector<BlockOut> outs(nb);
  // boundary detection of a built-in level set on the device (bit for bit
  // the loops below); the host keeps callbacks and sampled level sets
  std::vector<uint8_t> dev_mask;
  std::vector<long long> dev_cells, cell_first, entry_first;
  std::vector<double> dev_dist;
  DeviceTerms dev_terms;
  std::vector<int> dev_cut_index;  // block -> its index among the device's cut blocks, -1 none
  const bool on_device = T->setup_on_device && !reuse &&
                         (lsf->kind == GMG_LSF_SPHERE || lsf->kind == GMG_LSF_CAPSULE ||
                          lsf->kind == GMG_LSF_ELLIPSOID) && device_setup_available();
  if (on_device) {
    // the stencils and terms too when the boundary and wall values are constants
    const bool terms = !phib && !T->wall_fn;
    const int rc = device_boundary_detection(T, f.spec, dev_mask, dev_cells, dev_dist, terms ? &dev_terms : nullptr,
                                             phib_const);
    if (rc) return rc;
    if (terms) {
      dev_cut_index.assign(nb, -1);
      for (size_t i = 0; i < dev_terms.cut_ids.size(); i++) dev_cut_index[dev_terms.cut_ids[i]] = (int)i;
    }
    cell_first.assign(nb + 1, 0);
    for (int b = 0; b < nb; b++) cell_first[b + 1] = cell_first[b] + T->lev(T->blocks[b].level).ncell;
    entry_first.assign(nb + 1, 0);
    for (int b = 0; b < nb; b++)
      entry_first[b + 1] =
          std::lower_bound(dev_cells.begin(), dev_cells.end(), cell_first[b + 1]) - dev_cells.begin();
  }
  T->setup_device = on_device;
  // Dirichlet values at the centres of a block's faces on upper domain walls
  // (axis k, face cell j over the other axes in increasing order), for the
  // field evaluation on upper cell faces
  auto wall_values = [&](BlockOut &o, const HostBlock &B, const LevelInfo &L) {
    const int n = L.n;
    const double h = L.h;
    {
      const int nf = D == 3 ? n * n : n;
      bool upper = false;
      std::vector<double> wv((size_t)D * nf, 0.0);
      for (int k = 0; k < D; k++)
        for (int j = 0; j < nf; j++) {
          const int u = j % n, v = D == 3 ? j / n : 0;
          int p[3] = {0, 0, 0};
          p[k] = n - 1;
          p[k == 0 ? 1 : 0] = u;
          if (D == 3) p[k == 2 ? 1 : 2] = v;
          int G[3];
          for (int d = 0; d < 3; d++) G[d] = d < D ? B.ix[d] * n + p[d] : 0;
          G[k] += 1;
          if (in_domain(L, D, G)) continue;
          upper = true;
          if (T->wall_type[2 * k + 1] != GMG_WALL_DIRICHLET) continue;
          double a[3];
          cell_center(T, B, L, p, a);
          a[k] += 0.5 * h;
          wv[(size_t)k * nf + j] = T->wall_fn ? T->wall_fn(a, T->wall_user) : T->wall_val[2 * k + 1];
        }
      if (upper) o.wv = std::move(wv);
    }
  };
  auto process = [&](int id, BlockOut &o) {
    const HostBlock &B = T->blocks[id];
    const LevelInfo &L = T->lev(B.level);
    const int n = L.n, nc = L.ncell;
    const double h = L.h;
    const double Lmask = T->prm.mask_factor * std::sqrt((double)D) * h;
    // distances (1 = no root) only for blocks with a masked cell
    std::vector<double> dd, pb, st, bt;
    auto dist_of = [&](int c) {
      if (dd.empty()) dd.assign((size_t)nc * 2 * D, 1.0);
      return &dd[(size_t)c * 2 * D];
    };
    bool cut = false;
    if (on_device && !dev_cut_index.empty()) {  // everything from the device
      o.mask.assign(dev_mask.begin() + cell_first[id], dev_mask.begin() + cell_first[id + 1]);
      const int ci = dev_cut_index[id];
      if (ci >= 0) {
        const long long a = dev_terms.cell_off[ci], e = dev_terms.cell_off[ci + 1];
        o.cut = true;
        o.dd.assign(dev_terms.dd.begin() + a * 2 * D, dev_terms.dd.begin() + e * 2 * D);
        o.pb.assign(dev_terms.pb.begin() + a * 2 * D, dev_terms.pb.begin() + e * 2 * D);
        o.st.assign(dev_terms.st.begin() + a * S, dev_terms.st.begin() + e * S);
        bt.assign(dev_terms.bt.begin() + a, dev_terms.bt.begin() + e);
        for (int c = 0; c < nc; c++) o.anybt = o.anybt || bt[c] != 0.0;
      } else {
        o.anybt = wall_terms(T, B, L, bt);
      }
      wall_values(o, B, L);
      if (o.anybt) o.bt = std::move(bt);
      return;
    }
    if (on_device) {
      o.mask.assign(dev_mask.begin() + cell_first[id], dev_mask.begin() + cell_first[id + 1]);
      for (long long e = entry_first[id]; e < entry_first[id + 1]; e++) {
        double *dc = dist_of((int)(dev_cells[e] - cell_first[id]));
        for (int k = 0; k < 2 * D; k++) {
          dc[k] = dev_dist[(size_t)e * 2 * D + k];
          if (dc[k] < 1.0) cut = true;
        }
      }
    } else {
      o.mask.assign(nc, 0);
    }
    uint8_t *mask = o.mask.data();
    for (int c = 0; c < nc; c++) {
      int p[3] = {c % n, (c / n) % n, D == 3 ? c / (n * n) : 0};
      if (!have || on_device) break;
      double a[3];
      cell_center(T, B, L, p, a);
      double fa = f(a);
      if (fa < 0.0) mask[c] |= 2;
      // Eq. (boundary-mask) with a central-difference gradient
      double gn = 0.0;
      for (int k = 0; k < D; k++) {
        double xp[3] = {a[0], a[1], a[2]}, xm[3] = {a[0], a[1], a[2]};
        xp[k] = a[k] + h;
        xm[k] = a[k] - h;
        double g = (f(xp) - f(xm)) / (2.0 * h);
        gn = gn + g * g;
      }
      gn = std::sqrt(gn);
      if (!(std::fabs(fa) < Lmask * gn)) continue;
      mask[c] |= 1;
      double *dc = dist_of(c);
      bool found = false;
      for (int k = 0; k < D; k++)
        for (int s = 0; s < 2; s++) {
          int G[3];
          for (int d = 0; d < 3; d++) G[d] = d < D ? B.ix[d] * n + p[d] : 0;
          G[k] += s ? 1 : -1;
          if (!in_domain(L, D, G)) continue;
          double bp[3] = {a[0], a[1], a[2]};
          bp[k] = s ? a[k] + h : a[k] - h;
          dc[2 * k + s] = line_search(f, D, a, bp, T->prm.eps_tol);
          if (dc[2 * k + s] < 1.0) found = true;
        }
      if (!found && T->prm.w_min > 0.0 && h > T->prm.w_min) unresolved_search(T, f, B, L, p, a, fa, dc);
      for (int k = 0; k < 2 * D; k++)
        if (dc[k] < 1.0) cut = true;
    }
    if (cut) {  // Eq. (lpl-1d-lsf) stencils and the moved terms
      block_terms(T, B, L, dd.data(), cut, phib, phib_user, phib_const, st, bt, pb);
      for (int c = 0; c < nc; c++) o.anybt = o.anybt || bt[c] != 0.0;
      o.st = std::move(st);
      o.dd = std::move(dd);
      o.pb = std::move(pb);
    } else {  // the regular stencil: only Dirichlet wall terms
      o.anybt = wall_terms(T, B, L, bt);
    }
    o.cut = cut;
    wall_values(o, B, L);
    if (o.anybt) o.bt = std::move(bt);
  };
  // Re-meshing (Sec. 4.5: boundary detection only for newly added cells):
  // a block that also exists in `reuse` (same level and coordinates) takes
  // that tree's set-up, which depends only on the block's own cells.
  std::unordered_map<long long, int> old_ids;
  auto key = [](int level, const int *ix) {
    return ((long long)(level + 64) << 57) | ((long long)ix[2] << 38) | ((long long)ix[1] << 19) | (long long)ix[0];
  };
  if (reuse)
    for (size_t b = 0; b < reuse->blocks.size(); b++) old_ids[key(reuse->blocks[b].level, reuse->blocks[b].ix)] = (int)b;
  auto reuse_block = [&](int id, BlockOut &o) {
    if (!reuse) return false;
    const HostBlock &B = T->blocks[id];
    auto it = old_ids.find(key(B.level, B.ix));
    if (it == old_ids.end()) return false;
    const gmg_tree *R = reuse;
    const int b = it->second, nc = T->lev(B.level).ncell, nf = D == 3 ? T->lev(B.level).n * T->lev(B.level).n
                                                                      : T->lev(B.level).n;
    o.mask.assign(R->mask_h.begin() + R->mask_base_h[b], R->mask_h.begin() + R->mask_base_h[b] + nc);
    o.cut = R->st_base_h[b] >= 0;
    if (o.cut) {
      o.st.assign(R->stencil_h.begin() + R->st_base_h[b], R->stencil_h.begin() + R->st_base_h[b] + (size_t)S * nc);
      o.dd.assign(R->dist_h.begin() + R->dist_base_h[b], R->dist_h.begin() + R->dist_base_h[b] + (size_t)2 * D * nc);
      o.pb.assign(R->bphib_h.begin() + R->dist_base_h[b], R->bphib_h.begin() + R->dist_base_h[b] + (size_t)2 * D * nc);
    }
    o.anybt = R->bt_base_h[b] >= 0;
    if (o.anybt) o.bt.assign(R->bterm_h.begin() + R->bt_base_h[b], R->bterm_h.begin() + R->bt_base_h[b] + nc);
    if (R->wallv_base_h[b] >= 0)
      o.wv.assign(R->wallv_h.begin() + R->wallv_base_h[b], R->wallv_h.begin() + R->wallv_base_h[b] + (size_t)D * nf);
    return true;
  };
  std::atomic<long long> n_reused{0};
  auto setup_block = [&](int id, BlockOut &o) {
    if (reuse_block(id, o))
      n_reused.fetch_add(1);
    else
      process(id, o);
  };
  const bool callbacks = lsf->kind == GMG_LSF_CALLBACK || phib || T->wall_fn;
  int nthreads = callbacks ? 1 : (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 64u);
  if (const char *e = std::getenv("GMG_SETUP_THREADS")) nthreads = std::max(1, std::atoi(e));
  if (nthreads <= 1 || nb < 64) {
    for (int id = 0; id < nb; id++) setup_block(id, outs[id]);
  } else {
    std::atomic<int> next{0};
    std::vector<std::thread> pool;
    for (int w = 0; w < nthreads; w++)
      pool.emplace_back([&] {
        for (int id; (id = next.fetch_add(16)) < nb;)
          for (int k = id; k < std::min(nb, id + 16); k++) setup_block(k, outs[k]);
      });
    for (auto &th : pool) th.join();
  }
  T->setup_reused = n_reused.load();
  T->setup_computed = nb - T->setup_reused;
  for (int id = 0; id < nb; id++) {
    BlockOut &o = outs[id];
    const int nc = (int)o.mask.size();
    T->mask_base_h[id] = (long long)T->mask_h.size();
    T->mask_h.insert(T->mask_h.end(), o.mask.begin(), o.mask.end());
    if (o.cut) {
      T->st_base_h[id] = (long long)T->stencil_h.size();
      T->stencil_h.insert(T->stencil_h.end(), o.st.begin(), o.st.end());
      for (int c = 0; c < nc; c++) {  // cells whose stencil differs from the regular one
        bool special = false;
        for (int k = 0; k < 2 * D; k++) special = special || o.dd[(size_t)c * 2 * D + k] < 1.0;
        T->spec_h.push_back(special ? 1 : 0);
      }
      T->dist_base_h[id] = (long long)T->dist_h.size();
      T->dist_h.insert(T->dist_h.end(), o.dd.begin(), o.dd.end());
      T->bphib_h.insert(T->bphib_h.end(), o.pb.begin(), o.pb.end());
    }
    if (!o.wv.empty()) {
      T->wallv_base_h[id] = (long long)T->wallv_h.size();
      T->wallv_h.insert(T->wallv_h.end(), o.wv.begin(), o.wv.end());
    }
    if (o.anybt) {
      T->bt_base_h[id] = (long long)T->bterm_h.size();
      T->bterm_h.insert(T->bterm_h.end(), o.bt.begin(), o.bt.end());
    }
    o = BlockOut();  // release the block's buffers
  }
  // coarsest level: explicit inverse of its operator (homogeneous walls)
  const LevelInfo &Lc = T->lev(T->lmin);
  const int ncl = Lc.ncell, n = Lc.n, nbc = Lc.count, M = nbc * ncl;
  if (M > 8192) return set_error("coarsest level too large for the direct solve"), GMG_ERR_INVALID_ARG;
  std::vector<double> A((size_t)M * M, 0.0);
  const double inv_h2 = 1.0 / (Lc.h * Lc.h);
  for (int i = 0; i < nbc; i++) {
    int id = Lc.first + i;
    const HostBlock &B = T->blocks[id];
    const double *stb = T->st_base_h[id] >= 0 ? &T->stencil_h[T->st_base_h[id]] : nullptr;
    for (int c = 0; c < ncl; c++) {
      int p[3] = {c % n, (c / n) % n, D == 3 ? c / (n * n) : 0};
      int row = i * ncl + c;
      A[(size_t)row * M + row] += stb ? stb[c] : -2.0 * D * inv_h2;
      for (int k = 0; k < D; k++)
        for (int s = 0; s < 2; s++) {
          double cf = stb ? stb[(size_t)(1 + 2 * k + s) * ncl + c] : inv_h2;
          int G[3];
          for (int d = 0; d < 3; d++) G[d] = d < D ? B.ix[d] * n + p[d] : 0;
          G[k] += s ? 1 : -1;
          if (!in_domain(Lc, D, G)) {
            A[(size_t)row * M + row] += (T->wall_type[2 * k + s] == GMG_WALL_DIRICHLET ? -1.0 : 1.0) * cf;
            continue;
          }
          int bix[3] = {0, 0, 0}, q[3] = {0, 0, 0};
          for (int d = 0; d < D; d++) {
            bix[d] = G[d] / n;
            q[d] = G[d] - bix[d] * n;
          }
          // same-level block: coarsest level holds every block of the root grid
          int j = -1;
          for (int t = 0; t < nbc; t++) {
            const HostBlock &O = T->blocks[Lc.first + t];
            if (O.ix[0] == bix[0] && O.ix[1] == bix[1] && O.ix[2] == bix[2]) {
              j = t;
              break;
            }
          }
          int col = j * ncl + q[0] + n * (q[1] + n * q[2]);
          A[(size_t)row * M + col] += cf;
        }
    }
  }
  T->nc = M;
  T->ncr = M;
  T->nroot = 1;
  if (!invert(M, A, T->cinv_h)) return set_error("singular coarsest-level operator"), GMG_ERR_INVALID_ARG;
  build_cut_lists(T);
  T->stencils_ready = true;
  return GMG_OK;
}

// The cells of every cut block whose stencil differs from the regular one
// (spec flag set), listed per colour in cell order, with their stored
// coefficients: the kernels fetch a block's short lists up front instead of
// reading the dense stencil pool cell by cell.
void build_cut_lists(gmg_tree *T) {
  const int D = T->D, S = 2 * D + 1;
  const size_t nb = T->blocks.size();
  T->cut_list_h.assign(4 * nb, 0);
  T->cut_cell_h.clear();
  T->cut_max_h.assign(T->levels.size(), 0);
  std::vector<std::vector<double>> coef(S);
  for (size_t b = 0; b < nb; b++) {
    const long long sb = T->st_base_h[b];
    if (sb < 0) continue;
    const int lv = T->blocks[b].level;
    const int n = T->lev(lv).n, nc = T->lev(lv).ncell;
    const long long fb = sb / S;
    int *ent = &T->cut_list_h[4 * b];
    ent[0] = (int)T->cut_cell_h.size();
    for (int col = 0; col < 2; col++) {
      int m = 0;
      for (int c = 0; c < nc; c++) {
        const int x = c % n, y = (c / n) % n, z = D == 3 ? c / (n * n) : 0;
        if (((x + y + z) & 1) != col || !T->spec_h[fb + c]) continue;
        T->cut_cell_h.push_back(c);
        for (int k = 0; k < S; k++) coef[k].push_back(T->stencil_h[sb + (size_t)k * nc + c]);
        m++;
      }
      ent[1 + col] = m;
    }
    int &mx = T->cut_max_h[lv - T->lmin];
    mx = std::max(mx, ent[1] + ent[2]);
  }
  T->n_cut = (long long)T->cut_cell_h.size();
  T->cut_coef_h.clear();
  T->cut_coef_h.reserve((size_t)S * T->n_cut);
  for (int k = 0; k < S; k++) T->cut_coef_h.insert(T->cut_coef_h.end(), coef[k].begin(), coef[k].end());
}

}  // namespace gmg

extern "C" {

int gmg_set_boundary_value(gmg_tree *t, gmg_fn phib, void *phib_user, double phib_const) {
  using namespace gmg;
  if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
  if (!t->stencils_ready || t->bound || t->ntree != 1)
    return set_error("the boundary value changes after gmg_store_stencils and before gmg_tree_bind, on a single tree"),
           GMG_ERR_STATE;
  std::vector<double> st, bt, pb;
  for (size_t id = 0; id < t->blocks.size(); id++) {
    const long long db = t->dist_base_h[id];
    if (db < 0) continue;  // no cut: the block's terms do not involve phi_b
    const HostBlock &B = t->blocks[id];
    const LevelInfo &L = t->lev(B.level);
    const int nc = L.ncell;
    block_terms(t, B, L, &t->dist_h[db], true, phib, phib_user, phib_const, st, bt, pb);
    std::copy(pb.begin(), pb.end(), t->bphib_h.begin() + db);
    bool any = false;
    for (int c = 0; c < nc; c++) any = any || bt[c] != 0.0;
    if (t->bt_base_h[id] >= 0) {
      std::copy(bt.begin(), bt.end(), t->bterm_h.begin() + t->bt_base_h[id]);
    } else if (any) {
      t->bt_base_h[id] = (long long)t->bterm_h.size();
      t->bterm_h.insert(t->bterm_h.end(), bt.begin(), bt.end());
    }
  }
  t->phib_fn = phib;
  t->phib_user = phib_user;
  t->phib_const = phib_const;
  return GMG_OK;
}

int gmg_get_boundary_terms(const gmg_tree *t, int level, double *out) {
  using namespace gmg;
  if (!t || !out || !t->stencils_ready || level < t->lmin || level > t->lmax)
    return set_error("bad arguments or stencils not stored"), GMG_ERR_INVALID_ARG;
  const LevelInfo &L = t->lev(level);
  size_t k = 0;
  for (int i = 0; i < L.count; i++) {
    const long long bb = t->bt_base_h[L.first + i];
    for (int c = 0; c < L.ncell; c++) out[k++] = bb >= 0 ? t->bterm_h[bb + c] : 0.0;
  }
  return GMG_OK;
}

}  // extern "C"
