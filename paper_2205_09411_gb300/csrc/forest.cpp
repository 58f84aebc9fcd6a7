// Forests: many independent problems in one block structure.
//
// gmg_forest_create merges set-up trees (each with one root block, its own
// level set, boundary values and refinement) into one gmg_tree whose level l
// holds the level-l blocks of every tree, tree after tree.  The trees share
// no neighbours, so every kernel of a V-cycle runs over all trees at once
// while each tree's arithmetic stays that of its own V-cycle (Sec. 2.2):
// the coarsest level holds one block per tree with its own direct-solve
// inverse, norms are reduced per tree, and a tree that has converged is
// frozen like a right-hand-side slot.
#include <cmath>
#include <string>
#include <vector>

#include "gmg_internal.h"

namespace gmg {

namespace {

bool same_shape(const gmg_tree *a, const gmg_tree *b, std::string *why) {
  if (a->D != b->D || a->N != b->N) return *why = "trees differ in dimension or block size", false;
  if (a->lmin != b->lmin) return *why = "trees differ in their coarsest level", false;
  if (std::fabs(a->h1 - b->h1) > 1e-15 * a->h1) return *why = "trees differ in root cell size", false;
  if (a->prm.n_down != b->prm.n_down || a->prm.n_up != b->prm.n_up)
    return *why = "trees differ in their sweep counts", false;
  for (int w = 0; w < 2 * a->D; w++)
    if (a->wall_type[w] != b->wall_type[w]) return *why = "trees differ in wall types", false;
  if (a->ncr != b->ncr) return *why = "trees differ in their coarsest-level size", false;
  return true;
}

}  // namespace

int forest_merge(gmg_tree *const *trees, int n, gmg_tree **out) {
  const gmg_tree *t0 = trees[0];
  std::string why;
  for (int i = 0; i < n; i++) {
    const gmg_tree *t = trees[i];
    if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
    if (!t->stencils_ready) return set_error("every tree needs gmg_store_stencils first"), GMG_ERR_STATE;
    if (t->ntree != 1 || t->nroot != 1 || t->cb[0] * t->cb[1] * t->cb[2] != 1)
      return set_error("every tree of a forest must have exactly one root block"), GMG_ERR_INVALID_ARG;
    if (!same_shape(t0, t, &why)) return set_error(why), GMG_ERR_INVALID_ARG;
  }
  gmg_tree *F = new gmg_tree();
  F->D = t0->D;
  F->N = t0->N;
  F->lmin = t0->lmin;
  F->max_coarse = t0->max_coarse;
  F->h1 = t0->h1;
  F->prm = t0->prm;
  for (int d = 0; d < 3; d++) {
    F->cb[d] = 1;
    F->lo[d] = t0->lo[d];
  }
  for (int w = 0; w < 6; w++) F->wall_type[w] = t0->wall_type[w];
  F->lmax = F->lmin;
  for (int i = 0; i < n; i++) F->lmax = std::max(F->lmax, trees[i]->lmax);
  F->max_level = F->lmax;
  F->ntree = n;
  F->nroot = n;
  F->ncr = t0->ncr;
  F->nc = n * t0->ncr;

  // new ids: level by level, tree by tree, each tree's own order inside
  std::vector<std::vector<int>> map(n);
  for (int i = 0; i < n; i++) map[i].assign(trees[i]->blocks.size(), -1);
  F->levels.resize(F->lmax - F->lmin + 1);
  int next = 0;
  long long off = 0;
  for (int l = F->lmin; l <= F->lmax; l++) {
    LevelInfo &L = F->levels[l - F->lmin];
    const gmg_tree *ref = nullptr;
    for (int i = 0; i < n && !ref; i++)
      if (l <= trees[i]->lmax) ref = trees[i];
    const LevelInfo &R = ref->lev(l);
    L.l = l;
    L.n = R.n;
    L.ncell = R.ncell;
    L.h = R.h;
    L.first = next;
    L.off = off;
    for (int i = 0; i < n; i++) {
      const gmg_tree *t = trees[i];
      if (l > t->lmax) continue;
      const LevelInfo &Li = t->lev(l);
      for (int k = 0; k < Li.count; k++) map[i][Li.first + k] = next++;
    }
    L.count = next - L.first;
    off += (long long)L.count * L.ncell;
  }
  const int nb = next;
  F->total_cells = off;
  F->blocks.resize(nb);
  F->nbr_h.assign((size_t)nb * kNbr, -2);
  F->parent_h.assign(nb, -1);
  F->pofs_h.assign(nb, 0);
  F->flags_h.assign(nb, 0);
  F->st_base_h.assign(nb, -1);
  F->bt_base_h.assign(nb, -1);
  F->dist_base_h.assign(nb, -1);
  F->wallv_base_h.assign(nb, -1);
  F->mask_base_h.assign(nb, -1);
  F->tree_of_h.assign(nb, 0);
  F->tree_boff_h.assign(n + 1, 0);
  F->tree_leaf_off_h.assign(n + 1, 0);
  F->tree_lo_h.assign((size_t)3 * n, 0.0);
  long long st_off = 0, bt_off = 0, di_off = 0, ma_off = 0, sp_off = 0, wv_off = 0;
  for (int i = 0; i < n; i++) {
    const gmg_tree *t = trees[i];
    for (int d = 0; d < 3; d++) F->tree_lo_h[3 * i + d] = t->lo[d];
    const auto remap = [&](int id) { return id >= 0 ? map[i][id] : id; };
    for (size_t b = 0; b < t->blocks.size(); b++) {
      const int g = map[i][b];
      HostBlock h = t->blocks[b];
      h.parent = remap(h.parent);
      for (int c = 0; c < 8; c++) h.child[c] = remap(h.child[c]);
      F->blocks[g] = h;
      F->parent_h[g] = h.parent;
      F->pofs_h[g] = t->pofs_h[b];
      F->flags_h[g] = t->flags_h[b];
      for (int k = 0; k < kNbr; k++) F->nbr_h[(size_t)g * kNbr + k] = remap(t->nbr_h[b * kNbr + k]);
      F->tree_of_h[g] = i;
      if (t->st_base_h[b] >= 0) F->st_base_h[g] = t->st_base_h[b] + st_off;
      if (t->bt_base_h[b] >= 0) F->bt_base_h[g] = t->bt_base_h[b] + bt_off;
      if (t->dist_base_h[b] >= 0) F->dist_base_h[g] = t->dist_base_h[b] + di_off;
      if (t->mask_base_h[b] >= 0) F->mask_base_h[g] = t->mask_base_h[b] + ma_off;
      if (t->wallv_base_h[b] >= 0) F->wallv_base_h[g] = t->wallv_base_h[b] + wv_off;
    }
    // spec flags run parallel to the stencil pool (one flag per cell and
    // cut block, at st_base / (2D + 1))
    if ((long long)t->spec_h.size() * (2 * F->D + 1) != (long long)t->stencil_h.size())
      return delete F, set_error("inconsistent stencil store"), GMG_ERR_INVALID_ARG;
    if (sp_off * (2 * F->D + 1) != st_off) return delete F, set_error("inconsistent stencil store"), GMG_ERR_INVALID_ARG;
    F->stencil_h.insert(F->stencil_h.end(), t->stencil_h.begin(), t->stencil_h.end());
    F->spec_h.insert(F->spec_h.end(), t->spec_h.begin(), t->spec_h.end());
    F->bterm_h.insert(F->bterm_h.end(), t->bterm_h.begin(), t->bterm_h.end());
    F->dist_h.insert(F->dist_h.end(), t->dist_h.begin(), t->dist_h.end());
    F->bphib_h.insert(F->bphib_h.end(), t->bphib_h.begin(), t->bphib_h.end());
    F->wallv_h.insert(F->wallv_h.end(), t->wallv_h.begin(), t->wallv_h.end());
    F->mask_h.insert(F->mask_h.end(), t->mask_h.begin(), t->mask_h.end());
    st_off += (long long)t->stencil_h.size();
    sp_off += (long long)t->spec_h.size();
    bt_off += (long long)t->bterm_h.size();
    di_off += (long long)t->dist_h.size();
    ma_off += (long long)t->mask_h.size();
    wv_off += (long long)t->wallv_h.size();
    // the coarsest level's inverse of tree i (root i)
    F->cinv_h.insert(F->cinv_h.end(), t->cinv_h.begin(), t->cinv_h.end());
    // leaves tree-major, each tree in its own leaf order
    F->tree_leaf_off_h[i] = F->n_leaf_cells;
    for (int id : t->leaf_ids_h) F->leaf_ids_h.push_back(map[i][id]);
    F->n_leaf_cells += t->n_leaf_cells;
    // the blocks of tree i, for its norms
    F->tree_boff_h[i] = (int)F->tree_blocks_h.size();
    for (size_t b = 0; b < t->blocks.size(); b++) F->tree_blocks_h.push_back(map[i][b]);
  }
  F->tree_boff_h[n] = (int)F->tree_blocks_h.size();
  F->tree_leaf_off_h[n] = F->n_leaf_cells;
  // leaves on more than one level: the end-of-cycle restriction keeps
  // covered cells consistent (as for one adaptive tree)
  F->adaptive = false;
  for (int id : F->leaf_ids_h)
    if (F->blocks[id].level != F->lmax) F->adaptive = true;
  build_cut_lists(F);
  F->stencils_ready = true;
  *out = F;
  return GMG_OK;
}

}  // namespace gmg

extern "C" {

int gmg_forest_create(gmg_tree *const *trees, int n_trees, gmg_tree **out) {
  if (!trees || !out || n_trees < 1) return gmg::set_error("bad arguments"), GMG_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n_trees; i++)
    if (trees[i] && trees[i]->bound) return gmg::set_error("forest trees must not be bound"), GMG_ERR_STATE;
  return gmg::forest_merge(trees, n_trees, out);
}

int gmg_num_trees(const gmg_tree *t) { return t ? t->ntree : 0; }

int gmg_forest_tree_info(const gmg_tree *t, int tree, long long *leaf_offset, long long *n_leaf_cells) {
  if (!t || tree < 0 || tree >= t->ntree) return gmg::set_error("tree index out of range"), GMG_ERR_INVALID_ARG;
  if (t->ntree == 1) {
    if (leaf_offset) *leaf_offset = 0;
    if (n_leaf_cells) *n_leaf_cells = t->n_leaf_cells;
    return GMG_OK;
  }
  if (leaf_offset) *leaf_offset = t->tree_leaf_off_h[tree];
  if (n_leaf_cells) *n_leaf_cells = t->tree_leaf_off_h[tree + 1] - t->tree_leaf_off_h[tree];
  return GMG_OK;
}

}  // extern "C"
