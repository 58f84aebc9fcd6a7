// Internal declarations of the GB300 octree multigrid library (not part of
// the C ABI).  Host structures describe the block tree; the device view
// (GmgView) is what the kernels receive by value.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "gmg.h"

namespace gmg {

constexpr int kMaxLevels = 40;
constexpr int kCoopMaxBlocks = 160;  // levels with at most this many blocks join the cooperative coarse cycle
struct GridBar;
constexpr int kNbr = 27;  // 3x3x3 neighbour offsets (2D uses the dz = 0 plane)

// block flags
constexpr int kHasChildren = 1;
inline __host__ __device__ int wall_bit(int axis, int side) { return 2 << (2 * axis + side); }
// face f = 2 axis + side has a same-level neighbour with children (set at bind)
inline __host__ __device__ int face_covered_bit(int f) { return 1 << (16 + f); }

struct HostBlock {
  int level;
  int ix[3];
  int parent;
  int pofs[3];  // offset of this block's footprint in the parent, in parent cells
  int child[8];
  int has_children;
};

// One level of the hierarchy: blocks [first, first + count) in global id order.
struct LevelInfo {
  int l = 0, n = 0, ncell = 0, first = 0, count = 0;
  double h = 0.0;
  int bext[3] = {1, 1, 1};
  long long off = 0;  // first cell of the level in the field arrays
  std::vector<int> map;  // block coordinates -> global id (or -1)
};

// Per-level arguments passed to kernels.
struct LvArgs {
  int first, count, n, ncell;
  long long off;   // first cell of the level in the b / old / stencil-indexed fields
  double h;
  long long poff;  // first cell of the level in phi (off, or off + total cells in the second buffer)
  int nd, nu;      // red/black sweeps of the level on the way down / up
  double h2, ih2;  // h^2 and 1 / h^2, computed on the host (no FP64 division on the device)
};

// Everything a kernel needs to address the tree in device memory.
template <typename T>
struct GmgView {
  const int *nbr;        // [nb][27] same-level neighbour id, -1 none, -2 outside
  const int *pnb;        // [nb][27] the parent's same-level neighbours (nbr of the parent)
  const int *parent;     // [nb]
  const int *pofs;       // [nb] packed px | py << 10 | pz << 20
  const int *flags;      // [nb] kHasChildren | wall bits
  const long long *st_base;  // [nb] element offset of the block's stencil, -1 regular
  const long long *bt_base;  // [nb] element offset of the block's boundary term, -1 none
  const int *leaf_ids;   // [n_leaf_blocks]
  T *phi, *b, *old;      // level fields (all levels, block-contiguous)
  const T *st;           // stencil pool: per cut block (2D+1) x ncell, [diag, -x, +x, -y, +y, -z, +z]
  const unsigned char *spec;  // per cut block ncell flags at st_base/(2D+1): 1 = stencil differs from the regular one
  // cut lists: the flagged cells of each cut block, colour 0 ((x+y+z) even)
  // then colour 1; cut_list[b] = {first entry, colour-0 count, colour-1
  // count, 0}; entry e holds its cell index cut_cell[e] and its 2D+1
  // coefficients cut_coef[k * n_cut + e] (k as in st)
  const int4 *cut_list;
  const int *cut_cell;
  const T *cut_coef;
  long long n_cut;
  int wneu;              // bit w set: wall w is Neumann (ghost +phi), else Dirichlet (-phi)
  // right-hand-side slots: slot r's fields start r * rs_phi (phi) and
  // r * rs_f (b, old) elements after slot 0's; tables and stencils are shared
  int nrhs;
  long long rs_phi, rs_f;
  // independent problems: a forest holds ntree trees; (slot r, tree i) is
  // unit r * ntree + i
  int ntree;
  const int *tree_of;    // [nb] tree of each block (forests; unused when ntree == 1)
  const int *active;     // [nrhs * ntree] 0 = unit frozen (converged or empty): its CTAs return at once
  // GMG_MIXED_BF16: phi of the finest level as BF16 bits (top 16 bits of
  // the float), level-local offsets (the level's LvArgs::poff is 0 for it),
  // slot r at r * rs_h; null otherwise
  unsigned short *hphi;
  long long rs_h;
};

// Layout of a block inside a level field (phi, b, old; every level, both
// precisions): the block's ncell cells form one run in which the cells of
// colour 0 ((x + y + z) even, red) come first and those of colour 1 (black)
// after them, each colour in the natural order x fastest.  A half-sweep of
// one colour then reads the other colour's contiguous half and writes its
// own, in whole sectors.  Cell c = x + n (y + n z) of a block of side n
// (even, or n = 1) sits at cs_pos(c) = colour * ncell / 2 + c / 2: the two
// cells x = 2i and 2i + 1 of a row share c / 2 and differ in colour.
__host__ __device__ __forceinline__ int cs_pos_xyz(int x, int y, int z, int n, int ncell) {
  return ((x + y + z) & 1) * (ncell >> 1) + ((x + n * (y + n * z)) >> 1);
}
__host__ __device__ __forceinline__ int cs_pos(int c, int n, int ncell, int D) {
  const int x = c % n, y = (c / n) % n, z = D == 3 ? c / (n * n) : 0;
  return cs_pos_xyz(x, y, z, n, ncell);
}
// the inverse: natural coordinates of position p of the run
__host__ __device__ __forceinline__ void cs_xyz(int p, int n, int ncell, int D, int *x, int *y, int *z) {
  const int half = ncell >> 1;
  const int colour = (half > 0 && p >= half) ? 1 : 0;
  const int c2 = 2 * (p - colour * half);  // natural index of the row pair's even cell
  const int x0 = c2 % n;
  *y = (c2 / n) % n;
  *z = D == 3 ? c2 / (n * n) : 0;
  *x = x0 + ((colour + *y + *z) & 1);
}

template <typename T>
__host__ __device__ __forceinline__ int unit_of(const GmgView<T> &V, int r, int bid) {
  return V.ntree > 1 ? r * V.ntree + V.tree_of[bid] : r;
}

// The view of one right-hand-side slot.
template <typename T>
__host__ __device__ __forceinline__ GmgView<T> slot_view(const GmgView<T> &V, int r) {
  GmgView<T> W = V;
  W.phi = V.phi + r * V.rs_phi;
  W.b = V.b + r * V.rs_f;
  W.old = V.old + r * V.rs_f;
  W.hphi = V.hphi ? V.hphi + r * V.rs_h : nullptr;
  return W;
}

struct gmg_tree_impl;

// Plan of one launch of the cluster kernel for the bottom of the V-cycle
// (cluster_tail.cuh): levels l_lo .. l_top, each split into 2^D octants, one
// per CTA of a cluster; byte offsets of each level's arrays in shared memory,
// level index i = l_top - l.
constexpr int kClusterThreads = 512;
constexpr int kClusterMaxLevels = 12;
struct ClusterArgs {
  int l_lo, l_top;
  int children;    // level l_top holds the 2^D children of each root: child k = block first + 2^D root + k
  int pz;          // parts along z in 3D (2 or 4): clusters of 4 pz CTAs; 2D: 4 CTAs
  int ncr, nroot;  // coarsest-level unknowns per root, roots
  const double *cinv;
  int stage_rows;  // this CTA's rows of the coarse inverse are staged in shared memory
  int full_from;   // levels i >= full_from (at most 8 cells a side) are held whole by every CTA
  unsigned int off_tile[kClusterMaxLevels], off_b[kClusterMaxLevels], off_old[kClusterMaxLevels];
  unsigned int off_eidx[kClusterMaxLevels], off_cf[kClusterMaxLevels];
  unsigned int off_bd, off_rows;  // FP64 b of the coarsest level (all parts); staged inverse rows
};

// Launches the cluster kernel: nunits clusters of A.pz 4 CTAs in 3D, 4 in
// 2D (cluster_tail.cu).
template <typename T, int D>
cudaError_t launch_cycle_cluster(const GmgView<T> &V, const LvArgs *lvtab, int lmin, const ClusterArgs &A,
                                 int nunits, size_t smem, cudaStream_t s, bool pdl);
// Clusters of P CTAs with `smem` dynamic bytes each that fit on the device
// at once (0 if none does).
template <typename T, int D>
int cycle_cluster_capacity(size_t smem, int P);


}  // namespace gmg

struct gmg_tree {
  // geometry and parameters
  int D = 3, N = 8, cb[3] = {1, 1, 1}, max_level = 1, lmin = 1, lmax = 1, max_coarse = 512;
  double lo[3] = {0, 0, 0}, h1 = 1.0;
  gmg_params prm{};
  std::vector<gmg::HostBlock> blocks;  // global id order (levels ascending, Morton inside)
  std::vector<gmg::LevelInfo> levels;  // index l - lmin
  std::vector<int> nbr_h, parent_h, pofs_h, flags_h, leaf_ids_h;
  long long total_cells = 0, n_leaf_cells = 0;
  bool adaptive = false;
  int nrhs = 1;   // right-hand-side slots (fields are replicated per slot)
  int nroot = 1;  // independent root blocks (trees of a forest), each with its own coarse solve
  int ncr = 0;    // coarsest-level unknowns per root (nc = nroot * ncr)
  // forests (gmg_forest_create): ntree trees with one root each (root k =
  // tree k); blocks of tree i: tree_blocks_h[tree_boff_h[i] .. tree_boff_h[i+1]);
  // leaves are tree-major, tree i's leaf cells at tree_leaf_off_h[i]
  int ntree = 1;
  std::vector<int> tree_of_h, tree_blocks_h, tree_boff_h;
  std::vector<long long> tree_leaf_off_h;
  std::vector<double> tree_lo_h;  // [ntree][3] domain corners
  int units() const { return nrhs * ntree; }

  // walls
  int wall_type[6] = {0, 0, 0, 0, 0, 0};
  double wall_val[6] = {0, 0, 0, 0, 0, 0};
  gmg_fn wall_fn = nullptr;
  void *wall_user = nullptr;

  // set-up results (host)
  bool stencils_ready = false;
  gmg_lsf lsf_spec{};             // the level set and boundary value the set-up used (for re-meshing)
  gmg_fn phib_fn = nullptr;
  void *phib_user = nullptr;
  double phib_const = 0.0;
  long long setup_computed = 0, setup_reused = 0;  // blocks set up / taken from the previous tree
  std::vector<long long> st_base_h, bt_base_h;
  std::vector<double> stencil_h;  // concatenated per cut block: (2D+1) x ncell
  std::vector<double> bterm_h;    // concatenated per block with boundary terms: ncell
  std::vector<uint8_t> spec_h;    // per cut block ncell flags (any d < 1), parallel to stencil_h
  // cut lists (the device's copy of the flagged cells, per colour; see GmgView)
  std::vector<int> cut_list_h;     // [nb][4]
  std::vector<int> cut_cell_h;     // [n_cut]
  std::vector<double> cut_coef_h;  // [(2D+1) * n_cut]
  std::vector<int> cut_max_h;      // per level (l - lmin): largest entry count of one block
  long long n_cut = 0;
  std::vector<double> dist_h;     // per cut block: ncell x 2D distances (inspection, field evaluation)
  std::vector<double> bphib_h;    // parallel to dist_h: boundary value phi_b(x0) where d < 1
  std::vector<long long> dist_base_h;
  std::vector<double> wallv_h;    // per block on an upper domain wall: D x n^(D-1) Dirichlet face values
  std::vector<long long> wallv_base_h;
  std::vector<uint8_t> mask_h;    // per block ncell (inspection)
  std::vector<long long> mask_base_h;
  int nc = 0;                     // coarsest-level unknowns
  std::vector<double> cinv_h;     // inverses of the coarsest-level operator, per root (nroot x ncr x ncr)

  // device workspace
  bool bound = false, owns_ws = false;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  int *d_nbr = nullptr, *d_pnb = nullptr, *d_parent = nullptr, *d_pofs = nullptr, *d_flags = nullptr, *d_leaf = nullptr;
  long long *d_st_base = nullptr, *d_bt_base = nullptr, *d_cbase = nullptr;
  double *d_phi = nullptr, *d_b = nullptr, *d_old = nullptr;
  float *f_phi = nullptr, *f_b = nullptr, *f_old = nullptr;
  double *d_st = nullptr, *d_bterm = nullptr, *d_cinv = nullptr, *d_partials = nullptr, *d_red = nullptr;
  int *d_active = nullptr, *h_active = nullptr;  // unit mask (device, pinned host mirror)
  int *d_tree_of = nullptr, *d_tree_blocks = nullptr, *d_tree_boff = nullptr;
  // field evaluation (gmg_efield): per-cell flags, distances and boundary
  // values of cut blocks, upper-wall values, leaf position of each block
  unsigned char *d_cellflag = nullptr;
  double *d_dist = nullptr, *d_bphib = nullptr, *d_wallv = nullptr;
  long long *d_dist_base = nullptr, *d_wallv_base = nullptr, *d_mask_base = nullptr;
  int *d_leafpos = nullptr;
  float *f_st = nullptr;
  unsigned char *d_spec = nullptr;
  int4 *d_cut_list = nullptr;
  int *d_cut_cell = nullptr;
  double *d_cut_coef = nullptr;
  float *f_cut_coef = nullptr;
  gmg::LvArgs *d_lvtab = nullptr;  // per-level descriptors (phi in the first buffer)
  double *h_red = nullptr;  // pinned host mirror of d_red ([units][4])
  long long launches = 0;

  std::vector<char> level_has_leaves;  // index l - lmin

  // CUDA graphs of the solve phases (captured on first use)
  struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
  };
  enum {
    kGraphResid64 = 0,
    kGraphResidMixed,
    kGraphCycle64,
    kGraphCycleMixed,
    kGraphVcycle64,
    kGraphFmg64,
    kGraphCycleBf16,
    kGraphSlots
  };
  GraphSlot graphs[kGraphSlots];
  bool use_graphs = true;
  bool use_coop = true;       // coarse levels in one cooperative launch
  bool use_fused = false;     // temporally blocked FP32 sweeps on uniform levels
  int cta_threads = 0;        // threads per CTA of the block kernels (0: by block size)
  int inner_cycles = 1;       // FP32 V-cycles per defect-correction step of the mixed path
  bool bf16_top = false;      // while a GMG_MIXED_BF16 step is enqueued: the finest level's FP32 state is BF16
  int slots_per_cta = 1;      // right-hand-side slots of a block per CTA in the half-sweeps (1, 2, 4)
  bool fmg_steps = false;     // solve steps are FMG cycles instead of V-cycles
  bool use_pdl = true;        // per-level kernels with programmatic dependent launch
  bool use_level_legs = false; // a level whose CTAs fit at once runs each leg as one cooperative launch
  bool setup_on_device = true;  // boundary detection of built-in level sets on the device when one is present
  bool setup_device = false;    // the last set-up ran its boundary detection on the device
  int cluster_mode = 1;       // bottom of the cycle on a thread-block cluster: 0 off, 1 when all units fit at once, 2 whenever eligible
  int cluster_parts = 0;      // CTAs of the cluster in 3D: 8, 16, or 0 for 16 when the tree and the device allow it
  std::vector<char> level_complete;  // every block has all 26 neighbours on its level (or walls)
  int coop_split = 0;         // highest level run inside that launch
  int coop_max_blocks = gmg::kCoopMaxBlocks;  // levels with at most this many blocks join it
  std::vector<int> sweeps_down, sweeps_up;  // per level (index l - lmin); empty: the parameters'
  int n_down_at(int l) const { return sweeps_down.empty() ? prm.n_down : sweeps_down[l - lmin]; }
  int n_up_at(int l) const { return sweeps_up.empty() ? prm.n_up : sweeps_up[l - lmin]; }
  long long spin_limit = 1LL << 24;
  gmg::GridBar *d_bar = nullptr;
  cudaStream_t cap_stream = nullptr;
  bool step_pending = false;  // gmg_iterate_begin enqueued a step that gmg_iterate_end has not read
  cudaStream_t step_stream = nullptr;

  // kernel timing (gmg_profile_enable)
  struct ProfRec {
    cudaEvent_t a, b;
    int kind, prec, level;
  };
  bool prof_on = false;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> prof_pool;
  size_t prof_used = 0;

  gmg::LevelInfo &lev(int l) { return levels[l - lmin]; }
  int leaf_ncell() const { return levels.back().ncell; }  // cells of a leaf block (every leaf is on a level >= 1)
  const gmg::LevelInfo &lev(int l) const { return levels[l - lmin]; }
};

namespace gmg {
// Threads per CTA of the smoothing, residual, restriction and FAS kernels on
// level l: small blocks take smaller CTAs, so that more of them (and more of
// their tile loads) are resident per SM.
inline int cta_threads(const gmg_tree *t, int l) {
  if (t->cta_threads) return t->cta_threads;
  return t->lev(l).ncell <= 512 ? 64 : 256;
}

// Threads per CTA of the FP64 residual-norm kernel: as the level kernels
// (at most 256, so that four CTAs of 16^3 blocks fit an SM).
inline int resnorm_threads(const gmg_tree *t, int l) { return cta_threads(t, l); }

void set_error(const std::string &msg);
int build_tree(gmg_tree *T, const gmg_domain *dom);
int host_setup(gmg_tree *T, const gmg_lsf *lsf, gmg_fn phib, void *phib_user, double phib_const,
               const gmg_tree *reuse = nullptr);
void build_cut_lists(gmg_tree *T);
struct LsfSpec;
// Boundary detection on the device for a built-in level set (setup_dev.cu):
// mask[cell] for every cell in block order (bit 0 Eq. (boundary-mask), bit
// 1 centre inside), the masked cells (index in that order, ascending) and
// their 2D relative distances.  Bit for bit the host set-up's values.
// With `terms`, also the stencils and right-hand-side terms of the cut
// blocks (blocks with a distance below 1) for a constant boundary value
// phib and constant wall values, dense per cut block in block order: the
// host's block_terms bit for bit.
struct DeviceTerms {
  std::vector<int> cut_ids;          // cut blocks, ascending
  std::vector<long long> cell_off;   // [ncut + 1] first cell of each in the arrays below
  std::vector<double> dd, st, bt, pb;  // distances (2D), stencil (coefficient-major per block), terms, phi_b at roots (2D)
};
bool device_setup_available();
int device_boundary_detection(const gmg_tree *T, const LsfSpec &spec, std::vector<uint8_t> &mask,
                              std::vector<long long> &masked_cells, std::vector<double> &dist, DeviceTerms *terms,
                              double phib);
}  // namespace gmg
