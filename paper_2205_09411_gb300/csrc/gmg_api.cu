// C ABI of the GB300 octree multigrid library (include/gmg.h): workspace
// layout in HBM, the V-cycle schedule (Sec. 2.2) and the FP64 / mixed
// solve loops, on top of the level kernels of kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "gmg_internal.h"
#include "coarse_cycle.cuh"
#include "efield.cuh"
#include "csweep.cuh"
#include "fused_sweeps.cuh"
#include "kernels.cuh"

namespace gmg {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

#define CUDA_TRY(expr)                                                                       \
  do {                                                                                       \
    cudaError_t _e = (expr);                                                                 \
    if (_e != cudaSuccess) {                                                                 \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                         \
      return GMG_ERR_CUDA;                                                                   \
    }                                                                                        \
  } while (0)

__global__ void __launch_bounds__(kResThreads) k_reduce_partials(const double *partials, int nb, const int *tree_blocks,
                                                                 const int *tree_boff, int ntree, double *out,
                                                                 const GridBar *bar) {
  pdl_start();
  // unit blockIdx.x = (slot r, tree i): the blocks of tree i in slot r
  const int r = blockIdx.x / ntree, tr = blockIdx.x % ntree;
  partials += (size_t)r * nb * 3;
  out += (size_t)blockIdx.x * 4;
  const int b0 = tree_boff[tr], b1 = tree_boff[tr + 1];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int k = b0 + threadIdx.x; k < b1; k += blockDim.x) {
    const size_t i = (size_t)tree_blocks[k];
    a += partials[i * 3];
    b = fmax(b, partials[i * 3 + 1]);
    c += partials[i * 3 + 2];
  }
  block_reduce3(a, b, c, out);  // fixed order: warp shuffles, then the warps in order
  if (threadIdx.x == 0) out[3] = bar ? (double)bar->err : 0.0;  // a timed-out barrier of the coarse cycle
}

// Leaf-cell kernels over the slots r0 .. r0 + nr - 1: a CTA takes leaf
// blocks lb = blockIdx.x, +gridDim.x, ...; element k of the leaf-ordered
// array io (nr x nleaf cells) is cell (k % nleaf) of slot r0 + k / nleaf;
// field arrays of slot r start at r * rs.

// b <- g - boundary terms on leaf cells (g in leaf-cell order)
__global__ void k_leaf_rhs(const int *__restrict__ leaf_ids, const long long *__restrict__ cbase,
                           const long long *__restrict__ bt_base, const double *__restrict__ bterm,
                           const double *__restrict__ g, double *__restrict__ b, int nlb, int ncell, long long rs,
                           int r0, int nr, int n, int D) {
  const long long nleaf = (long long)nlb * ncell;
  for (int lb = blockIdx.x; lb < nlb; lb += gridDim.x) {
    const int id = leaf_ids[lb];
    const long long base = cbase[id], bb = bt_base[id];
    for (int r = 0; r < nr; r++)
      for (int c = threadIdx.x; c < ncell; c += blockDim.x)
        b[(r0 + r) * rs + base + cs_pos(c, n, ncell, D)] = g[r * nleaf + (long long)lb * ncell + c] - (bb >= 0 ? bterm[bb + c] : 0.0);
  }
}

// leaf gather (dir 0: field -> io) / scatter (dir 1: io -> field)
__global__ void k_leaf_copy(const int *__restrict__ leaf_ids, const long long *__restrict__ cbase, double *field,
                            double *io, int nlb, int ncell, long long rs, int r0, int nr, int dir, int n, int D) {
  const long long nleaf = (long long)nlb * ncell;
  for (int lb = blockIdx.x; lb < nlb; lb += gridDim.x) {
    const long long base = cbase[leaf_ids[lb]];
    for (int r = 0; r < nr; r++)
      for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const long long f = (r0 + r) * rs + base + cs_pos(c, n, ncell, D), k = r * nleaf + (long long)lb * ncell + c;
        if (dir == 0)
          io[k] = field[f];
        else
          field[f] = io[k];
      }
  }
}

// phi64 += e32 on leaf cells of the active units (mixed path: solution
// accumulation in FP64)
// With eh (GMG_MIXED_BF16), e of the blocks from h_first on (the finest
// level) is read from its BF16 run: slot r at r * rs_h, level-local offset
// cbase - h_off.
__global__ void k_leaf_accumulate(const int *__restrict__ leaf_ids, const long long *__restrict__ cbase,
                                  double *__restrict__ phi, const float *__restrict__ e, int nlb, int ncell,
                                  long long rs, int nr, const int *__restrict__ active, const int *__restrict__ tree_of,
                                  int ntree, const unsigned short *__restrict__ eh, int h_first, long long h_off,
                                  long long rs_h) {
  pdl_start();
  for (int lb = blockIdx.x; lb < nlb; lb += gridDim.x) {
    const int id = leaf_ids[lb];
    const long long base = cbase[id];
    const int tr = ntree > 1 ? tree_of[id] : 0;
    for (int r = 0; r < nr; r++) {
      if (!active[r * ntree + tr]) continue;
      if (eh && id >= h_first) {
        const long long o = r * rs + base;
        const unsigned short *eb = eh + r * rs_h + (base - h_off);
        if ((ncell & 3) == 0) {  // four cells a thread: one 8-byte load of e, two double2 of phi
          for (int c = 4 * threadIdx.x; c < ncell; c += 4 * blockDim.x) {
            const uint2 d = __ldcs(reinterpret_cast<const uint2 *>(eb + c));
            double2 *p = reinterpret_cast<double2 *>(phi + o + c);
            double2 u = p[0], w = p[1];
            u.x += f32_to_f64(ld_val((bf16s)(d.x & 0xffffu)));
            u.y += f32_to_f64(ld_val((bf16s)(d.x >> 16)));
            w.x += f32_to_f64(ld_val((bf16s)(d.y & 0xffffu)));
            w.y += f32_to_f64(ld_val((bf16s)(d.y >> 16)));
            p[0] = u;
            p[1] = w;
          }
        } else {
          for (int c = threadIdx.x; c < ncell; c += blockDim.x) phi[o + c] += f32_to_f64(ld_val((bf16s)eb[c]));
        }
        continue;
      }
      const long long o = r * rs + base;
      if (((o | ncell) & 3) == 0) {  // four cells a thread: one float4 of e, two double2 of phi
        for (int c = 4 * threadIdx.x; c < ncell; c += 4 * blockDim.x) {
          const float4 d = __ldcs(reinterpret_cast<const float4 *>(e + o + c));
          double2 *p = reinterpret_cast<double2 *>(phi + o + c);
          double2 u = p[0], w = p[1];
          u.x += f32_to_f64(d.x);
          u.y += f32_to_f64(d.y);
          w.x += f32_to_f64(d.z);
          w.y += f32_to_f64(d.w);
          p[0] = u;
          p[1] = w;
        }
      } else {
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) phi[o + c] += f32_to_f64(e[o + c]);
      }
    }
  }
}

// Holds the stream for about `us` microseconds (bounded by construction):
// while kernel timing is on, it lets the host enqueue a whole phase so that
// the events around each kernel measure the kernel, not the host.
__global__ void k_delay(int us) {
  for (int i = 0; i < us; i++) __nanosleep(1000);
}

// Counts where the integer-operation conversions differ bit for bit from
// the hardware's: bad[0] double -> float (round to nearest even), bad[1]
// float -> double.
__global__ void k_selftest_conv(const double *__restrict__ x, const float *__restrict__ f, long long n,
                                unsigned long long *bad) {
  unsigned long long b0 = 0, b1 = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    b0 += __float_as_uint(f64_to_f32_rn(x[k])) != __float_as_uint(__double2float_rn(x[k]));
    b1 += __double_as_longlong(f32_to_f64(f[k])) != __double_as_longlong((double)f[k]);
  }
  if (b0) atomicAdd(bad, b0);
  if (b1) atomicAdd(bad + 1, b1);
}

__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ b, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    b[k] = (float)a[k];
}

}  // namespace gmg

using namespace gmg;

namespace {

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }
int n_leaf_blocks(const gmg_tree *t) { return (int)t->leaf_ids_h.size(); }
int leaf_grid(const gmg_tree *t) { return std::max(1, std::min(n_leaf_blocks(t), 152 * 16)); }

cudaEvent_t prof_event(gmg_tree *t) {
  if (t->prof_used == t->prof_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    t->prof_pool.push_back(e);
  }
  return t->prof_pool[t->prof_used++];
}

// Enqueue one kernel: counts it and, while profiling, brackets it with events.
template <typename F>
void launch(gmg_tree *t, cudaStream_t s, int kind, int prec, int level, F &&f) {
  if (t->prof_on) {
    gmg_tree::ProfRec r;
    r.a = prof_event(t);
    r.b = prof_event(t);
    r.kind = kind;
    r.prec = prec;
    r.level = level;
    cudaEventRecord(r.a, s);
    f();
    cudaEventRecord(r.b, s);
    t->prof.push_back(r);
  } else {
    f();
  }
  t->launches += 1;
}

// Launch of a solve-step kernel: with programmatic dependent launch (the
// kernel starts with pdl_start) unless the option is off or kernel timing
// is on (events between kernels).
template <typename... KArgs, typename... Args>
void klaunch(const gmg_tree *t, dim3 grid, dim3 block, size_t smem, cudaStream_t s, void (*k)(KArgs...),
             Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = (t->use_pdl && !t->prof_on) ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, args...);
}

template <typename T>
constexpr int prec_of() {
  return sizeof(T) == 8 ? 0 : 1;
}

LvArgs lv(const gmg_tree *T, int l) {
  const LevelInfo &L = T->lev(l);
  LvArgs a;
  a.first = L.first;
  a.count = L.count;
  a.n = L.n;
  a.ncell = L.ncell;
  a.off = L.off;
  a.h = L.h;
  a.poff = L.off;
  a.nd = T->n_down_at(l);
  a.nu = T->n_up_at(l);
  a.h2 = L.h * L.h;
  a.ih2 = 1.0 / (L.h * L.h);
  return a;
}

// GMG_MIXED_BF16: the finest level's phi of the FP32 correction is kept as
// BF16 in that level's part of the second FP32 phi buffer (which only the
// fused sweeps use, and not on this level): slot r's BF16 run starts at
// float offset r * total_cells + (level offset) of that buffer, so it lies
// inside the level's own part of the slot.  No extra memory.
unsigned short *bf16_phi(gmg_tree *t) {
  return reinterpret_cast<unsigned short *>(t->f_phi + (size_t)t->nrhs * t->total_cells + t->lev(t->lmax).off);
}

// Whether the finest level can hold BF16 state: it runs in the per-level
// kernels (above the cooperative / cluster levels), its block side has
// compiled kernels, and its runs start on 16-byte boundaries.  Otherwise
// GMG_MIXED_BF16 runs as GMG_MIXED.
bool bf16_eligible(const gmg_tree *t) {
  const int ls = t->use_coop ? t->coop_split : t->lmin;
  if (t->lmax <= ls || t->lmax <= t->lmin) return false;
  const int n = t->lev(t->lmax).n;
  const bool nt = t->D == 3 ? (n == 4 || n == 8 || n == 16) : (n == 8 || n == 16 || n == 32);
  return nt && t->total_cells % 4 == 0 && t->lev(t->lmax).off % 4 == 0;
}

template <typename T>
GmgView<T> view(gmg_tree *t);

template <>
GmgView<double> view<double>(gmg_tree *t) {
  GmgView<double> v;
  v.cut_list = t->d_cut_list;
  v.cut_cell = t->d_cut_cell;
  v.cut_coef = t->d_cut_coef;
  v.n_cut = t->n_cut;
  v.nbr = t->d_nbr;
  v.pnb = t->d_pnb;
  v.parent = t->d_parent;
  v.pofs = t->d_pofs;
  v.flags = t->d_flags;
  v.st_base = t->d_st_base;
  v.bt_base = t->d_bt_base;
  v.leaf_ids = t->d_leaf;
  v.phi = t->d_phi;
  v.b = t->d_b;
  v.old = t->d_old;
  v.st = t->d_st;
  v.spec = t->d_spec;
  v.wneu = 0;
  for (int w = 0; w < 6; w++) v.wneu |= (t->wall_type[w] == GMG_WALL_NEUMANN ? 1 : 0) << w;
  v.nrhs = t->nrhs;
  v.rs_phi = t->total_cells;
  v.rs_f = t->total_cells;
  v.ntree = t->ntree;
  v.tree_of = t->d_tree_of;
  v.active = t->d_active;
  v.hphi = nullptr;
  v.rs_h = 0;
  return v;
}

template <>
GmgView<float> view<float>(gmg_tree *t) {
  GmgView<float> v;
  v.cut_list = t->d_cut_list;
  v.cut_cell = t->d_cut_cell;
  v.cut_coef = t->f_cut_coef;
  v.n_cut = t->n_cut;
  v.nbr = t->d_nbr;
  v.pnb = t->d_pnb;
  v.parent = t->d_parent;
  v.pofs = t->d_pofs;
  v.flags = t->d_flags;
  v.st_base = t->d_st_base;
  v.bt_base = t->d_bt_base;
  v.leaf_ids = t->d_leaf;
  v.phi = t->f_phi;
  v.b = t->f_b;
  v.old = t->f_old;
  v.st = t->f_st;
  v.spec = t->d_spec;
  v.wneu = 0;
  for (int w = 0; w < 6; w++) v.wneu |= (t->wall_type[w] == GMG_WALL_NEUMANN ? 1 : 0) << w;
  v.nrhs = t->nrhs;
  v.rs_phi = t->total_cells;
  v.rs_f = t->total_cells;
  v.ntree = t->ntree;
  v.tree_of = t->d_tree_of;
  v.active = t->d_active;
  v.hphi = t->bf16_top ? bf16_phi(t) : nullptr;
  v.rs_h = 2 * t->total_cells;
  return v;
}

template <int V>
using IC = std::integral_constant<int, V>;

// Calls f(IC<NT>) with NT the compile-time block side for n (0 = runtime).
template <int D, typename F>
void with_nt(int n, F &&f) {
  if constexpr (D == 3) {
    switch (n) {
      case 4: f(IC<4>{}); return;
      case 8: f(IC<8>{}); return;
      case 16: f(IC<16>{}); return;
      default: f(IC<0>{}); return;
    }
  } else {
    switch (n) {
      case 8: f(IC<8>{}); return;
      case 16: f(IC<16>{}); return;
      case 32: f(IC<32>{}); return;
      default: f(IC<0>{}); return;
    }
  }
}

// Every kernel of the library asks for the same shared-memory carveout, so
// that consecutive kernels never make the SMs reconfigure L1/shared memory.
template <typename K>
void kernel_attrs(K *k, bool big_smem) {
  if (big_smem) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

template <typename T, int D, int NT>
void set_smem_limits_nt() {
  kernel_attrs(k_smooth<T, D, NT>, true);
  kernel_attrs(k_resid_restrict<T, D, NT>, true);
  kernel_attrs(k_fas<T, D, NT>, true);
  kernel_attrs(k_prolong<T, D, NT, 64>, true);
  if constexpr (NT != 0) {
    kernel_attrs(k_smooth_cs<T, D, NT, 1>, true);
    kernel_attrs(k_smooth_cs<T, D, NT, 2>, true);
    kernel_attrs(k_smooth_cs<T, D, NT, 4>, true);
  }
  kernel_attrs(k_prolong<T, D, NT, 128>, true);
  kernel_attrs(k_prolong<T, D, NT, 256>, true);
  kernel_attrs(k_resnorm<T, D, NT>, true);
  kernel_attrs(k_restrict_phi<T, D, NT>, false);
  if constexpr (NT != 0) kernel_attrs(k_level_leg<T, D, NT>, true);
}

template <typename T, int D>
void set_smem_limits() {
  for (int n : {4, 8, 16, 32, 2}) with_nt<D>(n, [&](auto nt) { set_smem_limits_nt<T, D, decltype(nt)::value>(); });
}

// the BF16 variants of the finest level's kernels (FP32 arithmetic)
template <int D, int NT>
void bf16_attrs() {
  if constexpr (NT != 0) {
    kernel_attrs(k_smooth_cs<float, D, NT, 1, true>, true);
    kernel_attrs(k_smooth_cs<float, D, NT, 2, true>, true);
    kernel_attrs(k_smooth_cs<float, D, NT, 4, true>, true);
    kernel_attrs(k_resid_restrict<float, D, NT, true>, true);
    kernel_attrs(k_prolong<float, D, NT, 64, true>, true);
    kernel_attrs(k_prolong<float, D, NT, 128, true>, true);
    kernel_attrs(k_prolong<float, D, NT, 256, true>, true);
    kernel_attrs(k_restrict_phi<float, D, NT, true>, false);
  }
}

template <int D, int NT>
void fused_attrs() {
  if constexpr (NT != 0) {
    kernel_attrs(k_smooth_tb<float, D, NT, 2>, true);
    kernel_attrs(k_smooth_tb<float, D, NT, 4>, true);
  }
}

void set_all_smem_limits() {
  static bool done = false;
  if (done) return;
  for (int n : {8, 16, 32}) {
    with_nt<2>(n, [&](auto nt) { fused_attrs<2, decltype(nt)::value>(); });
    with_nt<3>(n, [&](auto nt) { fused_attrs<3, decltype(nt)::value>(); });
  }
  for (int n : {4, 8, 16, 32}) {
    with_nt<2>(n, [&](auto nt) { bf16_attrs<2, decltype(nt)::value>(); });
    with_nt<3>(n, [&](auto nt) { bf16_attrs<3, decltype(nt)::value>(); });
  }
  set_smem_limits<double, 2>();
  set_smem_limits<double, 3>();
  set_smem_limits<float, 2>();
  set_smem_limits<float, 3>();
  kernel_attrs(k_coarse<double>, false);
  kernel_attrs(k_coarse<float>, false);
  kernel_attrs(k_reduce_partials, false);
  kernel_attrs(k_leaf_rhs, false);
  kernel_attrs(k_leaf_copy, false);
  kernel_attrs(k_leaf_accumulate, false);
  kernel_attrs(k_to_float, false);
  for (int n : {4, 8, 16, 32, 2}) {
    with_nt<3>(n, [&](auto nt) { kernel_attrs(k_efield<3, decltype(nt)::value>, true); });
    with_nt<2>(n, [&](auto nt) { kernel_attrs(k_efield<2, decltype(nt)::value>, true); });
  }
  kernel_attrs(k_delay, false);
  done = true;
}

// Half-sweep of a level on the colour-split layout (csweep.cuh): one CTA
// per (block, slot), or per (block, group of slots_per_cta slots) when the
// tree has several slots and the group's tiles fit in shared memory; blocks
// of a side without a compiled kernel take the tile-based smooth_block.
// bf: the level's phi is BF16 (GMG_MIXED_BF16's finest level; FP32 only).
template <typename T, int D, int NT>
void launch_smooth(const gmg_tree *t, const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int c, int threads,
                   size_t sm, cudaStream_t s, bool bf = false) {
  if constexpr (NT != 0) {
    int sg = t->nrhs > 1 ? t->slots_per_cta : 1;
    if constexpr (std::is_same<T, float>::value) {
      if (bf) {
        while (sg > 1 && cs_smem_bytes<T, D, NT, true>(sg) > 200 * 1024) sg /= 2;
        const int grid = L.count * ((t->nrhs + sg - 1) / sg);
        const size_t sms = cs_smem_bytes<T, D, NT, true>(sg);
        if (sg == 4)
          klaunch(t, grid, threads, sms, s, k_smooth_cs<T, D, NT, 4, true>, V, L, Lp, c);
        else if (sg == 2)
          klaunch(t, grid, threads, sms, s, k_smooth_cs<T, D, NT, 2, true>, V, L, Lp, c);
        else
          klaunch(t, grid, threads, sms, s, k_smooth_cs<T, D, NT, 1, true>, V, L, Lp, c);
        return;
      }
    }
    while (sg > 1 && cs_smem_bytes<T, D, NT>(sg) > 200 * 1024) sg /= 2;
    const int grid = L.count * ((t->nrhs + sg - 1) / sg);
    const size_t sms = cs_smem_bytes<T, D, NT>(sg);
    if (sg == 4)
      klaunch(t, grid, threads, sms, s, k_smooth_cs<T, D, NT, 4>, V, L, Lp, c);
    else if (sg == 2)
      klaunch(t, grid, threads, sms, s, k_smooth_cs<T, D, NT, 2>, V, L, Lp, c);
    else
      klaunch(t, grid, threads, sms, s, k_smooth_cs<T, D, NT, 1>, V, L, Lp, c);
    return;
  }
  klaunch(t, L.count * t->nrhs, threads, sm, s, k_smooth<T, D, NT>, V, L, Lp, c);
}

// k_prolong with the CTA size of the level's block kernels
template <typename T, int D, int NT>
void launch_prolong(const gmg_tree *t, int threads, int grid, size_t sm, cudaStream_t s, const GmgView<T> &V,
                    const LvArgs &L, const LvArgs &Lp, bool bf = false) {
  if constexpr (std::is_same<T, float>::value && NT != 0) {
    if (bf) {
      if (threads == 64)
        klaunch(t, grid, 64, sm, s, k_prolong<T, D, NT, 64, true>, V, L, Lp);
      else if (threads == 128)
        klaunch(t, grid, 128, sm, s, k_prolong<T, D, NT, 128, true>, V, L, Lp);
      else
        klaunch(t, grid, 256, sm, s, k_prolong<T, D, NT, 256, true>, V, L, Lp);
      return;
    }
  }
  if (threads == 64)
    klaunch(t, grid, 64, sm, s, k_prolong<T, D, NT, 64>, V, L, Lp);
  else if (threads == 128)
    klaunch(t, grid, 128, sm, s, k_prolong<T, D, NT, 128>, V, L, Lp);
  else
    klaunch(t, grid, 256, sm, s, k_prolong<T, D, NT, 256>, V, L, Lp);
}

template <typename T, int D, int NT>
void launch_resid_restrict(const gmg_tree *t, int grid, int threads, size_t sm, cudaStream_t s, const GmgView<T> &V,
                           const LvArgs &L, const LvArgs &Lp, bool bf = false) {
  if constexpr (std::is_same<T, float>::value && NT != 0) {
    if (bf) {
      klaunch(t, grid, threads, sm, s, k_resid_restrict<T, D, NT, true>, V, L, Lp);
      return;
    }
  }
  klaunch(t, grid, threads, sm, s, k_resid_restrict<T, D, NT>, V, L, Lp);
}

// Whether level l's FP32 phi is BF16 in the step being enqueued.
template <typename T>
bool bf16_level(const gmg_tree *t, int l) {
  return std::is_same<T, float>::value && t->bf16_top && l == t->lmax;
}

template <typename T>
size_t tile_bytes(const gmg_tree *t, int l) {
  return level_smem_bytes<T>(t->D, t->lev(l).n);
}

// A level's down leg (mode 0) or up leg (mode 1) in one cooperative launch
// (k_level_leg) when the level has a compiled block side, 256-thread CTAs,
// and all its (block, slot) CTAs fit on the GPU at once; *smem gets the
// launch's shared memory.
template <typename T, int D, int NT>
bool level_leg_ok(const gmg_tree *t, int l, size_t *smem) {
  if constexpr (NT == 0) {
    return false;
  } else {
    if (!t->use_level_legs || t->lev(l).n != NT || cta_threads(t, l) != kThreads) return false;
    const int hm = NT / 2 + 2;
    const size_t psm = sizeof(T) * (size_t)(D == 3 ? hm * hm * hm : hm * hm);
    const size_t sm = std::max(std::max(cs_smem_bytes<T, D, NT>(1), tile_bytes<T>(t, l)), psm);
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level_leg<T, D, NT>, kThreads, sm) != cudaSuccess)
      return false;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *smem = sm;
    return per_sm > 0 && (long long)t->lev(l).count * t->nrhs <= (long long)per_sm * sms;
  }
}

template <typename T, int D, int NT>
void launch_level_leg(gmg_tree *t, cudaStream_t s, const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int l,
                      int mode, size_t sm) {
  if constexpr (NT != 0) {
    cudaMemsetAsync(&t->d_bar->count, 0, sizeof(unsigned int), s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(L.count * t->nrhs));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    GridBar *bar = t->d_bar;
    const long long spin = t->spin_limit;
    launch(t, s, 11 + mode, prec_of<T>(), l,
           [&] { cudaLaunchKernelEx(&cfg, k_level_leg<T, D, NT>, V, L, Lp, mode, bar, spin); });
  }
}

// The cooperative launch of the coarse part of a V-cycle (coarse_cycle.cuh)
// on levels lmin .. ls.  mode 0: the whole coarse cycle, with the
// single-block levels at the bottom on one CTA per (root, slot) when they fit
// (the tail); mode 1: the down leg to the FAS right-hand side of level
// l_stop; mode 2: the up leg from level l_stop + 1 (the cluster kernel did
// the levels up to l_stop in between).
template <typename T, int D>
int coop_launch(gmg_tree *t, cudaStream_t s, int ls, int mode, int l_stop) {
  GmgView<T> V = view<T>(t);
  int l_one = t->lmin - 1;
  size_t tail_bytes = 0;
  int cinv_off = -1;
  if (mode != 0) {
    l_one = l_stop;
  } else {
    // the single-block levels at the bottom run on one CTA when the coarse
    // solve is small enough for one CTA
    if (t->ncr <= 256 && (t->nroot > 1 || t->cb[0] * t->cb[1] * t->cb[2] == 1))
      for (int l = t->lmin; l <= ls && t->lev(l).count == t->nroot; l++) {
        const int n = t->lev(l).n;
        const size_t add = tail_level_bytes<T, D>(n, t->cut_max_h[l - t->lmin]);
        if (tail_bytes + add > 160 * 1024 || l - t->lmin >= 11) break;
        tail_bytes += add;
        l_one = l;
      }
    // the tail's coarse inverse in shared memory when it fits beside the levels
    const size_t cinv_bytes = sizeof(double) * ((size_t)t->ncr * t->ncr + t->ncr);  // inverse and b in FP64
    if (l_one >= t->lmin && tail_bytes + cinv_bytes <= 192 * 1024) {
      cinv_off = (int)tail_bytes;
      tail_bytes += cinv_bytes;
    }
  }
  CycleArgs A{t->lmin, ls, t->ncr, t->nroot, t->d_cinv, t->d_bar, t->spin_limit, l_one, cinv_off, mode};
  size_t sm = 0;
  int maxb = (mode == 0 && l_one >= t->lmin) ? t->nroot : 1;
  for (int l = t->lmin; l <= ls; l++) {
    if (l <= l_one) continue;  // held in shared memory by the tail, or done by the cluster kernel
    const int hm = t->lev(l).n / 2 + 2;
    sm = std::max(sm, tile_bytes<T>(t, l));
    sm = std::max(sm, sizeof(T) * (size_t)(D == 3 ? hm * hm * hm : hm * hm));
    maxb = std::max(maxb, t->lev(l).count);
  }
  maxb *= t->nrhs;  // work items: (block, slot) pairs
  sm = std::max(sm, tail_bytes);
  int rc = GMG_OK;
  with_nt<D>(t->N, [&](auto nt) {
    constexpr int NT = decltype(nt)::value;
    auto kern = k_cycle_coop<T, D, NT>;
    int per_sm = 0;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCoopThreads, sm);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int G = std::max(1, std::min(maxb, per_sm * sms));
    if (per_sm < 1) {
      set_error("the coarse-cycle kernel cannot be made resident");
      rc = GMG_ERR_CUDA;
      return;
    }
    cudaMemsetAsync(&t->d_bar->count, 0, sizeof(unsigned int), s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kCoopThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const LvArgs *tab = t->d_lvtab;
    const int nlev = (int)t->levels.size();
    const int lmin = t->lmin;
    launch(t, s, 3, prec_of<T>(), t->lmin, [&] { cudaLaunchKernelEx(&cfg, kern, V, tab, nlev, lmin, A); });
  });
  if (rc) return rc;
  CUDA_TRY(cudaGetLastError());
  return GMG_OK;
}

// Plan of the cluster kernel (cluster_tail.cuh) for the bottom of a V-cycle
// whose coarse part covers levels lmin .. ls: the single-block levels from
// lmin up, and above them the level of the roots' 2^D children when it is
// complete.  A cluster of P CTAs splits each level of more than 8 cells a
// side into parts of N/2 x N/2 (x N/pz in 3D) cells, whose sides must be
// even; the parts' arrays must fit one CTA's shared memory and, with
// cluster_mode 1, all units' clusters must be resident at once.  In 3D,
// clusters of 16 CTAs (pz = 4) are tried first unless cluster_parts asks
// for 8.  Returns false when the tree does not qualify (the cooperative
// kernel's own tail then runs).
template <typename T, int D>
bool plan_cluster_pz(gmg_tree *t, int ls, int pz, ClusterArgs *A, size_t *smem) {
  const int P = D == 3 ? 4 * pz : 4;
  int l_single = t->lmin - 1;
  for (int l = t->lmin; l <= ls && t->lev(l).count == t->nroot; l++) l_single = l;
  if (l_single < t->lmin) return false;
  // split levels (more than 8 cells a side) need parts of even side; the
  // levels of at most 8 a side are held whole by every CTA and need an even side
  const int split_mod = D == 3 && pz == 4 ? 8 : 4;
  for (int l = t->lmin; l <= l_single; l++)
    if (t->lev(l).n % (t->lev(l).n > 8 ? split_mod : 2)) return false;
  bool children = false;
  constexpr int NCH = 1 << D;
  if (l_single + 1 <= ls && t->lev(l_single + 1).count == t->nroot * NCH) {
    children = true;
    const LevelInfo &R = t->lev(l_single), &Cl = t->lev(l_single + 1);
    for (int r = 0; r < t->nroot && children; r++)
      for (int k = 0; k < NCH && children; k++) {
        const HostBlock &b = t->blocks[Cl.first + NCH * r + k];
        const HostBlock &p = t->blocks[R.first + r];
        if (b.parent != R.first + r) children = false;
        for (int d = 0; d < D; d++)
          if (b.ix[d] - 2 * p.ix[d] != ((k >> d) & 1)) children = false;
      }
    // the children level's parts lie within one child each
    if (children && (2 * Cl.n) % split_mod) children = false;
  }
  const size_t limit = 224 * 1024;
  for (int attempt = 0; attempt < 2; attempt++) {
    const int l_top = children ? l_single + 1 : l_single;
    if (l_top - t->lmin + 1 > kClusterMaxLevels) return false;
    ClusterArgs a{};
    a.l_lo = t->lmin;
    a.l_top = l_top;
    a.children = children ? 1 : 0;
    a.pz = D == 3 ? pz : 1;
    a.ncr = t->ncr;
    a.nroot = t->nroot;
    a.cinv = t->d_cinv;
    size_t o = 0;
    auto take = [&](size_t bytes) {
      const size_t at = o;
      o = (o + bytes + 15) / 16 * 16;
      return (unsigned int)at;
    };
    bool ok = true;
    int nlo = 0;
    a.full_from = l_top - t->lmin + 1;
    for (int l = l_top; l >= t->lmin; l--) {
      const int i = l_top - l;
      const int N = (children && l == l_top) ? 2 * t->lev(l).n : t->lev(l).n;
      const bool full = i > 0 && N <= 8;
      if (full && a.full_from > i) a.full_from = i;
      if (!full && i > a.full_from) ok = false;  // full levels form the bottom of the range
      if (i == 0 && N <= 8) ok = false;          // the top level is split
      const int m0 = full ? N : N / 2, m2 = D == 3 ? (full ? N : N / a.pz) : 1;
      const int nc = m0 * m0 * m2;
      const size_t ring = (size_t)(m0 + 2) * (m0 + 2) * (D == 3 ? m2 + 2 : 1);
      const int cap = t->cut_max_h[l - t->lmin];
      if (cap > 65534) ok = false;
      a.off_tile[i] = take(sizeof(T) * ring);
      a.off_b[i] = take(sizeof(T) * (size_t)nc);
      a.off_old[i] = take(sizeof(T) * (size_t)nc);
      a.off_eidx[i] = take(2 * (size_t)nc);
      a.off_cf[i] = take(sizeof(T) * (size_t)cap * (2 * D + 1));
      nlo = full ? (t->ncr + P - 1) / P : nc;  // rows of the coarse solve per CTA
    }
    a.off_bd = take(sizeof(double) * (size_t)t->ncr);
    const size_t rows = sizeof(double) * (size_t)nlo * t->ncr;
    a.stage_rows = (o + rows <= limit && rows <= 64 * 1024) ? 1 : 0;
    a.off_rows = a.stage_rows ? take(rows) : 0;
    if (ok && o <= limit) {
      const int units = t->nrhs * t->nroot;
      if (t->cluster_mode == 1 && units > cycle_cluster_capacity<T, D>(o, P)) return false;
      *A = a;
      *smem = o;
      return true;
    }
    if (!children) return false;
    children = false;  // retry without the children level
  }
  return false;
}

template <typename T, int D>
bool plan_cluster(gmg_tree *t, int ls, ClusterArgs *A, size_t *smem) {
  if (t->cluster_mode == 0) return false;
  if (!(t->nroot > 1 || t->cb[0] * t->cb[1] * t->cb[2] == 1)) return false;
  if (D == 2) return plan_cluster_pz<T, D>(t, ls, 1, A, smem);
  if (t->cluster_parts != 8 && plan_cluster_pz<T, D>(t, ls, 4, A, smem)) return true;
  return t->cluster_parts != 16 && plan_cluster_pz<T, D>(t, ls, 2, A, smem);
}

// One FAS V-cycle on fields of type T (Sec. 2.2; readings UP and V).
// Levels lmin .. ls: with the cluster kernel at the bottom (and the
// cooperative kernel's down and up legs around it when ls is above the
// cluster's levels), else in one cooperative launch.
template <typename T, int D>
int coop_cycle(gmg_tree *t, cudaStream_t s, int ls) {
  ClusterArgs CA;
  size_t csm = 0;
  if (!plan_cluster<T, D>(t, ls, &CA, &csm)) return coop_launch<T, D>(t, s, ls, 0, 0);
  if (ls > CA.l_top) {
    const int rc = coop_launch<T, D>(t, s, ls, 1, CA.l_top);
    if (rc) return rc;
  }
  cudaError_t e = cudaSuccess;
  const GmgView<T> V = view<T>(t);
  launch(t, s, 10, prec_of<T>(), t->lmin, [&] {
    e = launch_cycle_cluster<T, D>(V, t->d_lvtab, t->lmin, CA, t->nrhs * t->nroot, csm, s, t->use_pdl && !t->prof_on);
  });
  if (e != cudaSuccess) {
    set_error(std::string("cluster kernel of the coarse cycle: ") + cudaGetErrorString(e));
    return GMG_ERR_CUDA;
  }
  if (ls > CA.l_top) return coop_launch<T, D>(t, s, ls, 2, CA.l_top);
  return GMG_OK;
}

// Fused sweeps (fused_sweeps.cuh) run on FP32 levels whose blocks have all
// their neighbours on the level, for 1 or 2 red/black steps per leg.
template <typename T>
bool fused_level(const gmg_tree *t, int l) {
  if (!std::is_same<T, float>::value || !t->use_fused) return false;
  if (bf16_level<T>(t, l)) return false;
  const int n = t->lev(l).n;
  const bool n_ok = t->D == 3 ? (n == 8 || n == 16) : (n == 8 || n == 16 || n == 32);
  const int nd = t->n_down_at(l), nu = t->n_up_at(l);
  const bool k_ok = (nd == 1 || nd == 2) && (nu == 1 || nu == 2);
  return n_ok && k_ok && t->level_complete[l - t->lmin];
}

template <typename T, int D>
void launch_fused(gmg_tree *t, cudaStream_t s, int l, int sweeps, long long in_poff, long long out_poff) {
  GmgView<T> V = view<T>(t);
  LvArgs L = lv(t, l);
  L.poff = in_poff;
  auto go = [&](auto nt, auto kk) {
    constexpr int NT = decltype(nt)::value, K = decltype(kk)::value;
    if constexpr (NT != 0) {
      const size_t sm = FusedGeo<T, D, NT, K>::smem_bytes();
      launch(t, s, 0, prec_of<T>(), l,
             [&] { klaunch(t, L.count * t->nrhs, kThreads, sm, s, k_smooth_tb<T, D, NT, K>, V, L, out_poff); });
    }
  };
  with_nt<D>(L.n, [&](auto nt) {
    if (sweeps == 1)
      go(nt, IC<2>{});
    else
      go(nt, IC<4>{});
  });
}

// One FAS V-cycle on fields of type T (Sec. 2.2; readings UP and V) on the
// levels lmin .. top (top < lmax inside an FMG cycle): the fine levels with
// one launch per phase, the levels up to coop_split in one cooperative
// launch.
template <typename T, int D>
int vcycle_impl(gmg_tree *t, cudaStream_t s, bool end_restrict, int top) {
  GmgView<T> V = view<T>(t);
  const int P = prec_of<T>();
  const int ls = std::min(t->use_coop ? t->coop_split : t->lmin, top);
  const long long other = (long long)t->nrhs * t->total_cells;  // offset of the second FP32 phi buffer
  const int R = t->nrhs;
  for (int l = top; l > ls; l--) {
    LvArgs L = lv(t, l), Lp = lv(t, l - 1);
    const bool bf = bf16_level<T>(t, l);
    const int Pl = bf ? 2 : P;
    if (bf) L.poff = 0;  // the BF16 run is level-local
    const size_t sm = tile_bytes<T>(t, l);
    const int nt_l = cta_threads(t, l), nt_p = cta_threads(t, l - 1);
    const bool fused = fused_level<T>(t, l);
    if (fused) {  // N_down steps in one pass into the second buffer
      launch_fused<T, D>(t, s, l, L.nd, L.off, L.off + other);
      L.poff = L.off + other;
    }
    with_nt<D>(L.n, [&](auto nt) {
      constexpr int NT = decltype(nt)::value;
      size_t lsm = 0;
      if (!fused && !bf && L.nd > 0 && level_leg_ok<T, D, NT>(t, l, &lsm)) {
        launch_level_leg<T, D, NT>(t, s, V, L, Lp, l, 0, lsm);
        return;
      }
      if (!fused)
        for (int k = 0; k < L.nd; k++)
          for (int c = 0; c < 2; c++)
            launch(t, s, 0, Pl, l, [&] { launch_smooth<T, D, NT>(t, V, L, Lp, c, nt_l, sm, s, bf); });
      launch(t, s, 1, Pl, l,
             [&] { launch_resid_restrict<T, D, NT>(t, L.count * R, nt_l, sm, s, V, L, Lp, bf); });
    });
    LvArgs Lpp = l - 2 >= t->lmin ? lv(t, l - 2) : Lp;
    const size_t smp = tile_bytes<T>(t, l - 1);
    with_nt<D>(Lp.n, [&](auto nt) {
      constexpr int NT = decltype(nt)::value;
      launch(t, s, 2, P, l - 1, [&] { klaunch(t, Lp.count * R, nt_p, smp, s, k_fas<T, D, NT>, V, Lp, Lpp); });
    });
  }
  if (t->use_coop) {
    int rc = coop_cycle<T, D>(t, s, ls);
    if (rc) return rc;
  } else {
    LvArgs Lc = lv(t, t->lmin);
    const long long rows = (long long)t->nc * R;
    launch(t, s, 3, P, t->lmin, [&] {
      klaunch(t, (unsigned)((rows + kThreads / 32 - 1) / (kThreads / 32)), kThreads, 0, s, k_coarse<T>, V, Lc, t->d_cinv,
                                                                                              t->ncr, t->nroot);
    });
  }
  for (int l = ls + 1; l <= top; l++) {
    LvArgs L = lv(t, l), Lp = lv(t, l - 1);
    const bool bf = bf16_level<T>(t, l);
    const int Pl = bf ? 2 : P;
    if (bf) L.poff = 0;
    const int hm = L.n / 2 + 2;
    const size_t psm = sizeof(T) * (size_t)(D == 3 ? hm * hm * hm : hm * hm);
    const size_t sm = tile_bytes<T>(t, l);
    const int nt_l = cta_threads(t, l);
    const bool fused = fused_level<T>(t, l);
    if (fused) L.poff = L.off + other;  // the down leg left phi in the second buffer
    with_nt<D>(L.n, [&](auto nt) {
      constexpr int NT = decltype(nt)::value;
      size_t lsm = 0;
      if (!fused && !bf && L.nu > 0 && level_leg_ok<T, D, NT>(t, l, &lsm)) {
        launch_level_leg<T, D, NT>(t, s, V, L, Lp, l, 1, lsm);
        return;
      }
      launch(t, s, 4, Pl, l,
             [&] { launch_prolong<T, D, NT>(t, cta_threads(t, l), L.count * R, psm, s, V, L, Lp, bf); });
      if (!fused)
        for (int k = 0; k < L.nu; k++)
          for (int c = 0; c < 2; c++)
            launch(t, s, 0, Pl, l, [&] { launch_smooth<T, D, NT>(t, V, L, Lp, c, nt_l, sm, s, bf); });
    });
    if (fused) launch_fused<T, D>(t, s, l, L.nu, L.off + other, L.off);  // back to the first buffer
  }
  if (t->adaptive && end_restrict) {
    for (int l = top; l >= 2 && l > t->lmin; l--) {
      LvArgs L = lv(t, l), Lp = lv(t, l - 1);
      const bool bf = bf16_level<T>(t, l);
      if (bf) L.poff = 0;
      with_nt<D>(L.n, [&](auto nt) {
        constexpr int NT = decltype(nt)::value;
        launch(t, s, 5, bf ? 2 : P, l, [&] {
          if constexpr (std::is_same<T, float>::value && NT != 0) {
            if (bf) {
              klaunch(t, L.count * R, cta_threads(t, l), 0, s, k_restrict_phi<T, D, NT, true>, V, L, Lp);
              return;
            }
          }
          klaunch(t, L.count * R, cta_threads(t, l), 0, s, k_restrict_phi<T, D, NT>, V, L, Lp);
        });
      });
    }
  }
  CUDA_TRY(cudaGetLastError());
  return GMG_OK;
}

template <typename T>
int vcycle_any(gmg_tree *t, cudaStream_t s, bool end_restrict = true) {
  return t->D == 3 ? vcycle_impl<T, 3>(t, s, end_restrict, t->lmax) : vcycle_impl<T, 2>(t, s, end_restrict, t->lmax);
}

// One FMG cycle (Sec. 2.2 "Multigrid cycle"; reading FMG): residuals and FAS
// right-hand sides from the finest level to the coarsest without smoothing,
// the exact coarsest-level solve, then for each finer level the prolonged
// coarse correction and one V-cycle with that level on top.
template <typename T, int D>
int fmg_impl(gmg_tree *t, cudaStream_t s) {
  GmgView<T> V = view<T>(t);
  const int P = prec_of<T>();
  const int R = t->nrhs;
  for (int l = t->lmax; l > t->lmin; l--) {
    LvArgs L = lv(t, l);
    const LvArgs Lp = lv(t, l - 1);
    const bool bf = bf16_level<T>(t, l);
    if (bf) L.poff = 0;
    const LvArgs Lpp = l - 2 >= t->lmin ? lv(t, l - 2) : Lp;
    const size_t sm = tile_bytes<T>(t, l), smp = tile_bytes<T>(t, l - 1);
    const int nt_l = cta_threads(t, l), nt_p = cta_threads(t, l - 1);
    with_nt<D>(L.n, [&](auto nt) {
      constexpr int NT = decltype(nt)::value;
      launch(t, s, 1, bf ? 2 : P, l,
             [&] { launch_resid_restrict<T, D, NT>(t, L.count * R, nt_l, sm, s, V, L, Lp, bf); });
    });
    with_nt<D>(Lp.n, [&](auto nt) {
      constexpr int NT = decltype(nt)::value;
      launch(t, s, 2, P, l - 1, [&] { klaunch(t, Lp.count * R, nt_p, smp, s, k_fas<T, D, NT>, V, Lp, Lpp); });
    });
  }
  {
    const LvArgs Lc = lv(t, t->lmin);
    const long long rows = (long long)t->nc * R;
    launch(t, s, 3, P, t->lmin, [&] {
      klaunch(t, (unsigned)((rows + kThreads / 32 - 1) / (kThreads / 32)), kThreads, 0, s, k_coarse<T>, V, Lc, t->d_cinv,
                                                                                              t->ncr, t->nroot);
    });
  }
  for (int l = t->lmin + 1; l <= t->lmax; l++) {
    LvArgs L = lv(t, l);
    const LvArgs Lp = lv(t, l - 1);
    const bool bf = bf16_level<T>(t, l);
    if (bf) L.poff = 0;
    const int hm = L.n / 2 + 2;
    const size_t psm = sizeof(T) * (size_t)(D == 3 ? hm * hm * hm : hm * hm);
    with_nt<D>(L.n, [&](auto nt) {
      constexpr int NT = decltype(nt)::value;
      launch(t, s, 4, bf ? 2 : P, l,
             [&] { launch_prolong<T, D, NT>(t, cta_threads(t, l), L.count * R, psm, s, V, L, Lp, bf); });
    });
    const int rc = vcycle_impl<T, D>(t, s, true, l);
    if (rc) return rc;
  }
  CUDA_TRY(cudaGetLastError());
  return GMG_OK;
}

template <typename T>
int fmg_any(gmg_tree *t, cudaStream_t s) {
  return t->D == 3 ? fmg_impl<T, 3>(t, s) : fmg_impl<T, 2>(t, s);
}

// Composite residual of the FP64 state over the leaf blocks: per-block
// partials, deterministic final reduction into d_red and a copy to the
// pinned host mirror; with `rout` also the float residual (mixed path).
//
// When one level holds all the leaves and its CTAs have kResThreads
// threads, the residual launch's last CTA also does the final reduction
// (ResFold), bit for bit as k_reduce_partials, and the step has one launch
// fewer; at most 64 units, so that one CTA's reduction stays short.
template <int D>
int residual_impl(gmg_tree *t, cudaStream_t s, float *rout) {
  GmgView<double> V = view<double>(t);
  int leaf_levels = 0, only = -1;
  for (int l = t->lmin; l <= t->lmax; l++)
    if (t->level_has_leaves[l - t->lmin]) {
      leaf_levels++;
      only = l;
    }
  ResFold F{};
  if (leaf_levels == 1 && resnorm_threads(t, only) == kResThreads && t->units() <= 64) {
    F.counter = &t->d_bar->fold;
    F.out = t->d_red;
    F.tree_blocks = t->d_tree_blocks;
    F.tree_boff = t->d_tree_boff;
    F.err = &t->d_bar->err;
    F.ntree = t->ntree;
    F.units = t->units();
    F.on = 1;
  }
  for (int l = t->lmin; l <= t->lmax; l++) {
    LvArgs L = lv(t, l), Lp = l > t->lmin ? lv(t, l - 1) : L;
    if (!t->level_has_leaves[l - t->lmin]) continue;
    const size_t sm = resnorm_smem_bytes<double>(D, L.n);
    with_nt<D>(L.n, [&](auto nt) {
      constexpr int NT = decltype(nt)::value;
      launch(t, s, 6, 0, l, [&] {
        klaunch(t, L.count * t->nrhs, resnorm_threads(t, l), sm, s, k_resnorm<double, D, NT>, V, L, Lp, t->d_partials, rout,
                                                                       (int)t->blocks.size(), F);
      });
    });
  }
  if (!F.on)
    launch(t, s, 7, 0, t->lmax, [&] {
      klaunch(t, t->units(), kResThreads, 0, s, k_reduce_partials, (const double *)t->d_partials, (int)t->blocks.size(), (const int *)t->d_tree_blocks,
                                                    t->d_tree_boff, t->ntree, t->d_red, t->d_bar);
    });
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(t->h_red, t->d_red, 4 * sizeof(double) * t->units(), cudaMemcpyDeviceToHost, s));
  return GMG_OK;
}

int residual_any(gmg_tree *t, cudaStream_t s, float *rout) {
  return t->D == 3 ? residual_impl<3>(t, s, rout) : residual_impl<2>(t, s, rout);
}

template <int D>
int restrict_all_phi64(gmg_tree *t, cudaStream_t s) {
  GmgView<double> V = view<double>(t);
  for (int l = t->lmax; l >= 2 && l > t->lmin; l--) {
    LvArgs L = lv(t, l), Lp = lv(t, l - 1);
    with_nt<D>(L.n, [&](auto nt) {
      constexpr int NT = decltype(nt)::value;
      launch(t, s, 5, 0, l, [&] {
        klaunch(t, L.count * t->nrhs, cta_threads(t, l), 0, s, k_restrict_phi<double, D, NT>, V, L, Lp);
      });
    });
  }
  CUDA_TRY(cudaGetLastError());
  return GMG_OK;
}

int restrict_all_phi64_any(gmg_tree *t, cudaStream_t s) {
  return t->D == 3 ? restrict_all_phi64<3>(t, s) : restrict_all_phi64<2>(t, s);
}

// one defect-correction step of the mixed path: e = 0, inner_cycles FP32
// V-cycles on A e = r, phi += e in FP64 (and covered cells restricted).  The
// FP32 cycles skip their closing restriction into covered cells: only the
// leaf values of e are used, and the next step starts again from e = 0.
//
// bf16 (GMG_MIXED_BF16): the finest level's e is kept as BF16 when the tree
// allows it (bf16_eligible); its FP32 part of the first buffer is then not
// cleared, as nothing reads it.
int mixed_step(gmg_tree *t, cudaStream_t s, bool bf16 = false) {
  const bool bf = bf16 && bf16_eligible(t);
  const size_t pitch = (size_t)t->total_cells * sizeof(float);
  if (bf) {
    // e = 0: the levels below the finest (their cells come first in each
    // slot) as FP32, the finest level's BF16 runs
    const long long off = t->lev(t->lmax).off;
    const long long cells = (long long)t->lev(t->lmax).count * t->lev(t->lmax).ncell;
    if (off > 0) CUDA_TRY(cudaMemset2DAsync(t->f_phi, pitch, 0, (size_t)off * sizeof(float), t->nrhs, s));
    CUDA_TRY(cudaMemset2DAsync(bf16_phi(t), pitch, 0, (size_t)cells * sizeof(unsigned short), t->nrhs, s));
  } else {
    // e = 0 in the first FP32 phi buffer of every slot (frozen slots too: harmless)
    CUDA_TRY(cudaMemsetAsync(t->f_phi, 0, (size_t)t->nrhs * t->total_cells * sizeof(float), s));
  }
  t->bf16_top = bf;
  for (int k = 0; k < t->inner_cycles; k++) {
    const int rc = t->fmg_steps ? fmg_any<float>(t, s) : vcycle_any<float>(t, s, k + 1 < t->inner_cycles);
    if (rc) {
      t->bf16_top = false;
      return rc;
    }
  }
  const unsigned short *eh = bf ? bf16_phi(t) : nullptr;
  const int h_first = t->lev(t->lmax).first;
  const long long h_off = t->lev(t->lmax).off;
  t->bf16_top = false;
  launch(t, s, 8, bf ? 2 : 0, t->lmax, [&] {
    klaunch(t, leaf_grid(t), 256, 0, s, k_leaf_accumulate, (const int *)t->d_leaf, (const long long *)t->d_cbase, t->d_phi, (const float *)t->f_phi, n_leaf_blocks(t),
                                                   t->leaf_ncell(), t->total_cells, t->nrhs, t->d_active, t->d_tree_of,
                                                   t->ntree, eh, h_first, h_off, 2 * t->total_cells);
  });
  CUDA_TRY(cudaGetLastError());
  if (t->adaptive) return restrict_all_phi64_any(t, s);
  return GMG_OK;
}

// Runs `enqueue` through a CUDA graph captured on first use (slot), or
// directly while kernel timing is on.
template <typename F>
int run_graph(gmg_tree *t, int slot, cudaStream_t s, F &&enqueue) {
  if (t->prof_on) {
    k_delay<<<1, 32, 0, s>>>(2000);
    return enqueue(s);
  }
  if (!t->use_graphs) return enqueue(s);
  gmg_tree::GraphSlot &g = t->graphs[slot];
  if (!g.exec) {
    if (!t->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&t->cap_stream, cudaStreamNonBlocking));
    const long long before = t->launches;
    CUDA_TRY(cudaStreamBeginCapture(t->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue(t->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(t->cap_stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    CUDA_TRY(e);
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    CUDA_TRY(ei);
    g.kernels = t->launches - before;
    t->launches = before;
  }
  CUDA_TRY(cudaGraphLaunch(g.exec, s));
  t->launches += g.kernels;
  return GMG_OK;
}

// Waits for the stream and checks the barrier flag; the norms of unit u
// (slot, tree) are then h_red[4u .. 4u + 2] = (sum r^2, max |r|, sum b^2).
int read_red(gmg_tree *t, cudaStream_t s) {
  CUDA_TRY(cudaStreamSynchronize(s));
  bool timeout = false;
  for (int u = 0; u < t->units(); u++) timeout = timeout || t->h_red[4 * u + 3] != 0.0;
  if (timeout) {  // a grid barrier timed out: report once, then clear
    CUDA_TRY(cudaMemset(t->d_bar, 0, sizeof(GridBar)));
    set_error("a grid barrier of the coarse-level cycle timed out");
    return GMG_ERR_TIMEOUT;
  }
  return GMG_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t nbr, pnb, parent, pofs, flags, leaf, cbase, st_base, bt_base, phi, b, old, fphi, fb, fold, st, fst, bterm, cinv,
      partials, red, active, tree_of, tree_blocks, tree_boff, bar, spec, lvtab, cellflag, mask_base, dist, bphib,
      dist_base, wallv, wallv_base, leafpos, cut_list, cut_cell, cut_coef, fcut_coef, total;
};

Layout layout(const gmg_tree *t) {
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  const size_t nb = t->blocks.size(), cells = (size_t)t->total_cells, R = (size_t)t->nrhs;
  L.nbr = take(nb * kNbr * sizeof(int));
  L.pnb = take(nb * kNbr * sizeof(int));
  L.parent = take(nb * sizeof(int));
  L.pofs = take(nb * sizeof(int));
  L.flags = take(nb * sizeof(int));
  L.leaf = take(t->leaf_ids_h.size() * sizeof(int));
  L.cbase = take(nb * sizeof(long long));
  L.st_base = take(nb * sizeof(long long));
  L.bt_base = take(nb * sizeof(long long));
  L.phi = take(R * cells * sizeof(double));  // per field: [nrhs][cells]
  L.b = take(R * cells * sizeof(double));
  L.old = take(R * cells * sizeof(double));
  L.fphi = take(2 * R * cells * sizeof(float));  // two buffers [2][nrhs][cells]: fused sweeps write the other one
  L.fb = take(R * cells * sizeof(float));
  L.fold = take(R * cells * sizeof(float));
  L.st = take(t->stencil_h.size() * sizeof(double));
  L.fst = take(t->stencil_h.size() * sizeof(float));
  L.bterm = take(t->bterm_h.size() * sizeof(double));
  L.cinv = take(t->cinv_h.size() * sizeof(double));
  L.partials = take(R * nb * 3 * sizeof(double));
  const size_t U = (size_t)t->units();
  L.red = take(U * 4 * sizeof(double));
  L.active = take(U * sizeof(int));
  L.tree_of = take(nb * sizeof(int));
  L.tree_blocks = take(nb * sizeof(int));
  L.tree_boff = take(((size_t)t->ntree + 1) * sizeof(int));
  L.cellflag = take(t->mask_h.size());
  L.mask_base = take(nb * sizeof(long long));
  L.dist = take(t->dist_h.size() * sizeof(double));
  L.bphib = take(t->bphib_h.size() * sizeof(double));
  L.dist_base = take(nb * sizeof(long long));
  L.wallv = take(t->wallv_h.size() * sizeof(double));
  L.wallv_base = take(nb * sizeof(long long));
  L.leafpos = take(nb * sizeof(int));
  L.bar = take(sizeof(GridBar));
  L.spec = take(t->spec_h.size());
  L.cut_list = take(nb * sizeof(int4));
  L.cut_cell = take((size_t)t->n_cut * sizeof(int));
  L.cut_coef = take(t->cut_coef_h.size() * sizeof(double));
  L.fcut_coef = take(t->cut_coef_h.size() * sizeof(float));
  L.lvtab = take(kMaxLevels * sizeof(LvArgs));
  L.total = o;
  return L;
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// levels up to coop_split run inside one cooperative kernel (few blocks each)
void set_coop_split(gmg_tree *t) {
  t->coop_split = t->lmin;
  for (int l = t->lmin; l <= t->lmax; l++)
    if (t->lev(l).count <= t->coop_max_blocks) t->coop_split = l;
}

void drop_graphs(gmg_tree *t) {
  for (auto &g : t->graphs)
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
}

// per-level descriptors of the cooperative kernel (sweep counts included)
int upload_lvtab(gmg_tree *t) {
  std::vector<LvArgs> tab(t->levels.size());
  for (int l = t->lmin; l <= t->lmax; l++) tab[l - t->lmin] = lv(t, l);
  CUDA_TRY(cudaMemcpy(t->d_lvtab, tab.data(), tab.size() * sizeof(LvArgs), cudaMemcpyHostToDevice));
  return GMG_OK;
}

}  // namespace

extern "C" {

void gmg_default_params(gmg_params *p) {
  if (!p) return;
  p->n_down = 2;
  p->n_up = 2;
  p->eps_tol = 1e-8;
  p->mask_factor = 1.5;
  p->w_min = 0.0;
}

int gmg_tree_create(const gmg_domain *domain, const gmg_params *params, gmg_tree **out) {
  if (!domain || !out) return set_error("null argument"), GMG_ERR_INVALID_ARG;
  *out = nullptr;
  gmg_tree *t = new gmg_tree();
  gmg_default_params(&t->prm);
  if (params) t->prm = *params;
  if (t->prm.n_down < 0 || t->prm.n_up < 0 || t->prm.n_down + t->prm.n_up < 1 || !(t->prm.eps_tol > 0.0) ||
      !(t->prm.mask_factor > 0.0) || t->prm.w_min < 0.0) {
    delete t;
    return set_error("invalid parameters"), GMG_ERR_INVALID_ARG;
  }
  int rc = build_tree(t, domain);
  if (rc != GMG_OK) {
    delete t;
    return rc;
  }
  *out = t;
  return GMG_OK;
}

void gmg_tree_destroy(gmg_tree *t) {
  if (!t) return;
  for (auto &g : t->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (t->cap_stream) cudaStreamDestroy(t->cap_stream);
  for (cudaEvent_t e : t->prof_pool) cudaEventDestroy(e);
  if (t->owns_ws && t->ws) cudaFree(t->ws);
  if (t->h_red) cudaFreeHost(t->h_red);
  if (t->h_active) cudaFreeHost(t->h_active);
  delete t;
}

int gmg_tree_info(const gmg_tree *t, int *lmin, int *lmax, long long *n_leaf_cells, long long *n_blocks) {
  if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
  if (lmin) *lmin = t->lmin;
  if (lmax) *lmax = t->lmax;
  if (n_leaf_cells) *n_leaf_cells = t->n_leaf_cells;
  if (n_blocks) *n_blocks = (long long)t->blocks.size();
  return GMG_OK;
}

int gmg_level_info(const gmg_tree *t, int level, int *n_blocks, int *block_n, double *h) {
  if (!t || level < t->lmin || level > t->lmax) return set_error("level out of range"), GMG_ERR_INVALID_ARG;
  const LevelInfo &L = t->lev(level);
  if (n_blocks) *n_blocks = L.count;
  if (block_n) *block_n = L.n;
  if (h) *h = L.h;
  return GMG_OK;
}

int gmg_level_blocks(const gmg_tree *t, int level, int *bix, int *has_children) {
  if (!t || level < t->lmin || level > t->lmax) return set_error("level out of range"), GMG_ERR_INVALID_ARG;
  const LevelInfo &L = t->lev(level);
  for (int i = 0; i < L.count; i++) {
    const HostBlock &B = t->blocks[L.first + i];
    if (bix)
      for (int d = 0; d < 3; d++) bix[3 * i + d] = B.ix[d];
    if (has_children) has_children[i] = B.has_children;
  }
  return GMG_OK;
}

int gmg_leaf_centers(const gmg_tree *t, double *xyz) {
  if (!t || !xyz) return set_error("null argument"), GMG_ERR_INVALID_ARG;
  long long k = 0;
  for (int id : t->leaf_ids_h) {
    const HostBlock &B = t->blocks[id];
    const LevelInfo &L = t->lev(B.level);
    const double *lo = t->ntree > 1 ? &t->tree_lo_h[3 * (size_t)t->tree_of_h[id]] : t->lo;
    for (int c = 0; c < L.ncell; c++) {
      int p[3] = {c % L.n, (c / L.n) % L.n, t->D == 3 ? c / (L.n * L.n) : 0};
      for (int d = 0; d < t->D; d++) xyz[k * t->D + d] = lo[d] + ((double)(B.ix[d] * L.n + p[d]) + 0.5) * L.h;
      k++;
    }
  }
  return GMG_OK;
}

int gmg_set_walls(gmg_tree *t, const int *types, const double *values, gmg_fn fn, void *user) {
  if (!t || !types) return set_error("null argument"), GMG_ERR_INVALID_ARG;
  if (t->bound) return set_error("walls must be set before gmg_tree_bind"), GMG_ERR_STATE;
  for (int w = 0; w < 2 * t->D; w++) {
    if (types[w] != GMG_WALL_DIRICHLET && types[w] != GMG_WALL_NEUMANN)
      return set_error("invalid wall type"), GMG_ERR_INVALID_ARG;
    t->wall_type[w] = types[w];
    t->wall_val[w] = values ? values[w] : 0.0;
  }
  t->wall_fn = fn;
  t->wall_user = user;
  t->stencils_ready = false;
  return GMG_OK;
}

int gmg_store_stencils(gmg_tree *t, const gmg_lsf *lsf, gmg_fn phib, void *phib_user, double phib_const) {
  if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
  if (t->bound) return set_error("stencils must be stored before gmg_tree_bind"), GMG_ERR_STATE;
  return host_setup(t, lsf, phib, phib_user, phib_const);
}

int gmg_tree_remesh(const gmg_tree *old, gmg_refine_fn refine, void *refine_user, int max_level, gmg_tree **out) {
  if (!old || !out) return set_error("null argument"), GMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!old->stencils_ready) return set_error("the previous tree has no set-up"), GMG_ERR_STATE;
  if (old->ntree != 1) return set_error("forests are re-meshed tree by tree"), GMG_ERR_INVALID_ARG;
  gmg_domain dom{};
  dom.dim = old->D;
  dom.block_n = old->N;
  for (int d = 0; d < 3; d++) {
    dom.coarse_blocks[d] = old->cb[d];
    dom.lo[d] = old->lo[d];
  }
  dom.h_root = old->h1;
  dom.max_level = max_level;
  dom.max_coarse_cells = old->max_coarse;
  dom.refine = refine;
  dom.refine_user = refine_user;
  gmg_tree *t = nullptr;
  int rc = gmg_tree_create(&dom, &old->prm, &t);
  if (rc) return rc;
  for (int w = 0; w < 6; w++) {
    t->wall_type[w] = old->wall_type[w];
    t->wall_val[w] = old->wall_val[w];
  }
  t->wall_fn = old->wall_fn;
  t->wall_user = old->wall_user;
  rc = host_setup(t, &old->lsf_spec, old->phib_fn, old->phib_user, old->phib_const, old);
  if (rc) {
    gmg_tree_destroy(t);
    return rc;
  }
  *out = t;
  return GMG_OK;
}

int gmg_setup_on_device(const gmg_tree *t) { return t && t->setup_device ? 1 : 0; }

int gmg_setup_counts(const gmg_tree *t, long long *computed, long long *reused) {
  if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
  if (computed) *computed = t->setup_computed;
  if (reused) *reused = t->setup_reused;
  return GMG_OK;
}

int gmg_transfer_solution(const gmg_tree *old, gmg_tree *t, void *stream) {
  if (!old || !t) return set_error("null argument"), GMG_ERR_INVALID_ARG;
  if (!old->bound || !t->bound) return set_error("both trees must be bound"), GMG_ERR_STATE;
  if (old->nrhs != t->nrhs || old->D != t->D || old->N != t->N || old->ntree != 1 || t->ntree != 1)
    return set_error("trees of different shape"), GMG_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  const size_t R = (size_t)t->nrhs, no = (size_t)old->total_cells, nn = (size_t)t->total_cells;
  std::vector<double> src(R * no), dst(R * nn, 0.0);
  CUDA_TRY(cudaMemcpyAsync(src.data(), old->d_phi, R * no * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  std::unordered_map<long long, int> old_ids;
  auto key = [](int level, const int *ix) {
    return ((long long)(level + 64) << 57) | ((long long)ix[2] << 38) | ((long long)ix[1] << 19) | (long long)ix[0];
  };
  for (size_t b = 0; b < old->blocks.size(); b++) old_ids[key(old->blocks[b].level, old->blocks[b].ix)] = (int)b;
  auto cbase = [](const gmg_tree *T, int id) {
    const LevelInfo &L = T->lev(T->blocks[id].level);
    return L.off + (long long)(id - L.first) * L.ncell;
  };
  const int D = t->D;
  for (size_t id = 0; id < t->blocks.size(); id++) {  // levels ascending: parents first
    const HostBlock &B = t->blocks[id];
    const LevelInfo &L = t->lev(B.level);
    const long long nb0 = cbase(t, (int)id);
    auto it = old_ids.find(key(B.level, B.ix));
    for (size_t r = 0; r < R; r++) {
      if (it != old_ids.end()) {
        const long long ob = cbase(old, it->second);
        std::memcpy(&dst[r * nn + nb0], &src[r * no + ob], (size_t)L.ncell * sizeof(double));
      } else if (B.parent >= 0) {  // new refinement: the parent's value (injection)
        const LevelInfo &P = t->lev(t->blocks[B.parent].level);
        const long long pb = cbase(t, B.parent);
        for (int c = 0; c < L.ncell; c++) {
          const int x = c % L.n, y = (c / L.n) % L.n, z = D == 3 ? c / (L.n * L.n) : 0;
          const int px = B.pofs[0] + x / 2, py = B.pofs[1] + y / 2, pz = D == 3 ? B.pofs[2] + z / 2 : 0;
          dst[r * nn + nb0 + cs_pos_xyz(x, y, z, L.n, L.ncell)] = dst[r * nn + pb + cs_pos_xyz(px, py, pz, P.n, P.ncell)];
        }
      }
    }
  }
  CUDA_TRY(cudaMemcpyAsync(t->d_phi, dst.data(), R * nn * sizeof(double), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemsetAsync(t->d_active, 1, (size_t)t->units() * sizeof(int), s));
  int rc = restrict_all_phi64_any(t, s);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(s));
  return GMG_OK;
}

int gmg_num_cut_blocks(const gmg_tree *t, int level) {
  if (!t || !t->stencils_ready || level < t->lmin || level > t->lmax) return 0;
  const LevelInfo &L = t->lev(level);
  int s = 0;
  for (int i = 0; i < L.count; i++) s += t->st_base_h[L.first + i] >= 0;
  return s;
}

int gmg_get_distances(const gmg_tree *t, int level, double *out) {
  if (!t || !out || !t->stencils_ready || level < t->lmin || level > t->lmax)
    return set_error("bad arguments or stencils not stored"), GMG_ERR_INVALID_ARG;
  const LevelInfo &L = t->lev(level);
  const int D = t->D;
  size_t k = 0;
  for (int i = 0; i < L.count; i++) {
    long long db = t->dist_base_h[L.first + i];
    for (int c = 0; c < L.ncell * 2 * D; c++) out[k++] = db >= 0 ? t->dist_h[db + c] : 1.0;
  }
  return GMG_OK;
}

int gmg_cut_counts(const gmg_tree *t, int level, int *counts) {
  if (!t || !counts || !t->stencils_ready || level < t->lmin || level > t->lmax)
    return set_error("bad arguments or stencils not stored"), GMG_ERR_INVALID_ARG;
  const LevelInfo &L = t->lev(level);
  for (int i = 0; i < L.count; i++) {
    counts[2 * i] = t->cut_list_h[4 * (size_t)(L.first + i) + 1];
    counts[2 * i + 1] = t->cut_list_h[4 * (size_t)(L.first + i) + 2];
  }
  return GMG_OK;
}

int gmg_get_mask(const gmg_tree *t, int level, int *out) {
  if (!t || !out || !t->stencils_ready || level < t->lmin || level > t->lmax)
    return set_error("bad arguments or stencils not stored"), GMG_ERR_INVALID_ARG;
  const LevelInfo &L = t->lev(level);
  size_t k = 0;
  for (int i = 0; i < L.count; i++) {
    long long mb = t->mask_base_h[L.first + i];
    for (int c = 0; c < L.ncell; c++) out[k++] = t->mask_h[mb + c] & 1;
  }
  return GMG_OK;
}

int gmg_workspace_bytes(const gmg_tree *t, size_t *bytes) {
  if (!t || !bytes) return set_error("null argument"), GMG_ERR_INVALID_ARG;
  if (!t->stencils_ready) return set_error("call gmg_store_stencils first"), GMG_ERR_STATE;
  *bytes = layout(t).total;
  return GMG_OK;
}

int gmg_tree_bind(gmg_tree *t, void *device_ptr, size_t bytes) {
  if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
  if (!t->stencils_ready) return set_error("call gmg_store_stencils first"), GMG_ERR_STATE;
  if (t->bound) return set_error("tree already bound"), GMG_ERR_STATE;
  Layout L = layout(t);
  if (device_ptr) {
    if (bytes < L.total) return set_error("workspace too small"), GMG_ERR_OOM;
    if (reinterpret_cast<uintptr_t>(device_ptr) % 256) return set_error("workspace not 256-byte aligned"), GMG_ERR_INVALID_ARG;
    t->ws = device_ptr;
    t->owns_ws = false;
  } else {
    cudaError_t e = cudaMalloc(&t->ws, L.total);
    if (e != cudaSuccess) return set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e)), GMG_ERR_OOM;
    t->owns_ws = true;
  }
  t->ws_bytes = L.total;
  char *w = static_cast<char *>(t->ws);
  t->d_nbr = reinterpret_cast<int *>(w + L.nbr);
  t->d_pnb = reinterpret_cast<int *>(w + L.pnb);
  t->d_parent = reinterpret_cast<int *>(w + L.parent);
  t->d_pofs = reinterpret_cast<int *>(w + L.pofs);
  t->d_flags = reinterpret_cast<int *>(w + L.flags);
  t->d_leaf = reinterpret_cast<int *>(w + L.leaf);
  t->d_cbase = reinterpret_cast<long long *>(w + L.cbase);
  long long *d_cbase = t->d_cbase;
  t->d_st_base = reinterpret_cast<long long *>(w + L.st_base);
  t->d_bt_base = reinterpret_cast<long long *>(w + L.bt_base);
  t->d_phi = reinterpret_cast<double *>(w + L.phi);
  t->d_b = reinterpret_cast<double *>(w + L.b);
  t->d_old = reinterpret_cast<double *>(w + L.old);
  t->f_phi = reinterpret_cast<float *>(w + L.fphi);
  t->f_b = reinterpret_cast<float *>(w + L.fb);
  t->f_old = reinterpret_cast<float *>(w + L.fold);
  t->d_st = reinterpret_cast<double *>(w + L.st);
  t->f_st = reinterpret_cast<float *>(w + L.fst);
  t->d_bterm = reinterpret_cast<double *>(w + L.bterm);
  t->d_cinv = reinterpret_cast<double *>(w + L.cinv);
  t->d_partials = reinterpret_cast<double *>(w + L.partials);
  t->d_red = reinterpret_cast<double *>(w + L.red);
  t->d_active = reinterpret_cast<int *>(w + L.active);
  t->d_tree_of = reinterpret_cast<int *>(w + L.tree_of);
  t->d_tree_blocks = reinterpret_cast<int *>(w + L.tree_blocks);
  t->d_tree_boff = reinterpret_cast<int *>(w + L.tree_boff);
  t->d_cellflag = reinterpret_cast<unsigned char *>(w + L.cellflag);
  t->d_mask_base = reinterpret_cast<long long *>(w + L.mask_base);
  t->d_dist = reinterpret_cast<double *>(w + L.dist);
  t->d_bphib = reinterpret_cast<double *>(w + L.bphib);
  t->d_dist_base = reinterpret_cast<long long *>(w + L.dist_base);
  t->d_wallv = reinterpret_cast<double *>(w + L.wallv);
  t->d_wallv_base = reinterpret_cast<long long *>(w + L.wallv_base);
  t->d_leafpos = reinterpret_cast<int *>(w + L.leafpos);
  t->d_bar = reinterpret_cast<GridBar *>(w + L.bar);
  t->d_spec = reinterpret_cast<unsigned char *>(w + L.spec);
  t->d_cut_list = reinterpret_cast<int4 *>(w + L.cut_list);
  t->d_cut_cell = reinterpret_cast<int *>(w + L.cut_cell);
  t->d_cut_coef = reinterpret_cast<double *>(w + L.cut_coef);
  t->f_cut_coef = reinterpret_cast<float *>(w + L.fcut_coef);
  t->d_lvtab = reinterpret_cast<LvArgs *>(w + L.lvtab);
  const size_t nb = t->blocks.size();
  std::vector<long long> cbase(nb);
  for (size_t i = 0; i < nb; i++) {
    const LevelInfo &Lv = t->lev(t->blocks[i].level);
    cbase[i] = Lv.off + (long long)((int)i - Lv.first) * Lv.ncell;
  }
  CUDA_TRY(cudaMemcpy(t->d_nbr, t->nbr_h.data(), nb * kNbr * sizeof(int), cudaMemcpyHostToDevice));
  {
    std::vector<int> pnb(nb * kNbr, -2);
    for (size_t i = 0; i < nb; i++) {
      const int P = t->parent_h[i];
      if (P >= 0)
        for (int k = 0; k < kNbr; k++) pnb[i * kNbr + k] = t->nbr_h[(size_t)P * kNbr + k];
    }
    CUDA_TRY(cudaMemcpy(t->d_pnb, pnb.data(), nb * kNbr * sizeof(int), cudaMemcpyHostToDevice));
  }
  CUDA_TRY(cudaMemcpy(t->d_parent, t->parent_h.data(), nb * sizeof(int), cudaMemcpyHostToDevice));
  if (t->ntree == 1) {  // a single tree: every block in tree 0
    t->tree_of_h.assign(nb, 0);
    t->tree_blocks_h.resize(nb);
    for (size_t i = 0; i < nb; i++) t->tree_blocks_h[i] = (int)i;
    t->tree_boff_h = {0, (int)nb};
  }
  CUDA_TRY(cudaMemcpy(t->d_tree_of, t->tree_of_h.data(), nb * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(t->d_tree_blocks, t->tree_blocks_h.data(), nb * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(t->d_tree_boff, t->tree_boff_h.data(), t->tree_boff_h.size() * sizeof(int),
                      cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(t->d_pofs, t->pofs_h.data(), nb * sizeof(int), cudaMemcpyHostToDevice));
  {  // block flags plus, per face, whether the same-level neighbour is covered
    std::vector<int> fl(t->flags_h);
    for (size_t i = 0; i < nb; i++)
      for (int f = 0; f < 2 * t->D; f++) {
        const int a = f >> 1, o = 2 * (f & 1) - 1;
        const int slot = (a == 2 ? o + 1 : 1) * 9 + (a == 1 ? o + 1 : 1) * 3 + (a == 0 ? o + 1 : 1);
        const int id = t->nbr_h[i * kNbr + slot];
        if (id >= 0 && t->blocks[id].has_children) fl[i] |= face_covered_bit(f);
      }
    CUDA_TRY(cudaMemcpy(t->d_flags, fl.data(), nb * sizeof(int), cudaMemcpyHostToDevice));
  }
  CUDA_TRY(cudaMemcpy(t->d_leaf, t->leaf_ids_h.data(), t->leaf_ids_h.size() * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(d_cbase, cbase.data(), nb * sizeof(long long), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(t->d_st_base, t->st_base_h.data(), nb * sizeof(long long), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(t->d_bt_base, t->bt_base_h.data(), nb * sizeof(long long), cudaMemcpyHostToDevice));
  if (!t->stencil_h.empty()) {
    CUDA_TRY(cudaMemcpy(t->d_st, t->stencil_h.data(), t->stencil_h.size() * sizeof(double), cudaMemcpyHostToDevice));
    k_to_float<<<grid_for((long long)t->stencil_h.size()), 256>>>(t->d_st, t->f_st, (long long)t->stencil_h.size());
  }
  if (!t->spec_h.empty()) CUDA_TRY(cudaMemcpy(t->d_spec, t->spec_h.data(), t->spec_h.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(t->d_cut_list, t->cut_list_h.data(), nb * sizeof(int4), cudaMemcpyHostToDevice));
  if (t->n_cut) {
    CUDA_TRY(cudaMemcpy(t->d_cut_cell, t->cut_cell_h.data(), (size_t)t->n_cut * sizeof(int), cudaMemcpyHostToDevice));
    const long long nco = (long long)t->cut_coef_h.size();
    CUDA_TRY(cudaMemcpy(t->d_cut_coef, t->cut_coef_h.data(), nco * sizeof(double), cudaMemcpyHostToDevice));
    k_to_float<<<grid_for(nco), 256>>>(t->d_cut_coef, t->f_cut_coef, nco);
  }
  {
    const int rc = upload_lvtab(t);
    if (rc) return rc;
  }
  if (!t->bterm_h.empty())
    CUDA_TRY(cudaMemcpy(t->d_bterm, t->bterm_h.data(), t->bterm_h.size() * sizeof(double), cudaMemcpyHostToDevice));
  {  // field evaluation tables
    auto up = [](void *d, const void *h, size_t bytes) {
      return bytes ? cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    std::vector<int> leafpos(nb, -1);
    for (size_t k = 0; k < t->leaf_ids_h.size(); k++) leafpos[t->leaf_ids_h[k]] = (int)k;
    CUDA_TRY(up(t->d_cellflag, t->mask_h.data(), t->mask_h.size()));
    CUDA_TRY(up(t->d_mask_base, t->mask_base_h.data(), nb * sizeof(long long)));
    CUDA_TRY(up(t->d_dist, t->dist_h.data(), t->dist_h.size() * sizeof(double)));
    CUDA_TRY(up(t->d_bphib, t->bphib_h.data(), t->bphib_h.size() * sizeof(double)));
    CUDA_TRY(up(t->d_dist_base, t->dist_base_h.data(), nb * sizeof(long long)));
    CUDA_TRY(up(t->d_wallv, t->wallv_h.data(), t->wallv_h.size() * sizeof(double)));
    CUDA_TRY(up(t->d_wallv_base, t->wallv_base_h.data(), nb * sizeof(long long)));
    CUDA_TRY(up(t->d_leafpos, leafpos.data(), nb * sizeof(int)));
  }
  CUDA_TRY(cudaMemcpy(t->d_cinv, t->cinv_h.data(), t->cinv_h.size() * sizeof(double), cudaMemcpyHostToDevice));
  const size_t cells = (size_t)t->total_cells * t->nrhs;
  CUDA_TRY(cudaMemset(t->d_phi, 0, cells * sizeof(double)));
  CUDA_TRY(cudaMemset(t->d_b, 0, cells * sizeof(double)));
  CUDA_TRY(cudaMemset(t->d_old, 0, cells * sizeof(double)));
  CUDA_TRY(cudaMemset(t->f_phi, 0, 2 * cells * sizeof(float)));
  CUDA_TRY(cudaMemset(t->f_b, 0, cells * sizeof(float)));
  CUDA_TRY(cudaMemset(t->f_old, 0, cells * sizeof(float)));
  // blocks on levels without leaves never write their residual partials
  CUDA_TRY(cudaMemset(t->d_partials, 0, (size_t)t->nrhs * nb * 3 * sizeof(double)));
  CUDA_TRY(cudaMemset(t->d_red, 0, (size_t)t->units() * 4 * sizeof(double)));
  CUDA_TRY(cudaMemset(t->d_active, 1, (size_t)t->units() * sizeof(int)));  // nonzero: active
  CUDA_TRY(cudaMemset(t->d_bar, 0, sizeof(GridBar)));
  set_coop_split(t);
  if (!t->h_red) CUDA_TRY(cudaMallocHost(&t->h_red, (size_t)t->units() * 4 * sizeof(double)));
  if (!t->h_active) CUDA_TRY(cudaMallocHost(&t->h_active, (size_t)t->units() * sizeof(int)));
  t->level_complete.assign(t->levels.size(), 1);
  for (size_t i = 0; i < nb; i++)
    for (int k = 0; k < kNbr; k++)
      if (t->nbr_h[i * kNbr + k] == -1) t->level_complete[t->blocks[i].level - t->lmin] = 0;
  t->level_has_leaves.assign(t->levels.size(), 0);
  for (int id : t->leaf_ids_h) t->level_has_leaves[t->blocks[id].level - t->lmin] = 1;
  set_all_smem_limits();
  CUDA_TRY(cudaDeviceSynchronize());
  t->bound = true;
  return GMG_OK;
}


int gmg_set_num_rhs(gmg_tree *t, int nrhs) {
  if (!t || nrhs < 1 || nrhs > 65536) return set_error("bad arguments"), GMG_ERR_INVALID_ARG;
  if (t->bound) return set_error("the slot count must be set before gmg_tree_bind"), GMG_ERR_STATE;
  t->nrhs = nrhs;
  return GMG_OK;
}

int gmg_num_rhs(const gmg_tree *t) { return t ? t->nrhs : 0; }

namespace {
// The device-side address of host memory that kernels can read and write
// directly: page-locked memory mapped into the device's address space (what
// cudaHostAlloc and cudaHostRegister give under unified addressing, and
// what pinned PyTorch tensors use).  The leaf gather and scatter kernels
// then move a host array over the CPU-GPU link themselves, with no staging
// copy.  nullptr for pageable memory, which is staged with cudaMemcpyAsync.
void *mapped_host(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear: an unknown pointer is pageable host memory
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}
}  // namespace

int gmg_set_rhs_slots(gmg_tree *t, int slot0, int nslots, const double *g, int where, void *stream) {
  if (!t || !g) return set_error("null argument"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  if (slot0 < 0 || nslots < 1 || slot0 + nslots > t->nrhs) return set_error("slot range"), GMG_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  const long long n = t->n_leaf_cells;
  const double *gd = g;
  if (where == GMG_HOST) {
    if (const void *m = mapped_host(g)) {
      gd = static_cast<const double *>(m);  // read by the scatter kernel itself
    } else {
      // stage through the FP64 'old' field (scratch until the next V-cycle)
      CUDA_TRY(cudaMemcpyAsync(t->d_old, g, (size_t)nslots * n * sizeof(double), cudaMemcpyHostToDevice, s));
      gd = t->d_old;
    }
  } else if (where != GMG_DEVICE) {
    return set_error("where must be GMG_HOST or GMG_DEVICE"), GMG_ERR_INVALID_ARG;
  }
  k_leaf_rhs<<<leaf_grid(t), 256, 0, s>>>(t->d_leaf, t->d_cbase, t->d_bt_base, t->d_bterm, gd, t->d_b,
                                          n_leaf_blocks(t), t->leaf_ncell(), t->total_cells, slot0, nslots, t->N, t->D);
  CUDA_TRY(cudaMemsetAsync(t->d_phi + (size_t)slot0 * t->total_cells, 0,
                           (size_t)nslots * t->total_cells * sizeof(double), s));
  CUDA_TRY(cudaGetLastError());
  return GMG_OK;
}

int gmg_set_rhs(gmg_tree *t, const double *g, int where, void *stream) {
  if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
  return gmg_set_rhs_slots(t, 0, t->nrhs, g, where, stream);
}

int gmg_set_solution(gmg_tree *t, const double *phi, int where, void *stream) {
  if (!t || !phi) return set_error("null argument"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  cudaStream_t s = as_stream(stream);
  const long long n = t->n_leaf_cells;
  double *src = const_cast<double *>(phi);
  if (where == GMG_HOST) {
    if (void *m = mapped_host(phi)) {
      src = static_cast<double *>(m);
    } else {
      CUDA_TRY(cudaMemcpyAsync(t->d_old, phi, (size_t)t->nrhs * n * sizeof(double), cudaMemcpyHostToDevice, s));
      src = t->d_old;
    }
  }
  k_leaf_copy<<<leaf_grid(t), 256, 0, s>>>(t->d_leaf, t->d_cbase, t->d_phi, src, n_leaf_blocks(t), t->leaf_ncell(),
                                           t->total_cells, 0, t->nrhs, 1, t->N, t->D);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(t->d_active, 1, (size_t)t->units() * sizeof(int), s));
  return restrict_all_phi64_any(t, s);
}

int gmg_get_solution_slots(gmg_tree *t, int slot0, int nslots, double *phi, int where, void *stream) {
  if (!t || !phi) return set_error("null argument"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  if (slot0 < 0 || nslots < 1 || slot0 + nslots > t->nrhs) return set_error("slot range"), GMG_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  const long long n = t->n_leaf_cells;
  const int ncell = t->leaf_ncell();
  if (where == GMG_DEVICE) {
    k_leaf_copy<<<leaf_grid(t), 256, 0, s>>>(t->d_leaf, t->d_cbase, t->d_phi, phi, n_leaf_blocks(t), ncell,
                                             t->total_cells, slot0, nslots, 0, t->N, t->D);
    CUDA_TRY(cudaGetLastError());
    return GMG_OK;
  }
  if (void *m = mapped_host(phi)) {  // the gather kernel writes the host array itself
    k_leaf_copy<<<leaf_grid(t), 256, 0, s>>>(t->d_leaf, t->d_cbase, t->d_phi, static_cast<double *>(m),
                                             n_leaf_blocks(t), ncell, t->total_cells, slot0, nslots, 0, t->N, t->D);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(s));
    return GMG_OK;
  }
  // the FP64 'old' field is dead between V-cycles: stage the gather there
  k_leaf_copy<<<leaf_grid(t), 256, 0, s>>>(t->d_leaf, t->d_cbase, t->d_phi, t->d_old, n_leaf_blocks(t), ncell,
                                           t->total_cells, slot0, nslots, 0, t->N, t->D);
  CUDA_TRY(cudaMemcpyAsync(phi, t->d_old, (size_t)nslots * n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return GMG_OK;
}

int gmg_get_solution(gmg_tree *t, double *phi, int where, void *stream) {
  if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
  return gmg_get_solution_slots(t, 0, t->nrhs, phi, where, stream);
}

int gmg_get_level(gmg_tree *t, int level, int which, double *out, void *stream) {
  if (!t || !out || level < t->lmin || level > t->lmax) return set_error("bad arguments"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  cudaStream_t s = as_stream(stream);
  const LevelInfo &L = t->lev(level);
  const size_t cells = (size_t)L.count * L.ncell;
  std::vector<double> run(cells);
  for (int r = 0; r < t->nrhs; r++) {
    const double *src = (which == 0 ? t->d_phi : t->d_b) + (size_t)r * t->total_cells + L.off;
    CUDA_TRY(cudaMemcpyAsync(run.data(), src, cells * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    // blocks in order, each from the colour-split layout to natural cell order
    for (size_t k = 0; k < (size_t)L.count; k++)
      for (int c = 0; c < L.ncell; c++)
        out[r * cells + k * L.ncell + c] = run[k * L.ncell + cs_pos(c, L.n, L.ncell, t->D)];
  }
  return GMG_OK;
}

namespace {
// unit mask: all units active, or the host array `mask` (nonzero = active)
int upload_mask(gmg_tree *t, const int *mask, cudaStream_t s) {
  const int U = t->units();
  if (!mask) {
    CUDA_TRY(cudaMemsetAsync(t->d_active, 1, (size_t)U * sizeof(int), s));
    return GMG_OK;
  }
  // the pinned mirror may still feed an earlier copy: wait for the stream
  CUDA_TRY(cudaStreamSynchronize(s));
  for (int u = 0; u < U; u++) t->h_active[u] = mask[u] ? 1 : 0;
  CUDA_TRY(cudaMemcpyAsync(t->d_active, t->h_active, (size_t)U * sizeof(int), cudaMemcpyHostToDevice, s));
  return GMG_OK;
}

void slot_norms(const gmg_tree *t, int u, double *rel, double *linf, double *bnorm) {
  const double s2 = t->h_red[4 * u], mx = t->h_red[4 * u + 1], b2 = t->h_red[4 * u + 2];
  if (rel) *rel = b2 > 0 ? std::sqrt(s2 / b2) : std::sqrt(s2);
  if (linf) *linf = mx;
  if (bnorm) *bnorm = std::sqrt(b2);
}
}  // namespace

int gmg_vcycle(gmg_tree *t, int n_cycles, void *stream) {
  if (!t || n_cycles < 0) return set_error("bad arguments"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  t->launches = 0;
  cudaStream_t s = as_stream(stream);
  int rc = upload_mask(t, nullptr, s);
  if (rc) return rc;
  for (int k = 0; k < n_cycles; k++) {
    rc = run_graph(t, gmg_tree::kGraphVcycle64, s, [&](cudaStream_t cs) { return vcycle_any<double>(t, cs); });
    if (rc) return rc;
  }
  return GMG_OK;
}

int gmg_fmg(gmg_tree *t, int n_cycles, void *stream) {
  if (!t || n_cycles < 0) return set_error("bad arguments"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  t->launches = 0;
  cudaStream_t s = as_stream(stream);
  int rc = upload_mask(t, nullptr, s);
  if (rc) return rc;
  for (int k = 0; k < n_cycles; k++) {
    rc = run_graph(t, gmg_tree::kGraphFmg64, s, [&](cudaStream_t cs) { return fmg_any<double>(t, cs); });
    if (rc) return rc;
  }
  return GMG_OK;
}

int gmg_efield(gmg_tree *t, double *out, int where, void *stream) {
  if (!t || !out) return set_error("null argument"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  if (where != GMG_HOST && where != GMG_DEVICE) return set_error("where must be GMG_HOST or GMG_DEVICE"), GMG_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  const size_t n = (size_t)t->nrhs * t->n_leaf_cells * t->D;
  double *dst = out;
  if (where == GMG_HOST) {  // staged in the dead FP64 'old' field when it is large enough, else allocated
    if (n <= (size_t)t->nrhs * t->total_cells) {
      dst = t->d_old;
    } else {
      CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&dst), n * sizeof(double), s));
    }
  }
  int rc = upload_mask(t, nullptr, s);
  if (rc) return rc;
  EfieldArgs E{t->d_cellflag, t->d_mask_base, t->d_dist, t->d_bphib, t->d_dist_base, t->d_wallv, t->d_wallv_base,
               t->d_leafpos, dst, t->n_leaf_cells, 0};
  for (int k = 0; k < t->D; k++) E.dirichlet_upper |= (t->wall_type[2 * k + 1] == GMG_WALL_DIRICHLET ? 1 : 0) << k;
  GmgView<double> V = view<double>(t);
  for (int l = t->lmin; l <= t->lmax; l++) {
    if (!t->level_has_leaves[l - t->lmin]) continue;
    const LvArgs L = lv(t, l), Lp = l > t->lmin ? lv(t, l - 1) : L;
    const size_t sm = tile_bytes<double>(t, l);
    auto go = [&](auto nt) {
      constexpr int NT = decltype(nt)::value;
      if (t->D == 3)
        k_efield<3, NT><<<L.count * t->nrhs, cta_threads(t, l), sm, s>>>(V, L, Lp, E);
      else
        k_efield<2, NT><<<L.count * t->nrhs, cta_threads(t, l), sm, s>>>(V, L, Lp, E);
    };
    if (t->D == 3)
      with_nt<3>(L.n, go);
    else
      with_nt<2>(L.n, go);
  }
  CUDA_TRY(cudaGetLastError());
  if (where == GMG_HOST) {
    CUDA_TRY(cudaMemcpyAsync(out, dst, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (dst != t->d_old) CUDA_TRY(cudaFreeAsync(dst, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  return GMG_OK;
}

int gmg_residual(gmg_tree *t, double *rel_l2, double *linf, void *stream) {
  if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  cudaStream_t s = as_stream(stream);
  t->launches = 0;
  int rc = upload_mask(t, nullptr, s);
  if (rc) return rc;
  rc = run_graph(t, gmg_tree::kGraphResid64, s, [&](cudaStream_t cs) { return residual_any(t, cs, nullptr); });
  if (rc) return rc;
  rc = read_red(t, s);
  if (rc) return rc;
  for (int u = 0; u < t->units(); u++) slot_norms(t, u, rel_l2 ? rel_l2 + u : nullptr, linf ? linf + u : nullptr, nullptr);
  return GMG_OK;
}

int gmg_iterate_begin(gmg_tree *t, int precision, const int *active, int residual_only, void *stream) {
  if (!t || !active) return set_error("null argument"), GMG_ERR_INVALID_ARG;
  if (precision != GMG_FP64 && precision != GMG_MIXED && precision != GMG_MIXED_BF16)
    return set_error("bad precision"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  if (t->step_pending) return set_error("gmg_iterate_end has not collected the previous step"), GMG_ERR_STATE;
  cudaStream_t s = as_stream(stream);
  t->launches = 0;
  const bool mixed = precision != GMG_FP64, bf16 = precision == GMG_MIXED_BF16;
  const int cycle_graph = bf16 ? gmg_tree::kGraphCycleBf16 : mixed ? gmg_tree::kGraphCycleMixed : gmg_tree::kGraphCycle64;
  float *rout = mixed ? t->f_b : nullptr;
  int rc = upload_mask(t, active, s);
  if (rc) return rc;
  if (residual_only)
    rc = run_graph(t, mixed ? gmg_tree::kGraphResidMixed : gmg_tree::kGraphResid64, s,
                   [&](cudaStream_t cs) { return residual_any(t, cs, rout); });
  else
    rc = run_graph(t, cycle_graph, s, [&](cudaStream_t cs) {
      int r = mixed ? mixed_step(t, cs, bf16) : (t->fmg_steps ? fmg_any<double>(t, cs) : vcycle_any<double>(t, cs));
      return r ? r : residual_any(t, cs, rout);
    });
  if (rc) return rc;
  t->step_pending = true;
  t->step_stream = s;
  return GMG_OK;
}

int gmg_iterate_end(gmg_tree *t, double *rel_l2, double *linf) {
  if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
  if (!t->step_pending) return set_error("no step in flight"), GMG_ERR_STATE;
  t->step_pending = false;
  const int rc = read_red(t, t->step_stream);
  if (rc) return rc;
  for (int u = 0; u < t->units(); u++) slot_norms(t, u, rel_l2 ? rel_l2 + u : nullptr, linf ? linf + u : nullptr, nullptr);
  return GMG_OK;
}

int gmg_iterate(gmg_tree *t, int precision, const int *active, int residual_only, double *rel_l2, double *linf,
                void *stream) {
  const int rc = gmg_iterate_begin(t, precision, active, residual_only, stream);
  return rc ? rc : gmg_iterate_end(t, rel_l2, linf);
}

int gmg_solve(gmg_tree *t, int precision, double rel_tol, int max_cycles, gmg_stats *stats, void *stream) {
  if (!t || max_cycles < 0 || !(rel_tol > 0.0)) return set_error("bad arguments"), GMG_ERR_INVALID_ARG;
  if (precision != GMG_FP64 && precision != GMG_MIXED && precision != GMG_MIXED_BF16)
    return set_error("bad precision"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  cudaStream_t s = as_stream(stream);
  t->launches = 0;
  const int R = t->units();
  std::vector<int> act(R, 1), cyc(R, 0);
  std::vector<double> rel(R, 0.0), prev(R, INFINITY);
  int cycles = 0, rc = GMG_OK;
  const bool mixed = precision != GMG_FP64, bf16 = precision == GMG_MIXED_BF16;
  const int cycle_graph = bf16 ? gmg_tree::kGraphCycleBf16 : mixed ? gmg_tree::kGraphCycleMixed : gmg_tree::kGraphCycle64;
  float *rout = mixed ? t->f_b : nullptr;
  // first residual; then each iteration = one cycle + the residual after it,
  // on the slots that have not reached the tolerance yet
  rc = upload_mask(t, nullptr, s);
  if (rc) return rc;
  rc = run_graph(t, mixed ? gmg_tree::kGraphResidMixed : gmg_tree::kGraphResid64, s,
                 [&](cudaStream_t cs) { return residual_any(t, cs, rout); });
  if (rc) return rc;
  for (;;) {
    rc = read_red(t, s);
    if (rc) return rc;
    int left = 0;
    for (int r = 0; r < R; r++) {
      if (!act[r]) continue;
      slot_norms(t, r, &rel[r], nullptr, nullptr);
      if (!std::isfinite(rel[r]) || (cyc[r] > 2 && rel[r] > 1e3 * prev[r])) {
        rc = GMG_ERR_NONFINITE;
        set_error("residual norm is not finite or diverges");
      }
      prev[r] = std::min(prev[r], rel[r]);
      if (rel[r] <= rel_tol) act[r] = 0;
      left += act[r];
    }
    if (rc || left == 0) break;
    if (cycles >= max_cycles) {
      rc = GMG_ERR_NOT_CONVERGED;
      set_error("tolerance not reached within max_cycles");
      break;
    }
    if (R > 1 || !act[0]) {
      rc = upload_mask(t, act.data(), s);
      if (rc) return rc;
    }
    rc = run_graph(t, cycle_graph, s, [&](cudaStream_t cs) {
      int r = mixed ? mixed_step(t, cs, bf16) : (t->fmg_steps ? fmg_any<double>(t, cs) : vcycle_any<double>(t, cs));
      return r ? r : residual_any(t, cs, rout);
    });
    if (rc) return rc;
    cycles++;
    for (int r = 0; r < R; r++) cyc[r] += act[r];
  }
  if (stats)
    for (int r = 0; r < R; r++) {
      stats[r].cycles = cyc[r];
      slot_norms(t, r, &stats[r].rel_l2, &stats[r].linf, &stats[r].bnorm);
    }
  return rc;
}

long long gmg_last_launch_count(const gmg_tree *t) { return t ? t->launches : 0; }

int gmg_set_option(gmg_tree *t, int option, long long value) {
  if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
  switch (option) {
    case GMG_OPT_GRAPHS: t->use_graphs = value != 0; break;
    case GMG_OPT_COARSE_COOP: t->use_coop = value != 0; break;
    case GMG_OPT_FUSED_SWEEPS: t->use_fused = value != 0; break;
    case GMG_OPT_COOP_MAX_BLOCKS:
      if (value < 0) return set_error("block limit must be >= 0"), GMG_ERR_INVALID_ARG;
      t->coop_max_blocks = (int)std::min<long long>(value, 1 << 30);
      if (t->bound) set_coop_split(t);
      break;
    case GMG_OPT_FMG_STEPS: t->fmg_steps = value != 0; break;
    case GMG_OPT_DEVICE_SETUP: t->setup_on_device = value != 0; break;
    case GMG_OPT_CLUSTER_TAIL:
      if (value < 0 || value > 2) return set_error("cluster tail must be 0 (off), 1 (auto) or 2 (whenever the tree qualifies)"), GMG_ERR_INVALID_ARG;
      t->cluster_mode = (int)value;
      break;
    case GMG_OPT_CLUSTER_PARTS:
      if (value != 0 && value != 8 && value != 16) return set_error("cluster parts must be 0 (auto), 8 or 16"), GMG_ERR_INVALID_ARG;
      t->cluster_parts = (int)value;
      break;
    case GMG_OPT_LEVEL_LEGS: t->use_level_legs = value != 0; break;
    case GMG_OPT_PDL:
      t->use_pdl = value != 0;
      drop_graphs(t);
      break;
    case GMG_OPT_SLOTS_PER_CTA:
      if (value != 1 && value != 2 && value != 4) return set_error("slots per CTA must be 1, 2 or 4"), GMG_ERR_INVALID_ARG;
      t->slots_per_cta = (int)value;
      break;
    case GMG_OPT_INNER_CYCLES:
      if (value < 1 || value > 8) return set_error("inner cycles must be 1 .. 8"), GMG_ERR_INVALID_ARG;
      t->inner_cycles = (int)value;
      break;
    case GMG_OPT_CTA_THREADS:
      if (value != 0 && value != 64 && value != 128 && value != 256)
        return set_error("CTA threads must be 0 (by block size), 64, 128 or 256"), GMG_ERR_INVALID_ARG;
      t->cta_threads = (int)value;
      break;
    case GMG_OPT_SPIN_LIMIT:
      if (value < 1) return set_error("spin limit must be positive"), GMG_ERR_INVALID_ARG;
      t->spin_limit = value;
      break;
    default: return set_error("unknown option"), GMG_ERR_INVALID_ARG;
  }
  drop_graphs(t);
  return GMG_OK;
}

int gmg_set_level_sweeps(gmg_tree *t, int level, int n_down, int n_up) {
  if (!t || level < t->lmin || level > t->lmax || n_down < 0 || n_up < 0 || n_down > 64 || n_up > 64)
    return set_error("bad arguments"), GMG_ERR_INVALID_ARG;
  if (t->sweeps_down.empty()) {
    t->sweeps_down.assign(t->levels.size(), t->prm.n_down);
    t->sweeps_up.assign(t->levels.size(), t->prm.n_up);
  }
  t->sweeps_down[level - t->lmin] = n_down;
  t->sweeps_up[level - t->lmin] = n_up;
  if (t->bound) {
    const int rc = upload_lvtab(t);
    if (rc) return rc;
  }
  drop_graphs(t);
  return GMG_OK;
}

int gmg_get_level_sweeps(const gmg_tree *t, int level, int *n_down, int *n_up) {
  if (!t || level < t->lmin || level > t->lmax) return set_error("level out of range"), GMG_ERR_INVALID_ARG;
  if (n_down) *n_down = t->n_down_at(level);
  if (n_up) *n_up = t->n_up_at(level);
  return GMG_OK;
}

int gmg_selftest_conversions(const double *x, const float *f, long long n, unsigned long long *mismatches,
                             void *stream) {
  if (n < 0 || (n > 0 && (!x || !f)) || !mismatches) return set_error("bad arguments"), GMG_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  CUDA_TRY(cudaMemsetAsync(mismatches, 0, 2 * sizeof(unsigned long long), s));
  if (n > 0) {
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    k_selftest_conv<<<(unsigned)blocks, 256, 0, s>>>(x, f, n, mismatches);
    CUDA_TRY(cudaGetLastError());
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  return GMG_OK;
}

int gmg_selftest_barrier_timeout(gmg_tree *t, long long spin_limit, void *stream) {
  if (!t || spin_limit < 1) return set_error("bad arguments"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  cudaStream_t s = as_stream(stream);
  CUDA_TRY(cudaMemsetAsync(t->d_bar, 0, sizeof(GridBar), s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(4);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CUDA_TRY(cudaLaunchKernelEx(&cfg, k_barrier_selftest, t->d_bar, spin_limit));
  GridBar h{};
  CUDA_TRY(cudaMemcpyAsync(&h, t->d_bar, sizeof(GridBar), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  CUDA_TRY(cudaMemsetAsync(t->d_bar, 0, sizeof(GridBar), s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return h.err;
}

int gmg_profile_enable(gmg_tree *t, int enable) {
  if (!t) return set_error("null tree"), GMG_ERR_INVALID_ARG;
  t->prof_on = enable != 0;
  return GMG_OK;
}

int gmg_profile_read(gmg_tree *t, int cap, int *kind, int *prec, int *level, long long *launches, double *ms) {
  if (!t || cap < 0) return set_error("bad arguments"), GMG_ERR_INVALID_ARG;
  struct Agg {
    int kind, prec, level;
    long long n;
    double ms;
  };
  std::vector<Agg> agg;
  for (auto &r : t->prof) {
    CUDA_TRY(cudaEventSynchronize(r.b));
    float e = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&e, r.a, r.b));
    bool found = false;
    for (auto &a : agg)
      if (a.kind == r.kind && a.prec == r.prec && a.level == r.level) {
        a.n += 1;
        a.ms += e;
        found = true;
        break;
      }
    if (!found) agg.push_back({r.kind, r.prec, r.level, 1, (double)e});
  }
  t->prof.clear();
  t->prof_used = 0;
  int k = 0;
  for (auto &a : agg) {
    if (k >= cap) break;
    kind[k] = a.kind;
    prec[k] = a.prec;
    level[k] = a.level;
    launches[k] = a.n;
    ms[k] = a.ms;
    k++;
  }
  return k;
}

const char *gmg_error_string(int code) {
  switch (code) {
    case GMG_OK: return "ok";
    case GMG_ERR_INVALID_ARG: return "invalid argument";
    case GMG_ERR_OOM: return "out of memory";
    case GMG_ERR_CUDA: return "CUDA error";
    case GMG_ERR_NOT_CONVERGED: return "not converged";
    case GMG_ERR_NONFINITE: return "non-finite or diverging residual";
    case GMG_ERR_STATE: return "call out of order";
    case GMG_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown error";
  }
}

const char *gmg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
