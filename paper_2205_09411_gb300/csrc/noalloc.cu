// gmg_residual_noalloc: the composite residual norm of a bound tree without
// any device allocation.  The per-block partial sums, which gmg_residual
// keeps in the tree's workspace, live here in one file-scope device array of
// fixed size instead, so that callers that may not allocate device memory
// (code running inside another runtime's memory pool, allocation-free
// real-time loops, plug-ins that may only use the buffers they are handed)
// can still evaluate the stopping norm.  The array exists once per device
// that loads the library and stays resident until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "gmg_internal.h"
#include "kernels.cuh"

namespace {

// Maximum number of blocks of a tree this entry point accepts: three FP64
// partials per block, 3 MiB in total, plus the final pair of norms.
constexpr int kNoAllocMaxBlocks = 131072;
__device__ __align__(256) double g_noalloc_scratch[3 * kNoAllocMaxBlocks + 2];

// Fixed-order reduction of the partials held in the scratch array (slot 0
// of a tree with several right-hand-side slots); writes
// ||r||_2 / ||b||_2 (or ||r||_2 when b = 0) and max |r| to out[0], out[1].
__global__ void __launch_bounds__(gmg::kResThreads) k_reduce_noalloc(int nb, double *out) {
  __shared__ double s[3];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += g_noalloc_scratch[(size_t)i * 3];
    b = fmax(b, g_noalloc_scratch[(size_t)i * 3 + 1]);
    c += g_noalloc_scratch[(size_t)i * 3 + 2];
  }
  gmg::block_reduce3(a, b, c, s);
  if (threadIdx.x == 0) {
    out[0] = s[2] > 0.0 ? sqrt(s[0] / s[2]) : sqrt(s[0]);
    out[1] = s[1];
  }
}

// The activity flag the residual kernel reads for its one unit: the call
// evaluates slot 0 of every tree together, always, and leaves the tree's
// own unit mask (which a solve on another stream may be using) untouched.
__device__ const int g_noalloc_active = 1;

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
struct DeviceState {
  double *scratch = nullptr;
  const int *active = nullptr;
};
DeviceState g_dev[kMaxDevices];

template <int D, int NT>
cudaError_t resnorm_attrs() {
  cudaError_t e = cudaFuncSetAttribute(gmg::k_resnorm<double, D, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gmg::k_resnorm<double, D, NT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

// Set-up of the current device, once per device: the device addresses of
// the scratch array and of the activity flag (host code holds only
// host-side stand-ins for these symbols), and the shared-memory attributes
// of every kernel variant the call launches.
int device_state(DeviceState *out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gmg::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)), GMG_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return gmg::set_error("device index out of range"), GMG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  DeviceState &st = g_dev[dev];
  if (!st.scratch) {
    void *p = nullptr, *a = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&a, g_noalloc_active);
    if (e != cudaSuccess)
      return gmg::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)), GMG_ERR_CUDA;
    const cudaError_t attrs[] = {resnorm_attrs<3, 4>(), resnorm_attrs<3, 8>(), resnorm_attrs<3, 16>(),
                                 resnorm_attrs<3, 0>(), resnorm_attrs<2, 8>(), resnorm_attrs<2, 16>(),
                                 resnorm_attrs<2, 32>(), resnorm_attrs<2, 0>(),
                                 cudaFuncSetAttribute(k_reduce_noalloc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                      (int)cudaSharedmemCarveoutMaxShared)};
    for (cudaError_t ea : attrs)
      if (ea != cudaSuccess)
        return gmg::set_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ea)), GMG_ERR_CUDA;
    st.scratch = static_cast<double *>(p);
    st.active = static_cast<const int *>(a);
  }
  *out = st;
  return GMG_OK;
}

template <int D, int NT>
void launch_resnorm(gmg_tree *t, int l, double *partials, const int *active, cudaStream_t s) {
  gmg::GmgView<double> V;
  V.nbr = t->d_nbr;
  V.pnb = t->d_pnb;
  V.parent = t->d_parent;
  V.pofs = t->d_pofs;
  V.flags = t->d_flags;
  V.st_base = t->d_st_base;
  V.bt_base = t->d_bt_base;
  V.leaf_ids = t->d_leaf;
  V.phi = t->d_phi;
  V.b = t->d_b;
  V.old = t->d_old;
  V.st = t->d_st;
  V.spec = t->d_spec;
  V.cut_list = t->d_cut_list;
  V.cut_cell = t->d_cut_cell;
  V.cut_coef = t->d_cut_coef;
  V.n_cut = t->n_cut;
  V.wneu = 0;
  for (int w = 0; w < 6; w++) V.wneu |= (t->wall_type[w] == GMG_WALL_NEUMANN ? 1 : 0) << w;
  V.nrhs = 1;  // slot 0 only, all trees of a forest as one unit
  V.rs_phi = V.rs_f = t->total_cells;
  V.hphi = nullptr;
  V.rs_h = 0;
  V.ntree = 1;
  V.tree_of = t->d_tree_of;
  V.active = active;
  const gmg::LevelInfo &Li = t->lev(l);
  gmg::LvArgs L{Li.first, Li.count, Li.n, Li.ncell, Li.off, Li.h, Li.off, 0, 0, Li.h * Li.h, 1.0 / (Li.h * Li.h)};
  gmg::LvArgs Lp = L;
  if (l > t->lmin) {
    const gmg::LevelInfo &Pi = t->lev(l - 1);
    Lp = gmg::LvArgs{Pi.first, Pi.count, Pi.n, Pi.ncell, Pi.off, Pi.h, Pi.off, 0, 0, Pi.h * Pi.h, 1.0 / (Pi.h * Pi.h)};
  }
  const size_t sm = gmg::resnorm_smem_bytes<double>(D, Li.n);
  gmg::ResFold off{};  // partials only; the final reduction is its own launch here
  gmg::k_resnorm<double, D, NT><<<L.count, gmg::resnorm_threads(t, l), sm, s>>>(V, L, Lp, partials, nullptr,
                                                                  (int)t->blocks.size(), off);
}

// the block sides the library's own residual launch specialises
template <int D>
void launch_resnorm_any(gmg_tree *t, int l, double *partials, const int *active, cudaStream_t s) {
  const int n = t->lev(l).n;
  if (D == 3 && n == 4) return launch_resnorm<D, 4>(t, l, partials, active, s);
  if (n == 8) return launch_resnorm<D, 8>(t, l, partials, active, s);
  if (n == 16) return launch_resnorm<D, 16>(t, l, partials, active, s);
  if (D == 2 && n == 32) return launch_resnorm<D, 32>(t, l, partials, active, s);
  launch_resnorm<D, 0>(t, l, partials, active, s);
}

}  // namespace

extern "C" int gmg_residual_noalloc(gmg_tree *t, double *out, void *stream) {
  if (!t || !out) return gmg::set_error("null argument"), GMG_ERR_INVALID_ARG;
  const long long nb = (long long)t->blocks.size();
  if (nb > kNoAllocMaxBlocks)
    return gmg::set_error("gmg_residual_noalloc: the tree has " + std::to_string(nb) +
                          " blocks, more than the fixed scratch holds (" + std::to_string(kNoAllocMaxBlocks) + ")"),
           GMG_ERR_INVALID_ARG;
  if (!t->bound) return gmg::set_error("tree not bound"), GMG_ERR_STATE;
  DeviceState st;
  int rc = device_state(&st);
  if (rc) return rc;
  double *scratch = st.scratch;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // blocks on levels without leaves write no partials: clear the previous
  // call's contents first
  cudaError_t e = cudaMemsetAsync(scratch, 0, (size_t)nb * 3 * sizeof(double), s);
  if (e != cudaSuccess) return gmg::set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)), GMG_ERR_CUDA;
  for (int l = t->lmin; l <= t->lmax; l++) {
    bool leaves = false;
    const gmg::LevelInfo &Li = t->lev(l);
    for (int i = 0; i < Li.count && !leaves; i++) leaves = !t->blocks[Li.first + i].has_children;
    if (!leaves) continue;
    if (t->D == 3)
      launch_resnorm_any<3>(t, l, scratch, st.active, s);
    else
      launch_resnorm_any<2>(t, l, scratch, st.active, s);
  }
  k_reduce_noalloc<<<1, gmg::kResThreads, 0, s>>>((int)nb, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gmg::set_error(std::string("kernel launch: ") + cudaGetErrorString(e)), GMG_ERR_CUDA;
  return GMG_OK;
}
