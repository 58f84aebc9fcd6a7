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

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
double *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code only holds a host-side stand-in for the symbol).
int scratch_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gmg::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)), GMG_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return gmg::set_error("device index out of range"), GMG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return gmg::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)), GMG_ERR_CUDA;
    g_addr[dev] = static_cast<double *>(p);
  }
  *out = g_addr[dev];
  return GMG_OK;
}

// Fixed-order reduction of the partials held in the scratch array (slot 0
// of a tree with several right-hand-side slots); writes
// ||r||_2 / ||b||_2 (or ||r||_2 when b = 0) and max |r| to out[0], out[1].
__global__ void __launch_bounds__(1024) k_reduce_noalloc(int nb, double *out) {
  __shared__ double s[3][1024];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += g_noalloc_scratch[(size_t)i * 3];
    b = fmax(b, g_noalloc_scratch[(size_t)i * 3 + 1]);
    c += g_noalloc_scratch[(size_t)i * 3 + 2];
  }
  s[0][threadIdx.x] = a;
  s[1][threadIdx.x] = b;
  s[2][threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s[0][threadIdx.x] += s[0][threadIdx.x + w];
      s[1][threadIdx.x] = fmax(s[1][threadIdx.x], s[1][threadIdx.x + w]);
      s[2][threadIdx.x] += s[2][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s[2][0] > 0.0 ? sqrt(s[0][0] / s[2][0]) : sqrt(s[0][0]);
    out[1] = s[1][0];
  }
}

template <int D, int NT>
void launch_resnorm(gmg_tree *t, int l, double *partials, cudaStream_t s) {
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
  V.nrhs = 1;  // slot 0 only (all trees of a forest)
  V.rs_phi = V.rs_f = t->total_cells;
  V.ntree = t->ntree;
  V.tree_of = t->d_tree_of;
  V.active = t->d_active;
  const gmg::LevelInfo &Li = t->lev(l);
  gmg::LvArgs L{Li.first, Li.count, Li.n, Li.ncell, Li.off, Li.h, Li.off, 0, 0, Li.h * Li.h, 1.0 / (Li.h * Li.h)};
  gmg::LvArgs Lp = L;
  if (l > t->lmin) {
    const gmg::LevelInfo &Pi = t->lev(l - 1);
    Lp = gmg::LvArgs{Pi.first, Pi.count, Pi.n, Pi.ncell, Pi.off, Pi.h, Pi.off, 0, 0, Pi.h * Pi.h, 1.0 / (Pi.h * Pi.h)};
  }
  const size_t sm = gmg::level_smem_bytes<double>(D, Li.n);
  cudaFuncSetAttribute(gmg::k_resnorm<double, D, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(gmg::k_resnorm<double, D, NT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  gmg::k_resnorm<double, D, NT><<<L.count, gmg::resnorm_threads(t, l), sm, s>>>(V, L, Lp, partials, nullptr,
                                                                  (int)t->blocks.size());
}

template <int D>
void launch_resnorm_any(gmg_tree *t, int l, double *partials, cudaStream_t s) {
  switch (t->lev(l).n) {
    case 8: launch_resnorm<D, 8>(t, l, partials, s); break;
    case 16: launch_resnorm<D, 16>(t, l, partials, s); break;
    default: launch_resnorm<D, 0>(t, l, partials, s); break;
  }
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
  double *scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // blocks on levels without leaves write no partials: clear the previous
  // call's contents first
  cudaError_t e = cudaMemsetAsync(scratch, 0, (size_t)nb * 3 * sizeof(double), s);
  if (e != cudaSuccess) return gmg::set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)), GMG_ERR_CUDA;
  // slot 0 active (the unit mask is set by every entry point that runs kernels)
  e = cudaMemsetAsync(t->d_active, 1, (size_t)t->ntree * sizeof(int), s);
  if (e != cudaSuccess) return gmg::set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)), GMG_ERR_CUDA;
  for (int l = t->lmin; l <= t->lmax; l++) {
    bool leaves = false;
    const gmg::LevelInfo &Li = t->lev(l);
    for (int i = 0; i < Li.count && !leaves; i++) leaves = !t->blocks[Li.first + i].has_children;
    if (!leaves) continue;
    if (t->D == 3)
      launch_resnorm_any<3>(t, l, scratch, s);
    else
      launch_resnorm_any<2>(t, l, scratch, s);
  }
  cudaFuncSetAttribute(k_reduce_noalloc, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  k_reduce_noalloc<<<1, 1024, 0, s>>>((int)nb, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gmg::set_error(std::string("kernel launch: ") + cudaGetErrorString(e)), GMG_ERR_CUDA;
  return GMG_OK;
}
