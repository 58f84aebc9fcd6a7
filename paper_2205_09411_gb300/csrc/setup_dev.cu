// Boundary detection on the device for the built-in level sets (Sec. 3.2,
// Sec. 3.6.1, Sec. 3.6.3): per cell the level set at its centre and the
// boundary mask of Eq. (boundary-mask), then, for the masked cells only,
// the line searches toward the 2D neighbour centres and the unresolved-root
// search.  The host set-up (tree_setup.cpp) takes these results in place of
// its own loops and builds the stencils from them.  This file is compiled
// with --fmad=false and the arithmetic is written in the host set-up's
// order, so every distance equals the host's bit for bit (sqrt and division
// are correctly rounded on both).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gmg_internal.h"
#include "lsf.cuh"

namespace gmg {

namespace {

struct DevLevel {
  int n, ncell;
  double h, lmask;  // cell size; L of Eq. (boundary-mask)
  int bext[3];      // blocks per side of the level's grid (domain extent)
};

struct DevSetupArgs {
  int D, nb;
  double lo[3];
  double eps, w_min;
  LsfSpec spec;
  const int *ix;           // [nb][3] block coordinates
  const int *lev;          // [nb] level index
  const long long *cofs;   // [nb + 1] first cell of each block (block order)
  const DevLevel *levels;  // per level index
};

struct DevLsf {
  LsfSpec spec;
  int D;
  __device__ double operator()(const double *x) const { return lsf_builtin(spec, D, x); }
};

__device__ void cell_centre(const DevSetupArgs &A, const int *B, const DevLevel &L, const int *p, double *x) {
  for (int d = 0; d < 3; d++) x[d] = d < A.D ? A.lo[d] + ((double)(B[d] * L.n + p[d]) + 0.5) * L.h : 0.0;
}

__device__ bool in_dom(const DevLevel &L, int D, const int *G) {
  for (int d = 0; d < D; d++)
    if (G[d] < 0 || G[d] >= L.bext[d] * L.n) return false;
  return true;
}

// Pass 1, one CTA per block: bit 1 of mask[c] when the centre is inside the
// object (f < 0), bit 0 when Eq. (boundary-mask) holds with the central
// difference gradient of step dx; count[b] = masked cells of the block.
__global__ void __launch_bounds__(256) k_setup_mask(DevSetupArgs A, unsigned char *mask, int *count) {
  __shared__ int s_cnt;
  const DevLsf f{A.spec, A.D};
  for (int b = blockIdx.x; b < A.nb; b += gridDim.x) {
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int *B = A.ix + 3 * (size_t)b;
    const DevLevel L = A.levels[A.lev[b]];
    const int n = L.n;
    int cnt = 0;
    for (int c = threadIdx.x; c < L.ncell; c += blockDim.x) {
      const int p[3] = {c % n, (c / n) % n, A.D == 3 ? c / (n * n) : 0};
      double a[3];
      cell_centre(A, B, L, p, a);
      const double fa = f(a);
      unsigned char m = fa < 0.0 ? 2 : 0;
      double gn = 0.0;
      for (int k = 0; k < A.D; k++) {
        double xp[3] = {a[0], a[1], a[2]}, xm[3] = {a[0], a[1], a[2]};
        xp[k] = a[k] + L.h;
        xm[k] = a[k] - L.h;
        const double g = (f(xp) - f(xm)) / (2.0 * L.h);
        gn = gn + g * g;
      }
      gn = sqrt(gn);
      if (fabs(fa) < L.lmask * gn) {
        m |= 1;
        cnt++;
      }
      mask[A.cofs[b] + c] = m;
    }
    if (cnt) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0) count[b] = s_cnt;
    __syncthreads();
  }
}

// Pass 2, one CTA per block: the block's masked cells, in cell order, from
// entry first[b] on (exclusive prefix of the counts).
__global__ void __launch_bounds__(256) k_setup_list(DevSetupArgs A, const unsigned char *mask, const long long *first,
                                                    long long *cells) {
  __shared__ int s_warp[8];
  for (int b = blockIdx.x; b < A.nb; b += gridDim.x) {
    const int nc = (int)(A.cofs[b + 1] - A.cofs[b]);
    const int per = (nc + blockDim.x - 1) / blockDim.x;  // contiguous chunk of cells per thread
    const int c0 = min(nc, (int)threadIdx.x * per), c1 = min(nc, c0 + per);
    int cnt = 0;
    for (int c = c0; c < c1; c++) cnt += mask[A.cofs[b] + c] & 1;
    // exclusive prefix of cnt over the CTA (thread order = cell order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; w++) before += s_warp[w];
    long long at = first[b] + before + incl - cnt;
    for (int c = c0; c < c1; c++)
      if (mask[A.cofs[b] + c] & 1) cells[at++] = A.cofs[b] + c;
    __syncthreads();
  }
}

// Sec. 3.6.3 as on the host: gradient descent from a with step w_min, at
// most floor(dx / w_min) steps; on a sign change the root is located on the
// segment and its distance goes to the axis neighbour closest to the end
// point (when that neighbour is inside the domain).
__device__ void unresolved(const DevSetupArgs &A, const DevLsf &f, const int *B, const DevLevel &L, const int *p,
                           const double *a, double fa, double *dd) {
  const int D = A.D;
  const double w = A.w_min, h = L.h;
  const int nsteps = (int)floor(h / w);
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
    gn = sqrt(gn);
    if (!(gn > 0.0)) return;
    const double sgn = fa > 0.0 ? -1.0 : 1.0;
    for (int k = 0; k < D; k++) x[k] = x[k] + w * (sgn * g[k] / gn);
    const double fx = f(x);
    if (fa * fx <= 0.0) {
      const double t = bisect_root(f, D, a, x, fa, 1.0, A.eps);
      double dist = 0.0;
      for (int k = 0; k < D; k++) dist = dist + (x[k] - a[k]) * (x[k] - a[k]);
      dist = t * sqrt(dist);
      double dv = dist / h;
      dv = dv < A.eps ? A.eps : (dv > 1.0 ? 1.0 : dv);
      int ax = 0;
      double best = fabs(x[0] - a[0]);
      for (int k = 1; k < D; k++)
        if (fabs(x[k] - a[k]) > best) {
          best = fabs(x[k] - a[k]);
          ax = k;
        }
      const int side = x[ax] - a[ax] > 0.0 ? 1 : 0;
      int G[3];
      for (int d = 0; d < 3; d++) G[d] = d < D ? B[d] * L.n + p[d] : 0;
      G[ax] += side ? 1 : -1;
      if (in_dom(L, D, G)) dd[2 * ax + side] = dv;
      return;
    }
  }
}

// Pass 3, one thread per masked cell: the 2D relative distances (1 where no
// root), line searches toward the neighbour centres inside the domain, and
// the unresolved-root search where none found a root.
__global__ void __launch_bounds__(128) k_setup_dist(DevSetupArgs A, const long long *cells, long long m,
                                                    const int *blk_of, double *dist) {
  const DevLsf f{A.spec, A.D};
  const int D = A.D;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x) {
    const long long gc = cells[e];
    const int b = blk_of[e];
    const int *B = A.ix + 3 * (size_t)b;
    const DevLevel L = A.levels[A.lev[b]];
    const int n = L.n, c = (int)(gc - A.cofs[b]);
    const int p[3] = {c % n, (c / n) % n, D == 3 ? c / (n * n) : 0};
    double a[3];
    cell_centre(A, B, L, p, a);
    const double fa = f(a);
    double dd[6] = {1.0, 1.0, 1.0, 1.0, 1.0, 1.0};
    bool found = false;
    for (int k = 0; k < D; k++)
      for (int s = 0; s < 2; s++) {
        int G[3];
        for (int d = 0; d < 3; d++) G[d] = d < D ? B[d] * n + p[d] : 0;
        G[k] += s ? 1 : -1;
        if (!in_dom(L, D, G)) continue;
        double bp[3] = {a[0], a[1], a[2]};
        bp[k] = s ? a[k] + L.h : a[k] - L.h;
        dd[2 * k + s] = line_search(f, D, a, bp, A.eps);
        if (dd[2 * k + s] < 1.0) found = true;
      }
    if (!found && A.w_min > 0.0 && L.h > A.w_min) unresolved(A, f, B, L, p, a, fa, dd);
    for (int k = 0; k < 2 * D; k++) dist[e * 2 * D + k] = dd[k];
  }
}

// Blocks with a located root: cut[b] <- 1 when a masked cell of block b has
// a distance below 1 (every writer stores the same value).
__global__ void k_setup_cutflag(const int *blk_of, const double *dist, long long m, int D, unsigned char *cut) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x) {
    bool any = false;
    for (int k = 0; k < 2 * D; k++) any = any || dist[e * 2 * D + k] < 1.0;
    if (any) cut[blk_of[e]] = 1;
  }
}

struct DevTermsArgs {
  int D, ncut;
  double phib;                  // the constant boundary value
  double wall_val[6];
  int wall_dirichlet;           // bit w: wall w is Dirichlet
  const int *cut_ids;           // [ncut] block ids, block order
  const long long *cut_off;     // [ncut + 1] first cell of each cut block in the dense arrays
  const long long *ent_first;   // [nb + 1] the block's entries in the masked-cell list
  const long long *cells;       // masked cells (block-order cell index)
  const double *dist;           // their distances
};

// One CTA per cut block: its distances made dense (1 where no root, the
// masked cells' values scattered in), then per cell the coefficients of
// Eq. (lpl-1d-lsf) with those toward a located root moved to the right-hand
// side at the constant boundary value (Sec. 3.3, 3.6.2), and the Dirichlet
// wall terms: the host's block_terms, in its order.
__global__ void __launch_bounds__(256) k_setup_terms(DevSetupArgs A, DevTermsArgs B, double *dd, double *stc, double *bt,
                                                     double *pb) {
  const int D = A.D, S = 2 * D + 1;
  for (int i = blockIdx.x; i < B.ncut; i += gridDim.x) {
    const int b = B.cut_ids[i];
    const int *bx = A.ix + 3 * (size_t)b;
    const DevLevel L = A.levels[A.lev[b]];
    const int n = L.n, nc = L.ncell;
    const long long o = B.cut_off[i];
    double *d = dd + o * 2 * D;
    for (int k = threadIdx.x; k < nc * 2 * D; k += blockDim.x) d[k] = 1.0;
    __syncthreads();
    for (long long e = B.ent_first[b] + threadIdx.x; e < B.ent_first[b + 1]; e += blockDim.x) {
      const int c = (int)(B.cells[e] - A.cofs[b]);
      for (int k = 0; k < 2 * D; k++) d[(size_t)c * 2 * D + k] = B.dist[e * 2 * D + k];
    }
    __syncthreads();
    const double h = L.h, inv_h2 = 1.0 / (h * h);
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const int p[3] = {c % n, (c / n) % n, D == 3 ? c / (n * n) : 0};
      const double *dc = d + (size_t)c * 2 * D;
      double diag = 0.0, bnd = 0.0, coef[6];
      for (int k = 0; k < D; k++) {
        const double dm = dc[2 * k], dp = dc[2 * k + 1];
        double cm = 2.0 * inv_h2 / ((dp + dm) * dm);
        double cp = 2.0 * inv_h2 / ((dp + dm) * dp);
        diag = diag - (cm + cp);
        double pm = 0.0, pp = 0.0;
        if (dm < 1.0) {
          pm = B.phib;
          bnd = bnd + cm * pm;
          cm = 0.0;
        }
        if (dp < 1.0) {
          pp = B.phib;
          bnd = bnd + cp * pp;
          cp = 0.0;
        }
        pb[(o + c) * 2 * D + 2 * k] = pm;
        pb[(o + c) * 2 * D + 2 * k + 1] = pp;
        coef[2 * k] = cm;
        coef[2 * k + 1] = cp;
      }
      stc[o * S + c] = diag;
      for (int k = 0; k < 2 * D; k++) stc[o * S + (size_t)(1 + k) * nc + c] = coef[k];
      double t = bnd;
      for (int k = 0; k < D; k++)
        for (int s = 0; s < 2; s++) {
          int G[3];
          for (int q = 0; q < 3; q++) G[q] = q < D ? bx[q] * n + p[q] : 0;
          G[k] += s ? 1 : -1;
          if (in_dom(L, D, G)) continue;
          const int w = 2 * k + s;
          if (!((B.wall_dirichlet >> w) & 1)) continue;
          t = t + coef[2 * k + s] * (2.0 * B.wall_val[w]);
        }
      bt[o + c] = t;
    }
    __syncthreads();
  }
}

// entry e's block: the block whose cell range holds cells[e]
__global__ void k_setup_blk(const long long *cofs, int nb, const long long *cells, long long m, int *blk_of) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nb;  // cofs[lo] <= cells[e] < cofs[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (cofs[mid] <= cells[e])
        lo = mid;
      else
        hi = mid;
    }
    blk_of[e] = lo;
  }
}

// Temporary device buffers and a stream of their own: stream-ordered
// allocation, so that set-ups of several trees in parallel host threads do
// not synchronise the whole device on every free.
struct DevBuf {
  cudaStream_t s = nullptr;
  std::vector<void *> ptrs;
  ~DevBuf() {
    for (void *p : ptrs) cudaFreeAsync(p, s);
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  }
  template <typename T>
  cudaError_t alloc(T **p, size_t n) {
    void *q = nullptr;
    const cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(n, 1) * sizeof(T), s);
    if (e == cudaSuccess) ptrs.push_back(q);
    *p = static_cast<T *>(q);
    return e;
  }
};

}  // namespace

bool device_setup_available() {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

int device_boundary_detection(const gmg_tree *T, const LsfSpec &spec, std::vector<uint8_t> &mask,
                              std::vector<long long> &masked_cells, std::vector<double> &dist, DeviceTerms *terms,
                              double phib) {
#define SETUP_TRY(expr)                                                                   \
  do {                                                                                    \
    const cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) {                                                              \
      set_error(std::string("device set-up: ") + #expr + ": " + cudaGetErrorString(_e)); \
      return GMG_ERR_CUDA;                                                                \
    }                                                                                     \
  } while (0)
  const int D = T->D, nb = (int)T->blocks.size();
  std::vector<int> ix((size_t)3 * nb), lev(nb);
  std::vector<long long> cofs(nb + 1, 0);
  std::vector<DevLevel> levels(T->levels.size());
  for (size_t i = 0; i < T->levels.size(); i++) {
    const LevelInfo &L = T->levels[i];
    DevLevel &d = levels[i];
    d.n = L.n;
    d.ncell = L.ncell;
    d.h = L.h;
    d.lmask = T->prm.mask_factor * std::sqrt((double)D) * L.h;
    for (int k = 0; k < 3; k++) d.bext[k] = L.bext[k];
  }
  for (int b = 0; b < nb; b++) {
    const HostBlock &B = T->blocks[b];
    for (int k = 0; k < 3; k++) ix[3 * (size_t)b + k] = B.ix[k];
    lev[b] = B.level - T->lmin;
    cofs[b + 1] = cofs[b] + T->lev(B.level).ncell;
  }
  const long long ncells = cofs[nb];
  DevBuf buf;
  SETUP_TRY(cudaStreamCreateWithFlags(&buf.s, cudaStreamNonBlocking));
  const cudaStream_t st = buf.s;
  DevSetupArgs A{};
  A.D = D;
  A.nb = nb;
  for (int k = 0; k < 3; k++) A.lo[k] = T->lo[k];
  A.eps = T->prm.eps_tol;
  A.w_min = T->prm.w_min;
  A.spec = spec;
  int *d_ix, *d_lev, *d_count;
  long long *d_cofs, *d_first;
  DevLevel *d_levels;
  unsigned char *d_mask;
  SETUP_TRY(buf.alloc(&d_ix, ix.size()));
  SETUP_TRY(buf.alloc(&d_lev, lev.size()));
  SETUP_TRY(buf.alloc(&d_cofs, cofs.size()));
  SETUP_TRY(buf.alloc(&d_levels, levels.size()));
  SETUP_TRY(buf.alloc(&d_mask, (size_t)ncells));
  SETUP_TRY(buf.alloc(&d_count, (size_t)nb));
  SETUP_TRY(buf.alloc(&d_first, (size_t)nb));
  SETUP_TRY(cudaMemcpyAsync(d_ix, ix.data(), ix.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  SETUP_TRY(cudaMemcpyAsync(d_lev, lev.data(), lev.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  SETUP_TRY(cudaMemcpyAsync(d_cofs, cofs.data(), cofs.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
  SETUP_TRY(cudaMemcpyAsync(d_levels, levels.data(), levels.size() * sizeof(DevLevel), cudaMemcpyHostToDevice, st));
  A.ix = d_ix;
  A.lev = d_lev;
  A.cofs = d_cofs;
  A.levels = d_levels;
  const int grid = std::max(1, std::min(nb, 152 * 16));
  k_setup_mask<<<grid, 256, 0, st>>>(A, d_mask, d_count);
  SETUP_TRY(cudaGetLastError());
  std::vector<int> count(nb);
  SETUP_TRY(cudaMemcpyAsync(count.data(), d_count, (size_t)nb * sizeof(int), cudaMemcpyDeviceToHost, st));
  SETUP_TRY(cudaStreamSynchronize(st));
  std::vector<long long> first(nb);
  long long m = 0;
  for (int b = 0; b < nb; b++) {
    first[b] = m;
    m += count[b];
  }
  long long *d_cells;
  int *d_blk;
  double *d_dist;
  SETUP_TRY(buf.alloc(&d_cells, (size_t)m));
  SETUP_TRY(buf.alloc(&d_blk, (size_t)m));
  SETUP_TRY(buf.alloc(&d_dist, (size_t)m * 2 * D));
  SETUP_TRY(cudaMemcpyAsync(d_first, first.data(), (size_t)nb * sizeof(long long), cudaMemcpyHostToDevice, st));
  k_setup_list<<<grid, 256, 0, st>>>(A, d_mask, d_first, d_cells);
  SETUP_TRY(cudaGetLastError());
  if (m > 0) {
    const int g2 = (int)std::min<long long>((m + 127) / 128, 152LL * 32);
    k_setup_blk<<<g2, 128, 0, st>>>(d_cofs, nb, d_cells, m, d_blk);
    k_setup_dist<<<g2, 128, 0, st>>>(A, d_cells, m, d_blk, d_dist);
    SETUP_TRY(cudaGetLastError());
  }
  if (terms) {  // stencils and terms of the cut blocks (constant boundary and wall values)
    unsigned char *d_cut;
    SETUP_TRY(buf.alloc(&d_cut, (size_t)nb));
    SETUP_TRY(cudaMemsetAsync(d_cut, 0, (size_t)nb, st));
    if (m > 0) {
      const int g2 = (int)std::min<long long>((m + 127) / 128, 152LL * 32);
      k_setup_cutflag<<<g2, 128, 0, st>>>(d_blk, d_dist, m, D, d_cut);
      SETUP_TRY(cudaGetLastError());
    }
    std::vector<unsigned char> cut(nb);
    SETUP_TRY(cudaMemcpyAsync(cut.data(), d_cut, (size_t)nb, cudaMemcpyDeviceToHost, st));
    SETUP_TRY(cudaStreamSynchronize(st));
    terms->cut_ids.clear();
    terms->cell_off.assign(1, 0);
    for (int b = 0; b < nb; b++)
      if (cut[b]) {
        terms->cut_ids.push_back(b);
        terms->cell_off.push_back(terms->cell_off.back() + (cofs[b + 1] - cofs[b]));
      }
    const int ncut = (int)terms->cut_ids.size();
    const long long cc = terms->cell_off.back();
    const int S = 2 * D + 1;
    terms->dd.resize((size_t)cc * 2 * D);
    terms->st.resize((size_t)cc * S);
    terms->bt.resize((size_t)cc);
    terms->pb.resize((size_t)cc * 2 * D);
    if (ncut > 0) {
      std::vector<long long> ent_first(nb + 1);
      for (int b = 0; b < nb; b++) ent_first[b] = first[b];
      ent_first[nb] = m;
      int *d_ids;
      long long *d_off, *d_ef;
      double *d_dd, *d_st, *d_bt, *d_pb;
      SETUP_TRY(buf.alloc(&d_ids, (size_t)ncut));
      SETUP_TRY(buf.alloc(&d_off, (size_t)ncut + 1));
      SETUP_TRY(buf.alloc(&d_ef, (size_t)nb + 1));
      SETUP_TRY(buf.alloc(&d_dd, terms->dd.size()));
      SETUP_TRY(buf.alloc(&d_st, terms->st.size()));
      SETUP_TRY(buf.alloc(&d_bt, terms->bt.size()));
      SETUP_TRY(buf.alloc(&d_pb, terms->pb.size()));
      SETUP_TRY(cudaMemcpyAsync(d_ids, terms->cut_ids.data(), (size_t)ncut * sizeof(int), cudaMemcpyHostToDevice, st));
      SETUP_TRY(cudaMemcpyAsync(d_off, terms->cell_off.data(), ((size_t)ncut + 1) * sizeof(long long),
                                cudaMemcpyHostToDevice, st));
      SETUP_TRY(cudaMemcpyAsync(d_ef, ent_first.data(), ((size_t)nb + 1) * sizeof(long long), cudaMemcpyHostToDevice, st));
      DevTermsArgs B{};
      B.D = D;
      B.ncut = ncut;
      B.phib = phib;
      for (int w = 0; w < 6; w++) {
        B.wall_val[w] = T->wall_val[w];
        if (w < 2 * D && T->wall_type[w] == GMG_WALL_DIRICHLET) B.wall_dirichlet |= 1 << w;
      }
      B.cut_ids = d_ids;
      B.cut_off = d_off;
      B.ent_first = d_ef;
      B.cells = d_cells;
      B.dist = d_dist;
      k_setup_terms<<<std::min(ncut, 152 * 8), 256, 0, st>>>(A, B, d_dd, d_st, d_bt, d_pb);
      SETUP_TRY(cudaGetLastError());
      SETUP_TRY(cudaMemcpyAsync(terms->dd.data(), d_dd, terms->dd.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      SETUP_TRY(cudaMemcpyAsync(terms->st.data(), d_st, terms->st.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      SETUP_TRY(cudaMemcpyAsync(terms->bt.data(), d_bt, terms->bt.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      SETUP_TRY(cudaMemcpyAsync(terms->pb.data(), d_pb, terms->pb.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
  }
  mask.resize((size_t)ncells);
  masked_cells.resize((size_t)m);
  dist.resize((size_t)m * 2 * D);
  SETUP_TRY(cudaMemcpyAsync(mask.data(), d_mask, (size_t)ncells, cudaMemcpyDeviceToHost, st));
  SETUP_TRY(cudaMemcpyAsync(masked_cells.data(), d_cells, (size_t)m * sizeof(long long), cudaMemcpyDeviceToHost, st));
  SETUP_TRY(cudaMemcpyAsync(dist.data(), d_dist, (size_t)m * 2 * D * sizeof(double), cudaMemcpyDeviceToHost, st));
  SETUP_TRY(cudaStreamSynchronize(st));
#undef SETUP_TRY
  return GMG_OK;
}

}  // namespace gmg
