// The coarse part of the V-cycle in one cooperative launch.
//
// The levels with few blocks (the root grid and the first refinement levels)
// hold little data: their phases cost latency, not bandwidth.  This kernel
// runs, for levels l_hi .. l_lo, the same sequence as the per-level kernels
// (Sec. 2.2: N_down red/black sweeps, residual + restriction, FAS right-hand
// side; exact solve on l_lo; prolongation and N_up sweeps on the way up)
// with a grid-wide barrier between dependent phases; the levels with one
// block per root run on one CTA per (root, slot) in shared memory (the
// tail), with CTA barriers only.  In the grid-synced part each CTA works
// through the blocks b = blockIdx.x, +gridDim.x, ... of a phase, so the
// arithmetic is exactly that of the per-level kernels.
#pragma once

#include "csweep.cuh"

namespace gmg {

struct GridBar {
  unsigned int count;  // arrivals during the current launch
  unsigned int fold;   // CTAs of the residual kernel done (ResFold; 0 between launches)
  int err;             // first error recorded by a wait that ran out
  int pad;
};

constexpr long long kSpinLimit = 1LL << 24;  // polls of a barrier before it reports a timeout (seconds)

// Grid-wide barrier of a cooperative launch (all CTAs co-resident).  The
// arrival counter only grows during a launch (the host zeroes it before
// each one).  Thread 0 of each CTA counts the barriers its CTA has passed
// (`epoch`, the same in every CTA), adds one to the counter with a release
// reduction (no reply to wait for) and polls with acquire loads and short
// sleeps until the counter reaches epoch x CTA count.  The wait is bounded:
// when it runs out it records GMG_ERR_TIMEOUT, so a barrier that can never
// complete ends the kernel instead of hanging it.  Returns the same verdict
// to every thread of the CTA: false once any CTA has recorded an error.
__device__ __forceinline__ bool grid_sync(GridBar *bar, unsigned int nctas, long long spin_limit,
                                          unsigned int *epoch) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int *verr = &bar->err;
    const unsigned int target = ++*epoch * nctas;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;\n" ::"l"(&bar->count) : "memory");
    long long spins = 0;
    for (;;) {
      unsigned int cur;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(cur) : "l"(&bar->count) : "memory");
      if ((int)(cur - target) >= 0 || *verr != 0) break;
      if (++spins > spin_limit) {
        atomicCAS(&bar->err, 0, GMG_ERR_TIMEOUT);
        break;
      }
      __nanosleep(32);
    }
    s_ok = *verr == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// level descriptors of the cycle, staged in shared memory by the kernel
struct LevelSet {
  LvArgs lv[kMaxLevels];
  int lmin;
};

struct CycleArgs {
  int l_lo, l_hi;
  int ncr, nroot;  // coarsest-level unknowns per root, independent roots (inverse per root)
  const double *cinv;
  GridBar *bar;
  long long spin_limit;
  int l_one;  // levels l_lo .. l_one hold one block per root and run one CTA per (root, slot) (< l_lo: none)
  int cinv_off;  // byte offset of the tail's FP64 b and copy of its root's inverse in shared memory (-1: none)
  int mode;      // 0 whole coarse cycle; 1 down leg to the FAS of l_one (no tail); 2 up leg from l_one + 1
};

// Block operations with the compile-time side NT for levels >= 1 and the
// runtime side for the coarse sub-levels inside the root blocks.
template <typename T, int D, int NT>
__device__ __forceinline__ void smooth_any(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid, int c,
                                           unsigned char *sm) {
  if constexpr (NT != 0) {
    if (L.n == NT) {  // the colour-split half-sweep, on the slot view (slot 0 of it)
      const int slot0[1] = {0};
      smooth_cs_block<T, D, NT, 1>(V, L, Lp, bid, slot0, c, sm);
      return;
    }
  }
  smooth_block<T, D, 0>(V, L, Lp, bid, c, sm);
}
template <typename T, int D, int NT>
__device__ __forceinline__ void resid_restrict_any(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid,
                                                   unsigned char *sm) {
  if (NT && L.n == NT)
    resid_restrict_block<T, D, NT>(V, L, Lp, bid, sm);
  else
    resid_restrict_block<T, D, 0>(V, L, Lp, bid, sm);
}
template <typename T, int D, int NT>
__device__ __forceinline__ void fas_any(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid,
                                        unsigned char *sm) {
  if (NT && L.n == NT)
    fas_block<T, D, NT>(V, L, Lp, bid, sm);
  else
    fas_block<T, D, 0>(V, L, Lp, bid, sm);
}
template <typename T, int D, int NT>
__device__ __forceinline__ void prolong_any(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid,
                                            unsigned char *sm) {
  if (NT && L.n == NT)
    prolong_block<T, D, NT>(V, L, Lp, bid, sm);
  else
    prolong_block<T, D, 0>(V, L, Lp, bid, sm);
}

// Exact solve on level Lc by warps w0, w0 + nw, ... : phi = A^-1 b per root
// and slot, one warp per row, FP64 accumulation.
template <typename T>
__device__ __forceinline__ void coarse_rows(const GmgView<T> &V, const LvArgs &Lc, const CycleArgs &A, int w0,
                                            int nw) {
  const int lane = threadIdx.x & 31;
  const int M = A.ncr * A.nroot;
  for (long long item = w0; item < (long long)M * V.nrhs; item += nw) {
    const int r = (int)(item / M), row = (int)(item % M);
    const int k = row / A.ncr, i = row - k * A.ncr;
    if (!V.active[V.ntree > 1 ? r * V.ntree + k : r]) continue;  // root k = tree k of a forest
    const double *a = A.cinv + ((size_t)k * A.ncr + i) * A.ncr;
    const T *b = V.b + r * V.rs_f + Lc.off + (size_t)k * A.ncr;
    double s = 0.0;
    for (int j = lane; j < A.ncr; j += 32) s += a[j] * (double)b[coarse_pos(j, Lc)];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) V.phi[r * V.rs_phi + Lc.poff + (size_t)k * A.ncr + coarse_pos(i, Lc)] = T(s);
  }
}

// ---------------------------------------------------------------------------
// Bottom of the cycle held in shared memory.  On levels l_lo .. l_one each
// independent root (one tree of a forest, or the only root) holds one block
// that covers its whole domain (the root block and its coarsened copies):
// all its faces are walls, and its block on one level covers its parent
// entirely; block k of each such level belongs to root k.  One CTA per
// (root, slot) loads phi and the FAS right-hand side of l_one once, runs
// sweeps, residual + restriction, FAS right-hand sides, the exact solve,
// prolongation and sweeps on shared-memory copies of every level (same
// formulas as the block kernels), and writes phi of l_one back.
template <typename T, int D>
struct TailLevel {
  T *tile, *b, *old;
  unsigned short *eidx;  // per cell: 0 regular stencil, e + 1 entry e of the block's cut list
  T *cf;                 // the list's coefficients, coefficient k of entry e at cf[k * m + e]
  int n, ncell, m;       // m: entries of the cut list (0: regular block)
  LvArgs L;
};

// shared memory of one tail level whose block lists at most mmax cells
template <typename T, int D>
__host__ __device__ __forceinline__ size_t tail_level_bytes(int n, int mmax) {
  const int nc = D == 3 ? n * n * n : n * n;
  const size_t cf = (sizeof(T) * (size_t)mmax * (2 * D + 1) + 15) / 16 * 16;
  return sizeof(T) * ((size_t)TileGeo<T, D>(n).size + 2 * (size_t)nc) + (size_t)((2 * nc + 15) / 16 * 16) + cf;
}

// The tail functions take their level descriptors by value: the copies sit
// in registers, where stores through the level's pointers cannot alias
// them (descriptors read from shared memory would be reloaded after every
// store).

// stencil of cell c of a tail level: false for the regular one
template <typename T, int D>
__device__ __forceinline__ bool tail_cut(const TailLevel<T, D> &Q, int c, int *e) {
  if (Q.m == 0) return false;
  *e = (int)Q.eidx[c] - 1;
  return *e >= 0;
}

// wall ghosts of a single-block level (all faces are walls): sign * mirror
template <typename T, int D>
__device__ __forceinline__ void tail_walls(const TailLevel<T, D> Q, int wneu) {
  const TileGeo<T, D> G(Q.n);
  const int n = Q.n, nf = D == 3 ? n * n : n;
  for (int i = threadIdx.x; i < 2 * D * nf; i += blockDim.x) {
    const int f = i / nf, j = i - f * nf;
    const int a = f >> 1, side = f & 1;
    int u, v, dummy;
    cell_xyz_rt<2>(j, n, &u, &v, &dummy);
    if (D == 2) v = 0;
    const int gn = side ? n : -1, mn = side ? n - 1 : 0;
    const int gx = a == 0 ? gn : u, gy = a == 1 ? gn : (a == 0 ? u : v), gz = a == 2 ? gn : v;
    const int mx = a == 0 ? mn : u, my = a == 1 ? mn : (a == 0 ? u : v), mz = a == 2 ? mn : v;
    Q.tile[G.idx(gx, gy, gz)] = (((wneu >> f) & 1) ? T(1) : T(-1)) * Q.tile[G.idx(mx, my, mz)];
  }
  __syncthreads();
}

// One half-sweep of a single-block level.  Every face is a wall, and a wall
// ghost is the sign times the cell that reads it (reading W), so the
// neighbour values are formed on the fly from the cell's own value instead
// of a separate ghost pass and barrier; the sums are those of nb_sum and
// offdiag_of.
template <typename T, int D>
__device__ __forceinline__ void tail_smooth(const GmgView<T> &V, const TailLevel<T, D> Q, int color) {
  const TileGeo<T, D> G(Q.n);
  const int n = Q.n;
  const T h2 = T(Q.L.h2), inv2d = T(1.0 / (2 * D));
  T sg[2 * D];
#pragma unroll
  for (int f = 0; f < 2 * D; f++) sg[f] = ((V.wneu >> f) & 1) ? T(1) : T(-1);
  for (int j = threadIdx.x; j < Q.ncell / 2; j += blockDim.x) {
    int x, y, z;
    colour_xyz<D>(j, n, color, &x, &y, &z);
    const int c = x + n * (y + n * z);
    const int t = G.idx(x, y, z);
    const T own = Q.tile[t];
    const T xm = x > 0 ? Q.tile[t - 1] : sg[0] * own, xp = x < n - 1 ? Q.tile[t + 1] : sg[1] * own;
    const T ym = y > 0 ? Q.tile[t - G.sy] : sg[2] * own, yp = y < n - 1 ? Q.tile[t + G.sy] : sg[3] * own;
    T zm = T(0), zp = T(0);
    if (D == 3) {
      zm = z > 0 ? Q.tile[t - G.sz] : sg[4] * own;
      zp = z < n - 1 ? Q.tile[t + G.sz] : sg[5] * own;
    }
    T nv;
    int e;
    if (!tail_cut(Q, c, &e)) {
      T sum = (xm + xp) + (ym + yp);
      if (D == 3) sum += zm + zp;
      nv = (sum - h2 * Q.b[c]) * inv2d;
    } else {
      T a[2 * D + 1];
#pragma unroll
      for (int k = 0; k < 2 * D + 1; k++) a[k] = Q.cf[k * Q.m + e];
      T sum = a[1] * xm + a[2] * xp + a[3] * ym + a[4] * yp;
      if (D == 3) sum += a[5] * zm + a[6] * zp;
      nv = (Q.b[c] - sum) / a[0];
    }
    Q.tile[t] = nv;
  }
  __syncthreads();
}

// residual of level F restricted into level C (C covered entirely by F):
// phi_C <- mean phi_F, b_C <- mean r_F
template <typename T, int D>
__device__ __forceinline__ void tail_resid_restrict(const GmgView<T> &V, const TailLevel<T, D> F,
                                                    const TailLevel<T, D> Cq) {
  tail_walls<T, D>(F, V.wneu);
  const TileGeo<T, D> G(F.n), Gc(Cq.n);
  const int n = F.n, hn = Cq.n;
  const T inv_h2 = T(F.L.ih2), w = T(1.0 / (1 << D));
  for (int j = threadIdx.x; j < Cq.ncell; j += blockDim.x) {
    int qx, qy, qz;
    cell_xyz_rt<D>(j, hn, &qx, &qy, &qz);
    T sp = T(0), sr = T(0);
#pragma unroll
    for (int dz = 0; dz < (D == 3 ? 2 : 1); dz++)
#pragma unroll
      for (int dy = 0; dy < 2; dy++)
#pragma unroll
        for (int dx = 0; dx < 2; dx++) {
          const int x = 2 * qx + dx, y = 2 * qy + dy, z = 2 * qz + dz;
          const int c = x + n * (y + n * z);
          const int t = G.idx(x, y, z);
          sp = sp + F.tile[t];
          int e;
          const bool cut = tail_cut(F, c, &e);
          sr = sr + resid_cell<T, D>(F.cf, cut ? 0 : -1, F.tile, t, G.sy, G.sz, F.m, e, inv_h2, F.b[c]);
        }
    Cq.tile[Gc.idx(qx, qy, qz)] = sp * w;
    Cq.b[j] = sr * w;
  }
  __syncthreads();
}

// FAS right-hand side b <- A phi + b (restricted residual), old <- phi
template <typename T, int D>
__device__ __forceinline__ void tail_fas(const GmgView<T> &V, const TailLevel<T, D> Q) {
  tail_walls<T, D>(Q, V.wneu);
  const TileGeo<T, D> G(Q.n);
  const int n = Q.n;
  const T inv_h2 = T(Q.L.ih2);
  for (int c = threadIdx.x; c < Q.ncell; c += blockDim.x) {
    int x, y, z;
    cell_xyz_rt<D>(c, n, &x, &y, &z);
    const int t = G.idx(x, y, z);
    const T ph = Q.tile[t];
    T ap;
    int e;
    if (!tail_cut(Q, c, &e)) {
      ap = inv_h2 * (nb_sum<T, D>(Q.tile, t, G.sy, G.sz) - T(2 * D) * ph);
    } else {
      T diag;
      const T sum = offdiag_st<T, D>(Q.cf, Q.tile, t, G.sy, G.sz, Q.m, e, &diag);
      ap = diag * ph + sum;
    }
    Q.b[c] = ap + Q.b[c];
    Q.old[c] = ph;
  }
  __syncthreads();
}

// The correction phi - old of a single-block level, in place in its tile
// (the level is dead once it has been prolongated), with its ghost layer:
// outside the block the correction is reflected at the walls, with the
// homogeneous sign of each wall crossed (reading P).
template <typename T, int D>
__device__ __forceinline__ void tail_corr_fill(const TailLevel<T, D> C, int wneu) {
  const TileGeo<T, D> G(C.n);
  const int n = C.n;
  for (int c = threadIdx.x; c < C.ncell; c += blockDim.x) {
    int x, y, z;
    cell_xyz_rt<D>(c, n, &x, &y, &z);
    const int t = G.idx(x, y, z);
    C.tile[t] = C.tile[t] - C.old[c];
  }
  __syncthreads();
  const int m = n + 2, tot = D == 3 ? m * m * m : m * m;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int p[3] = {i % m - 1, (i / m) % m - 1, D == 3 ? i / (m * m) - 1 : 0};
    int q[3] = {p[0], p[1], p[2]};
    T sg = T(1);
    bool out = false;
#pragma unroll
    for (int d = 0; d < D; d++) {
      if (p[d] < 0) {
        q[d] = 0;
        sg *= ((wneu >> (2 * d)) & 1) ? T(1) : T(-1);
        out = true;
      } else if (p[d] >= n) {
        q[d] = n - 1;
        sg *= ((wneu >> (2 * d + 1)) & 1) ? T(1) : T(-1);
        out = true;
      }
    }
    if (out) C.tile[G.idx(p[0], p[1], p[2])] = sg * C.tile[G.idx(q[0], q[1], q[2])];
  }
  __syncthreads();
}

// phi_F += trilinear prolongation of the correction of level C
template <typename T, int D>
__device__ __forceinline__ void tail_prolong(const GmgView<T> &V, const TailLevel<T, D> F, const TailLevel<T, D> Cq) {
  tail_corr_fill<T, D>(Cq, V.wneu);
  const TileGeo<T, D> G(F.n), Gc(Cq.n);
  const int n = F.n;
  for (int c = threadIdx.x; c < F.ncell; c += blockDim.x) {
    int x, y, z;
    cell_xyz_rt<D>(c, n, &x, &y, &z);
    const int u[3] = {x >> 1, y >> 1, z >> 1};
    const int o[3] = {(x & 1) ? 1 : -1, (y & 1) ? 1 : -1, (z & 1) ? 1 : -1};
    T v = T(0);
#pragma unroll
    for (int sz = 0; sz < (D == 3 ? 2 : 1); sz++)
#pragma unroll
      for (int sy = 0; sy < 2; sy++)
#pragma unroll
        for (int sx = 0; sx < 2; sx++) {
          T wgt = (sx ? T(0.25) : T(0.75)) * (sy ? T(0.25) : T(0.75));
          if (D == 3) wgt *= sz ? T(0.25) : T(0.75);
          v = v + wgt * Cq.tile[Gc.idx(u[0] + sx * o[0], u[1] + sy * o[1], D == 3 ? u[2] + sz * o[2] : 0)];
        }
    F.tile[G.idx(x, y, z)] += v;
  }
  __syncthreads();
}

template <typename T, int D>
__device__ void tail_cycle(const GmgView<T> &V, const LevelSet &LS, const CycleArgs &A, int top, int root,
                           unsigned char *smem_raw) {
  constexpr int kMaxTail = 12;
  __shared__ TailLevel<T, D> Q[kMaxTail];  // descriptors in shared memory, not per-thread local memory
  __shared__ int s_m[kMaxTail], s_e0[kMaxTail];
  const int ntl = top - A.l_lo + 1;
  {  // phi and b of the top tail level: cp.async, in flight during the set-up
    const LvArgs &L0 = LS.lv[top - LS.lmin];
    const int n = L0.n, nc = D == 3 ? n * n * n : n * n;
    // the tile's layout as the descriptors below will carve it: the top
    // level's tile first, its b right after
    T *tile = reinterpret_cast<T *>(smem_raw);
    T *bq = tile + TileGeo<T, D>(n).size;
    const TileGeo<T, D> G(n);
    const T *phi = V.phi + L0.poff + (long long)root * nc;
    const T *b = V.b + L0.off + (long long)root * nc;
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {  // the block's colour-split run in order
      int x, y, z;
      cs_xyz(q, n, nc, D, &x, &y, &z);
      cp_async_elem(tile + G.idx(x, y, z), phi + q);
      cp_async_elem(bq + x + n * (y + n * z), b + q);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  if ((int)threadIdx.x < ntl) {  // the levels' cut lists, read in parallel
    const int4 cl = V.cut_list[LS.lv[top - (int)threadIdx.x - LS.lmin].first + root];
    s_m[threadIdx.x] = cl.y + cl.z;
    s_e0[threadIdx.x] = cl.x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T *p = reinterpret_cast<T *>(smem_raw);
    for (int l = top; l >= A.l_lo; l--) {
      TailLevel<T, D> &q = Q[top - l];
      q.L = LS.lv[l - LS.lmin];
      q.n = q.L.n;
      q.ncell = D == 3 ? q.n * q.n * q.n : q.n * q.n;
      q.L.first += root;  // this root's block of the level
      q.L.off += (long long)root * q.ncell;
      q.L.poff += (long long)root * q.ncell;
      q.m = s_m[top - l];
      q.tile = p;
      p += TileGeo<T, D>(q.n).size;
      q.b = p;
      p += q.ncell;
      q.old = p;
      p += q.ncell;
      q.eidx = reinterpret_cast<unsigned short *>(p);
      p += (2 * q.ncell + 15) / 16 * 16 / sizeof(T);
      q.cf = p;
      p += (sizeof(T) * (size_t)q.m * (2 * D + 1) + 15) / 16 * 16 / sizeof(T);
    }
  }
  __syncthreads();
  // cut lists of the tail levels: entry index per cell, coefficients
  for (int l = top; l >= A.l_lo; l--) {
    const TailLevel<T, D> q = Q[top - l];
    if (q.m)
      for (int c = threadIdx.x; c < q.ncell; c += blockDim.x) q.eidx[c] = 0;
  }
  __syncthreads();
  for (int l = top; l >= A.l_lo; l--) {
    const TailLevel<T, D> q = Q[top - l];
    if (!q.m) continue;
    const int e0 = s_e0[top - l];
    for (int e = threadIdx.x; e < q.m; e += blockDim.x) {
      q.eidx[V.cut_cell[e0 + e]] = (unsigned short)(e + 1);
#pragma unroll
      for (int k = 0; k < 2 * D + 1; k++) q.cf[k * q.m + e] = V.cut_coef[k * V.n_cut + e0 + e];
    }
  }
  // the root's coarse inverse, copied while the tail smooths its way down
  const double *cinv = A.cinv + (size_t)root * A.ncr * A.ncr;
  if (A.cinv_off >= 0) {  // [b in FP64 (ncr) | inverse (ncr x ncr)]
    double *dst = reinterpret_cast<double *>(smem_raw + A.cinv_off) + A.ncr;
    for (int i = threadIdx.x; i < A.ncr * A.ncr; i += blockDim.x) cp_async_elem(dst + i, cinv + i);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    cinv = dst;
  }
  // the top level's phi and b have landed (the inverse may still be in flight)
  if (A.cinv_off >= 0)
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  else
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  for (int l = top; l > A.l_lo; l--) {
    const TailLevel<T, D> &F = Q[top - l], &Cq = Q[top - l + 1];
    for (int k = 0; k < F.L.nd; k++) {
      tail_smooth<T, D>(V, F, 0);
      tail_smooth<T, D>(V, F, 1);
    }
    tail_resid_restrict<T, D>(V, F, Cq);
    tail_fas<T, D>(V, Cq);
  }
  {  // exact solve on l_lo, FP64 accumulation
    if (A.cinv_off >= 0) {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();
    }
    const TailLevel<T, D> &q = Q[top - A.l_lo];
    const TileGeo<T, D> G(q.n);
    // b in FP64 once, not once per row (beside the staged inverse)
    double *bd = reinterpret_cast<double *>(smem_raw + A.cinv_off);
    const bool bd_ok = A.cinv_off >= 0;
    if (bd_ok) {
      for (int j = threadIdx.x; j < A.ncr; j += blockDim.x) bd[j] = (double)q.b[j];
      __syncthreads();
    }
    // 8 threads per row, each summing every 8th column, then a 3-step
    // reduction: on one SM the FP64 adds of a 32-lane reduction tree would
    // cost more than the multiply-adds themselves
    const int part = threadIdx.x & 7;
    const int rows_per_pass = blockDim.x >> 3;
    for (int r0 = 0; r0 < A.ncr; r0 += rows_per_pass) {
      const int row = r0 + (threadIdx.x >> 3);
      double s = 0.0;
      if (row < A.ncr) {
        const double *a = cinv + (size_t)row * A.ncr;
        if (bd_ok)
          for (int j = part; j < A.ncr; j += 8) s += a[j] * bd[j];
        else
          for (int j = part; j < A.ncr; j += 8) s += a[j] * (double)q.b[j];
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (row < A.ncr && part == 0) {
        int x, y, z;
        cell_xyz<D>(row, q.n, &x, &y, &z);
        q.tile[G.idx(x, y, z)] = T(s);
      }
    }
    __syncthreads();
  }
  for (int l = A.l_lo + 1; l <= top; l++) {
    const TailLevel<T, D> &F = Q[top - l], &Cq = Q[top - l + 1];
    tail_prolong<T, D>(V, F, Cq);
    for (int k = 0; k < F.L.nu; k++) {
      tail_smooth<T, D>(V, F, 0);
      tail_smooth<T, D>(V, F, 1);
    }
  }
  {  // phi of the top tail level back to global memory
    const TailLevel<T, D> &q = Q[0];
    const TileGeo<T, D> G(q.n);
    for (int c = threadIdx.x; c < q.ncell; c += blockDim.x) {
      int x, y, z;
      cell_xyz_rt<D>(c, q.n, &x, &y, &z);
      V.phi[q.L.poff + cs_pos_xyz(x, y, z, q.n, q.ncell)] = q.tile[G.idx(x, y, z)];
    }
  }
}

template <typename T, int D, int NT>
__global__ void __launch_bounds__(kCoopThreads) k_cycle_coop(GmgView<T> V, const LvArgs *lvtab, int nlev, int lmin,
                                                         CycleArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_start();
  __shared__ LevelSet LS;  // level table in shared memory (indexed by level at run time)
  // the units' activity flags, fixed during the launch: read once here, not
  // once per phase before each tile load
  constexpr int kActCache = 256;
  __shared__ int s_act[kActCache];
  const int nunits = V.nrhs * V.ntree;
  const bool act_cached = nunits <= kActCache;
  if (threadIdx.x < nlev) LS.lv[threadIdx.x] = lvtab[threadIdx.x];
  if (threadIdx.x == 0) LS.lmin = lmin;
  if (act_cached)
    for (int i = threadIdx.x; i < nunits; i += blockDim.x) s_act[i] = V.active[i];
  __syncthreads();
  auto is_active = [&](int u) { return act_cached ? s_act[u] != 0 : V.active[u] != 0; };
  const unsigned int G = gridDim.x;
  unsigned int epoch = 0;  // grid barriers passed (thread 0 keeps the count)
#define GMG_LV(l) LS.lv[(l)-LS.lmin]
  // (block, slot) items of level Lv handled by this CTA, slots fastest;
  // frozen slots are skipped (W: the slot's view, bid: the block)
#define GMG_ITEMS(Lv)                                                                          \
  for (int item = blockIdx.x, bid = 0; item < (Lv).count * V.nrhs; item += G)                  \
    if (const int r_ = item % V.nrhs; (bid = (Lv).first + item / V.nrhs, is_active(unit_of(V, r_, bid)))) \
      if (const GmgView<T> W = slot_view(V, r_); true)
  // levels l_hi .. l_one + 1: every CTA, grid barrier between phases
  for (int l = A.l_hi; A.mode != 2 && l > A.l_lo && l > A.l_one; l--) {
    const LvArgs &L = GMG_LV(l), &Lp = GMG_LV(l - 1);  // read from shared memory, not held in registers
    for (int k = 0; k < L.nd; k++)
      for (int c = 0; c < 2; c++) {
        GMG_ITEMS(L) {
          smooth_any<T, D, NT>(W, L, Lp, bid, c, smem_raw);
          __syncthreads();
        }
        if (!grid_sync(A.bar, G, A.spin_limit, &epoch)) return;
      }
    GMG_ITEMS(L) {
      resid_restrict_any<T, D, NT>(W, L, Lp, bid, smem_raw);
      __syncthreads();
    }
    if (!grid_sync(A.bar, G, A.spin_limit, &epoch)) return;
    const LvArgs &Lpp = l - 2 >= LS.lmin ? GMG_LV(l - 2) : Lp;
    GMG_ITEMS(Lp) {
      fas_any<T, D, NT>(W, Lp, Lpp, bid, smem_raw);
      __syncthreads();
    }
    if (A.mode == 1 && l == A.l_one + 1) return;  // the kernel ends: no barrier
    if (!grid_sync(A.bar, G, A.spin_limit, &epoch)) return;
  }
  if (A.mode == 1) return;  // the cluster kernel runs the bottom of the cycle next
  if (A.mode == 2) {
    // up leg only: the bottom levels were done by the cluster kernel
  } else if (A.l_one >= A.l_lo) {
    // single-block levels l_one .. l_lo: CTA 0 runs the bottom of the cycle
    // (sweeps, restriction, FAS, coarse solve, prolongation, sweeps) with
    // block-level barriers only
    for (int item = blockIdx.x; item < A.nroot * V.nrhs; item += G) {
      const int r = item % V.nrhs, root = item / V.nrhs;
      if (is_active(V.ntree > 1 ? r * V.ntree + root : r))
        tail_cycle<T, D>(slot_view(V, r), LS, A, A.l_one < A.l_hi ? A.l_one : A.l_hi, root, smem_raw);
      __syncthreads();
    }
  } else {
    coarse_rows<T>(V, GMG_LV(A.l_lo), A, blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5),
                   (int)(G * (blockDim.x / 32)));
  }
  if (A.mode == 0 && A.l_hi > A.l_one && !grid_sync(A.bar, G, A.spin_limit, &epoch)) return;
  for (int l = (A.l_one >= A.l_lo ? A.l_one : A.l_lo) + 1; l <= A.l_hi; l++) {
    const LvArgs &L = GMG_LV(l), &Lp = GMG_LV(l - 1);  // read from shared memory, not held in registers
    GMG_ITEMS(L) {
      prolong_any<T, D, NT>(W, L, Lp, bid, smem_raw);
      __syncthreads();
    }
    if (!grid_sync(A.bar, G, A.spin_limit, &epoch)) return;
    for (int k = 0; k < L.nu; k++)
      for (int c = 0; c < 2; c++) {
        GMG_ITEMS(L) {
          smooth_any<T, D, NT>(W, L, Lp, bid, c, smem_raw);
          __syncthreads();
        }
        // the last sweep of the range needs no barrier: the kernel ends
        if (!(l == A.l_hi && k == L.nu - 1 && c == 1) && !grid_sync(A.bar, G, A.spin_limit, &epoch)) return;
      }
  }
#undef GMG_ITEMS
#undef GMG_LV
}

// One leg of a level in one cooperative launch: a CTA per (block, slot),
// all resident at once, with a grid barrier between the phases that the
// per-level kernels would run as separate launches.  mode 0, the down leg:
// N_down red/black sweeps, then the residual and its restriction with phi
// (resid_restrict_block).  mode 1, the up leg: the prolongation of the
// coarse correction, then N_up red/black sweeps.  Every phase runs the
// per-level kernels' block functions on the same inputs, so the results are
// theirs bit for bit; a frozen unit's CTAs skip the work and still take
// part in each barrier.  A barrier that runs out records GMG_ERR_TIMEOUT and
// ends the launch.
template <typename T, int D, int NT>
__global__ void __launch_bounds__(kThreads, 4) k_level_leg(GmgView<T> V0, LvArgs L, LvArgs Lp, int mode, GridBar *bar,
                                                           long long spin_limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = (int)(blockIdx.x % (unsigned)V0.nrhs);
  const int bid = L.first + (int)(blockIdx.x / (unsigned)V0.nrhs);
  const bool on = V0.active[unit_of(V0, r, bid)] != 0;
  const GmgView<T> W = slot_view(V0, r);
  const int slot0[1] = {0};
  const unsigned int G = gridDim.x;
  unsigned int epoch = 0;
  if (mode == 1) {
    if (on) prolong_block<T, D, NT>(W, L, Lp, bid, smem_raw);
    if (!grid_sync(bar, G, spin_limit, &epoch)) return;
  }
  const int ns = mode == 0 ? L.nd : L.nu;
  for (int k = 0; k < ns; k++)
    for (int c = 0; c < 2; c++) {
      if (on) smooth_cs_block<T, D, NT, 1>(W, L, Lp, bid, slot0, c, smem_raw);
      // the up leg's last half-sweep needs no barrier: the launch ends
      if (!(mode == 1 && k == ns - 1 && c == 1) && !grid_sync(bar, G, spin_limit, &epoch)) return;
    }
  if (mode == 0 && on) resid_restrict_block<T, D, NT>(W, L, Lp, bid, smem_raw);
}

// A cooperative kernel whose barrier waits for one CTA more than it has:
// the wait must run out and record GMG_ERR_TIMEOUT (failure-detection test).
__global__ void k_barrier_selftest(GridBar *bar, long long spin_limit) {
  unsigned int epoch = 0;
  grid_sync(bar, gridDim.x + 1, spin_limit, &epoch);
}

}  // namespace gmg
