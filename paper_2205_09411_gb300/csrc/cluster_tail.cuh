// The bottom of the V-cycle on a thread-block cluster.
//
// On the levels that hold one block per root (the root block and its
// coarsened copies), and on the level of the root's 2^D children when it is
// complete, the whole domain of one root at level l is a cube of side N_l.
// A cluster of P = 2^D CTAs splits every such level into octants (quadrants
// in 2D): CTA k owns the cells whose coordinates have bit d of k set exactly
// when they lie in the upper half along axis d.  Each CTA keeps its octant of
// every level in shared memory (phi with a one-cell ghost ring, b, old, the
// octant's cut-list entries), and the levels never go to global memory
// between the load of the top level and the store of its phi at the end.
// The sequence is that of the single-CTA tail (Sec. 2.2: N_down red/black
// sweeps, residual + restriction, FAS right-hand side, exact solve on the
// coarsest level, prolongation and N_up sweeps on the way up), with the same
// expressions; ghost cells on an octant face inside the cube are read from
// the neighbouring CTA's shared memory (distributed shared memory), ghost
// cells beyond the cube are wall reflections (reading W).  A cluster barrier
// (release/acquire at cluster scope) separates dependent phases.  A
// half-sweep of colour c reads only cells of colour 1 - c across octant
// faces, which no CTA writes during it.
#pragma once

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace gmg {

namespace cg = cooperative_groups;

// One level of the cube, this CTA's octant.
template <typename T, int D>
struct Oct {
  T *tile;               // (m + 2)^D with the ghost ring, x fastest
  T *b, *old;            // m^D
  unsigned short *eidx;  // m^D: 0 regular stencil, e + 1 entry e of cf
  T *cf;                 // coefficient k of entry e at cf[k * mm + e]
  int N, m, mm;          // side of the cube, side of the octant, entries in cf
  int bid;               // block holding the octant (the root's block, or this CTA's child)
  int o[3];              // first cell of the octant in cube coordinates
  int full;              // 1: the whole cube (m = N, o = 0), computed alike by every CTA of the cluster
  LvArgs L;
};

template <int D>
__device__ __forceinline__ int oct_ti(int m, int x, int y, int z) {
  const int R = m + 2;
  return (x + 1) + R * ((y + 1) + (D == 3 ? R * (z + 1) : 0));
}

template <typename T>
__device__ __forceinline__ T *peer(T *p, int rank) {
  return cg::this_cluster().map_shared_rank(p, rank);
}

__device__ __forceinline__ void cluster_barrier() { cg::this_cluster().sync(); }

template <typename T>
__device__ __forceinline__ T wall_sign(int wneu, int f) {
  return ((wneu >> f) & 1) ? T(1) : T(-1);
}

// Face f = 2 axis + side of the octant: its ghost cell (g), the octant's own
// cell beside it (in), and, across a face inside the cube, the cell of the
// neighbouring octant (rank ^ (1 << axis)) whose ghost ring holds `in` (gn)
// for face cell j (the other axes take j's two coordinates in order).
// Written with selects, not indexed arrays, so that everything stays in
// registers.
template <int D>
__device__ __forceinline__ void face_cells(int m, int f, int j, int *g, int *in, int *gn) {
  const int a = f >> 1, side = f & 1;
  const int u = j % m, v = D == 3 ? j / m : 0;
  const int ag = side ? m : -1, ai = side ? m - 1 : 0, an = side ? -1 : m;
  const int y_other = a == 0 ? u : v, z_other = v;
  g[0] = a == 0 ? ag : u;
  in[0] = a == 0 ? ai : u;
  gn[0] = a == 0 ? an : u;
  g[1] = a == 1 ? ag : y_other;
  in[1] = a == 1 ? ai : y_other;
  gn[1] = a == 1 ? an : y_other;
  g[2] = D == 3 ? (a == 2 ? ag : z_other) : 0;
  in[2] = D == 3 ? (a == 2 ? ai : z_other) : 0;
  gn[2] = D == 3 ? (a == 2 ? an : z_other) : 0;
}

// Does face f of the octant lie on the cube's boundary (a wall)?
template <typename T, int D>
__device__ __forceinline__ bool face_is_wall(const Oct<T, D> &Q, int f) {
  const int a = f >> 1, side = f & 1;
  const int oa = a == 0 ? Q.o[0] : (a == 1 ? Q.o[1] : Q.o[2]);
  return side ? oa + Q.m >= Q.N : oa == 0;
}

// Pushes the octant's cells of colour `color` (-1: every colour) beside the
// faces inside the cube into the neighbouring octants' ghost rings.  The
// stores need no reply; the cluster barrier that follows makes them visible.
template <typename T, int D>
__device__ __forceinline__ void oct_push(const Oct<T, D> &Q, int rank, int color) {
  const int m = Q.m, nf = D == 3 ? m * m : m;
  const int osum = Q.o[0] + Q.o[1] + Q.o[2];
  for (int i = threadIdx.x; i < 2 * D * nf; i += blockDim.x) {
    const int f = i / nf, j = i - f * nf;
    if (face_is_wall(Q, f)) continue;
    int g[3], in[3], gn[3];
    face_cells<D>(m, f, j, g, in, gn);
    if (color >= 0 && ((osum + in[0] + in[1] + in[2]) & 1) != color) continue;
    T *rt = peer(Q.tile, rank ^ (1 << (f >> 1)));
    rt[oct_ti<D>(m, gn[0], gn[1], gn[2])] = Q.tile[oct_ti<D>(m, in[0], in[1], in[2])];
  }
}

// Ghost cells on the faces that are walls of the cube: the wall sign times
// the adjacent cell (reading W), for the kernels that read the whole ring.
template <typename T, int D>
__device__ __forceinline__ void oct_walls(const Oct<T, D> &Q, int wneu) {
  const int m = Q.m, nf = D == 3 ? m * m : m;
  for (int i = threadIdx.x; i < 2 * D * nf; i += blockDim.x) {
    const int f = i / nf, j = i - f * nf;
    if (!face_is_wall(Q, f)) continue;
    int g[3], in[3], gn[3];
    face_cells<D>(m, f, j, g, in, gn);
    Q.tile[oct_ti<D>(m, g[0], g[1], g[2])] = wall_sign<T>(wneu, f) * Q.tile[oct_ti<D>(m, in[0], in[1], in[2])];
  }
}

// The whole ghost ring (faces, edges, corners) of the octant from the cube:
// a position beyond the cube is clamped to the cube on each axis it leaves,
// with the product of the walls' signs (reading P); the value comes from the
// octant that owns the clamped cell.  Each thread issues the reads of up to
// kRingBatch positions before it stores any, so that their latencies overlap.
constexpr int kRingBatch = 4;
template <typename T, int D>
__device__ __forceinline__ void oct_ring(const Oct<T, D> &Q, int wneu) {
  const int m = Q.m, R = m + 2, tot = D == 3 ? R * R * R : R * R;
  for (int base = threadIdx.x; base < tot; base += kRingBatch * blockDim.x) {
    T val[kRingBatch];
    int at[kRingBatch];
#pragma unroll
    for (int u = 0; u < kRingBatch; u++) {
      const int i = base + u * blockDim.x;
      at[u] = -1;
      if (i >= tot) continue;
      const int p[3] = {i % R - 1, (i / R) % R - 1, D == 3 ? i / (R * R) - 1 : 0};
      bool ring = false;
#pragma unroll
      for (int d = 0; d < D; d++) ring = ring || p[d] < 0 || p[d] >= m;
      if (!ring) continue;
      int q[3] = {0, 0, 0}, own = 0;
      T sg = T(1);
#pragma unroll
      for (int d = 0; d < D; d++) {
        int P = Q.o[d] + p[d];
        if (P < 0) {
          P = 0;
          sg *= wall_sign<T>(wneu, 2 * d);
        } else if (P >= Q.N) {
          P = Q.N - 1;
          sg *= wall_sign<T>(wneu, 2 * d + 1);
        }
        const int hi = P >= Q.m ? 1 : 0;
        own |= hi << d;
        q[d] = P - hi * Q.m;
      }
      const T *src = Q.full ? Q.tile : peer(Q.tile, own);
      val[u] = sg * src[oct_ti<D>(m, q[0], q[1], q[2])];
      at[u] = i;
    }
#pragma unroll
    for (int u = 0; u < kRingBatch; u++)
      if (at[u] >= 0) Q.tile[at[u]] = val[u];
  }
}

template <typename T, int D>
__device__ __forceinline__ bool oct_cut(const Oct<T, D> &Q, int c, int *e) {
  if (Q.mm == 0) return false;
  *e = (int)Q.eidx[c] - 1;
  return *e >= 0;
}

// One half-sweep of colour `color` (global cube parity) on the octant.
// Across a face inside the cube the neighbour comes from the ghost ring
// (pushed after the neighbouring octant's last update of that colour);
// across a wall it is the wall sign times the cell itself (reading W).
template <typename T, int D>
__device__ __forceinline__ void oct_smooth(const Oct<T, D> &Q, int color, int wneu) {
  const int m = Q.m, R = m + 2, sz = R * R;
  const T h2 = T(Q.L.h2), inv2d = T(1.0 / (2 * D));
  const int lc = (color + Q.o[0] + Q.o[1] + Q.o[2]) & 1;  // colour in octant coordinates
  const int nc = D == 3 ? m * m * m : m * m;
  int wl = 0;  // bit f: face f is a wall of the cube
#pragma unroll
  for (int f = 0; f < 2 * D; f++) wl |= face_is_wall(Q, f) ? 1 << f : 0;
  for (int j = threadIdx.x; j < nc / 2; j += blockDim.x) {
    int x, y, z;
    colour_xyz<D>(j, m, lc, &x, &y, &z);
    const int c = x + m * (y + m * z);
    const int t = oct_ti<D>(m, x, y, z);
    const T own = Q.tile[t];
    // a wall ghost is +-own: the sign is exact, so a negation replaces the product
    const int at = (x == 0 ? 1 : 0) | (x == m - 1 ? 2 : 0) | (y == 0 ? 4 : 0) | (y == m - 1 ? 8 : 0) |
                   (D == 3 && z == 0 ? 16 : 0) | (D == 3 && z == m - 1 ? 32 : 0);
    const int w = at & wl;
    T xm = Q.tile[t - 1], xp = Q.tile[t + 1], ym = Q.tile[t - R], yp = Q.tile[t + R];
    T zm = T(0), zp = T(0);
    if (D == 3) {
      zm = Q.tile[t - sz];
      zp = Q.tile[t + sz];
    }
    if (w) {
      if (w & 1) xm = ((wneu >> 0) & 1) ? own : -own;
      if (w & 2) xp = ((wneu >> 1) & 1) ? own : -own;
      if (w & 4) ym = ((wneu >> 2) & 1) ? own : -own;
      if (w & 8) yp = ((wneu >> 3) & 1) ? own : -own;
      if (D == 3 && (w & 16)) zm = ((wneu >> 4) & 1) ? own : -own;
      if (D == 3 && (w & 32)) zp = ((wneu >> 5) & 1) ? own : -own;
    }
    T nv;
    int e;
    if (!oct_cut(Q, c, &e)) {
      T sum = (xm + xp) + (ym + yp);
      if (D == 3) sum += zm + zp;
      nv = (sum - h2 * Q.b[c]) * inv2d;
    } else {
      T a[2 * D + 1];
#pragma unroll
      for (int k = 0; k < 2 * D + 1; k++) a[k] = Q.cf[k * Q.mm + e];
      T sum = a[1] * xm + a[2] * xp + a[3] * ym + a[4] * yp;
      if (D == 3) sum += a[5] * zm + a[6] * zp;
      nv = (Q.b[c] - sum) / a[0];
    }
    Q.tile[t] = nv;
  }
}

// Residual of F restricted into C: phi_C <- mean phi_F, b_C <- mean r_F
// (the children of a coarse cell of this octant lie in this octant).  F's
// ghost ring must be current.  When C is a full level and F is split, the
// coarse cells go to the octant's place in C, in this CTA's copy and in
// every other CTA's (rank: this CTA), so that each CTA holds all of C.
template <typename T, int D>
__device__ __forceinline__ void oct_resid_restrict(const Oct<T, D> &F, const Oct<T, D> &C, int rank) {
  constexpr int P = 1 << D;
  const int m = F.m, R = m + 2, sz = R * R, hm = m / 2;
  const T inv_h2 = T(F.L.ih2), w = T(1.0 / (1 << D));
  const int nc = D == 3 ? hm * hm * hm : hm * hm;
  const bool bcast = C.full && !F.full;
  const int co[3] = {bcast ? F.o[0] / 2 : 0, bcast ? F.o[1] / 2 : 0, bcast ? F.o[2] / 2 : 0};
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    int qx, qy, qz;
    cell_xyz_rt<D>(j, hm, &qx, &qy, &qz);
    T sp = T(0), sr = T(0);
#pragma unroll
    for (int dz = 0; dz < (D == 3 ? 2 : 1); dz++)
#pragma unroll
      for (int dy = 0; dy < 2; dy++)
#pragma unroll
        for (int dx = 0; dx < 2; dx++) {
          const int x = 2 * qx + dx, y = 2 * qy + dy, z = 2 * qz + dz;
          const int c = x + m * (y + m * z);
          const int t = oct_ti<D>(m, x, y, z);
          sp = sp + F.tile[t];
          int e;
          const bool cut = oct_cut(F, c, &e);
          sr = sr + resid_cell<T, D>(F.cf, cut ? 0 : -1, F.tile, t, R, sz, F.mm, e, inv_h2, F.b[c]);
        }
    const int X = co[0] + qx, Y = co[1] + qy, Z = co[2] + qz;
    const int ti = oct_ti<D>(C.m, X, Y, Z), ci = X + C.m * (Y + C.m * Z);
    C.tile[ti] = sp * w;
    C.b[ci] = sr * w;
    if (bcast)
#pragma unroll
      for (int k = 1; k < P; k++) {
        const int rk = rank ^ k;
        peer(C.tile, rk)[ti] = sp * w;
        peer(C.b, rk)[ci] = sr * w;
      }
  }
}

// FAS right-hand side b <- A phi + b, old <- phi (face ghosts filled).
template <typename T, int D>
__device__ __forceinline__ void oct_fas(const Oct<T, D> &Q) {
  const int m = Q.m, R = m + 2, sz = R * R;
  const T inv_h2 = T(Q.L.ih2);
  const int nc = D == 3 ? m * m * m : m * m;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    int x, y, z;
    cell_xyz_rt<D>(c, m, &x, &y, &z);
    const int t = oct_ti<D>(m, x, y, z);
    const T ph = Q.tile[t];
    T ap;
    int e;
    if (!oct_cut(Q, c, &e)) {
      ap = inv_h2 * (nb_sum<T, D>(Q.tile, t, R, sz) - T(2 * D) * ph);
    } else {
      T diag;
      const T sum = offdiag_st<T, D>(Q.cf, Q.tile, t, R, sz, Q.mm, e, &diag);
      ap = diag * ph + sum;
    }
    Q.b[c] = ap + Q.b[c];
    Q.old[c] = ph;
  }
}

// phi_F += trilinear prolongation of C's correction (C's tile holds the
// correction with its whole ghost ring).
template <typename T, int D>
__device__ __forceinline__ void oct_prolong(const Oct<T, D> &F, const Oct<T, D> &C) {
  const int m = F.m, cm = C.m;
  // a full C holds the whole cube: F's octant sits at F.o / 2 in it
  const bool off = C.full && !F.full;
  const int cofs[3] = {off ? F.o[0] / 2 : 0, off ? F.o[1] / 2 : 0, off ? F.o[2] / 2 : 0};
  const int nc = D == 3 ? m * m * m : m * m;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    int x, y, z;
    cell_xyz_rt<D>(c, m, &x, &y, &z);
    const int u[3] = {cofs[0] + (x >> 1), cofs[1] + (y >> 1), cofs[2] + (z >> 1)};
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
          v = v + wgt * C.tile[oct_ti<D>(cm, u[0] + sx * o[0], u[1] + sy * o[1], D == 3 ? u[2] + sz * o[2] : 0)];
        }
    F.tile[oct_ti<D>(m, x, y, z)] += v;
  }
}

// global-memory index of octant cell (x, y, z) of level Q (b / old fields;
// phi adds L.poff - L.off)
template <typename T, int D>
__device__ __forceinline__ long long oct_gidx(const Oct<T, D> &Q, int children, int x, int y, int z) {
  const long long base = Q.L.off + (long long)(Q.bid - Q.L.first) * Q.L.ncell;
  if (children) return base + cs_pos_xyz(x, y, D == 3 ? z : 0, Q.m, Q.L.ncell);
  return base + cs_pos_xyz(Q.o[0] + x, Q.o[1] + y, D == 3 ? Q.o[2] + z : 0, Q.N, Q.L.ncell);
}

template <typename T, int D>
__global__ void __launch_bounds__(kClusterThreads, 1) k_cycle_cluster(GmgView<T> V0, const LvArgs *lvtab, int lmin,
                                                                       ClusterArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int P = 1 << D;
  pdl_start();
  const int rank = (int)(blockIdx.x % P);
  const int item = (int)(blockIdx.x / P);
  const int r = item % V0.nrhs, root = item / V0.nrhs;
  // the whole cluster takes the same exit: the unit's flag is one word
  if (!V0.active[V0.ntree > 1 ? r * V0.ntree + root : r]) return;
  const GmgView<T> V = slot_view(V0, r);
  const int ntl = A.l_top - A.l_lo + 1;
  __shared__ Oct<T, D> Qs[kClusterMaxLevels];
  __shared__ int s_e0[kClusterMaxLevels], s_ecum[kClusterMaxLevels + 1];
  if (threadIdx.x < ntl) {
    const int i = threadIdx.x, l = A.l_top - i;
    Oct<T, D> q;
    q.L = lvtab[l - lmin];
    const bool ch = A.children && i == 0;
    q.N = ch ? 2 * q.L.n : q.L.n;
    q.full = i >= A.full_from ? 1 : 0;
    q.m = q.full ? q.N : q.N / 2;
#pragma unroll
    for (int d = 0; d < 3; d++) q.o[d] = (d < D && !q.full) ? ((rank >> d) & 1) * q.m : 0;
    q.bid = q.L.first + (ch ? P * root + rank : root);
    q.tile = reinterpret_cast<T *>(smem_raw + A.off_tile[i]);
    q.b = reinterpret_cast<T *>(smem_raw + A.off_b[i]);
    q.old = reinterpret_cast<T *>(smem_raw + A.off_old[i]);
    q.eidx = reinterpret_cast<unsigned short *>(smem_raw + A.off_eidx[i]);
    q.cf = reinterpret_cast<T *>(smem_raw + A.off_cf[i]);
    const int4 cl = V.cut_list[q.bid];
    q.mm = cl.y + cl.z;
    s_e0[i] = cl.x;
    Qs[i] = q;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // running totals of the levels' entries (one flat loop below)
    s_ecum[0] = 0;
    for (int i = 0; i < ntl; i++) s_ecum[i + 1] = s_ecum[i] + Qs[i].mm;
  }
  {  // phi and b of the top level's octant, in flight during the set-up
    const Oct<T, D> &q = Qs[0];
    const int m = q.m, nc = D == 3 ? m * m * m : m * m;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      int x, y, z;
      cell_xyz_rt<D>(c, m, &x, &y, &z);
      const long long g = oct_gidx(q, A.children, x, y, z);
      cp_async_elem(q.tile + oct_ti<D>(m, x, y, z), V.phi + (q.L.poff - q.L.off) + g);
      cp_async_elem(q.b + c, V.b + g);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  // this CTA's rows of the coarse inverse (its octant's cells of l_lo)
  const Oct<T, D> Qlo = Qs[ntl - 1];
  const double *cinv = A.cinv + (size_t)root * A.ncr * A.ncr;
  // rows of the coarse solve this CTA computes: its octant's cells, or on a
  // full coarsest level the cells rank, rank + P, ...
  const int nlo = Qlo.full ? (A.ncr - rank + P - 1) / P : (D == 3 ? Qlo.m * Qlo.m * Qlo.m : Qlo.m * Qlo.m);
  auto row_of = [&](int c) {
    if (Qlo.full) return rank + P * c;
    int x, y, z;
    cell_xyz_rt<D>(c, Qlo.m, &x, &y, &z);
    return (Qlo.o[0] + x) + Qlo.N * ((Qlo.o[1] + y) + (D == 3 ? Qlo.N * (Qlo.o[2] + z) : 0));
  };
  if (A.stage_rows) {
    double *rows = reinterpret_cast<double *>(smem_raw + A.off_rows);
    for (int i = threadIdx.x; i < nlo * A.ncr; i += blockDim.x) {
      const int c = i / A.ncr, j = i - c * A.ncr;
      cp_async_elem(rows + i, cinv + (size_t)row_of(c) * A.ncr + j);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  // cut lists: per cell of the octant its entry, and the blocks' coefficients
  for (int i = 0; i < ntl; i++) {
    const Oct<T, D> &q = Qs[i];
    if (!q.mm) continue;
    const int nc = D == 3 ? q.m * q.m * q.m : q.m * q.m;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) q.eidx[c] = 0;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < s_ecum[ntl]; k += blockDim.x) {  // every entry of every level
    int i = 0;
    while (k >= s_ecum[i + 1]) i++;
    const Oct<T, D> &q = Qs[i];
    const int e = k - s_ecum[i], ge = s_e0[i] + e;
    const int c = V.cut_cell[ge];
    T cf[2 * D + 1];
#pragma unroll
    for (int kk = 0; kk < 2 * D + 1; kk++) cf[kk] = V.cut_coef[kk * V.n_cut + ge];
#pragma unroll
    for (int kk = 0; kk < 2 * D + 1; kk++) q.cf[kk * q.mm + e] = cf[kk];
    if (A.children && i == 0) {
      q.eidx[c] = (unsigned short)(e + 1);
    } else {  // a cell of the root's block: this octant's?
      int X, Y, Z;
      cell_xyz_rt<D>(c, q.N, &X, &Y, &Z);
      const int x = X - q.o[0], y = Y - q.o[1], z = Z - q.o[2];
      if (x >= 0 && x < q.m && y >= 0 && y < q.m && (D == 2 || (z >= 0 && z < q.m)))
        q.eidx[x + q.m * (y + q.m * z)] = (unsigned short)(e + 1);
    }
  }
  if (A.stage_rows)
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  else
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  // every CTA of the cluster is running and its top level is in place
  cluster_barrier();
  const int wneu = V.wneu;
  oct_push<T, D>(Qs[0], rank, -1);  // the top level's ghosts across the octant faces
  cluster_barrier();
  for (int i = 0; i + 1 < ntl; i++) {
    const Oct<T, D> F = Qs[i], C = Qs[i + 1];
    // each half-sweep of a split level pushes the cells it updated that
    // border another octant; the ring then holds both colours' current
    // values.  A full level needs no exchange: CTA barriers only.
    for (int k = 0; k < F.L.nd; k++)
      for (int col = 0; col < 2; col++) {
        oct_smooth<T, D>(F, col, wneu);
        __syncthreads();
        if (!F.full) {
          oct_push<T, D>(F, rank, col);
          cluster_barrier();
        }
      }
    oct_walls<T, D>(F, wneu);
    __syncthreads();
    oct_resid_restrict<T, D>(F, C, rank);
    __syncthreads();
    if (!C.full) {
      oct_push<T, D>(C, rank, -1);
      cluster_barrier();
    } else if (!F.full) {
      cluster_barrier();  // every octant's share of C has arrived
    }
    oct_walls<T, D>(C, wneu);
    __syncthreads();
    oct_fas<T, D>(C);
    __syncthreads();
  }
  {  // exact solve on l_lo: b in FP64, then this CTA's rows
    if (A.stage_rows) asm volatile("cp.async.wait_all;\n" ::: "memory");
    const Oct<T, D> &q = Qs[ntl - 1];
    double *bd = reinterpret_cast<double *>(smem_raw + A.off_bd);
    // every CTA is past its FAS of l_lo: its tile may be written and b read
    cluster_barrier();
    if (q.full) {
      for (int j = threadIdx.x; j < A.ncr; j += blockDim.x) bd[j] = (double)q.b[j];
    } else {
      for (int j = threadIdx.x; j < A.ncr; j += blockDim.x) {
        int X, Y, Z;
        cell_xyz_rt<D>(j, q.N, &X, &Y, &Z);
        const int own = (X >= q.m ? 1 : 0) | (Y >= q.m ? 2 : 0) | (D == 3 && Z >= q.m ? 4 : 0);
        const int x = X - (own & 1 ? q.m : 0), y = Y - (own & 2 ? q.m : 0), z = D == 3 ? Z - (own & 4 ? q.m : 0) : 0;
        bd[j] = (double)peer(q.b, own)[x + q.m * (y + q.m * z)];
      }
    }
    __syncthreads();
    const double *rows = reinterpret_cast<const double *>(smem_raw + A.off_rows);
    const int part = threadIdx.x & 7;
    const int rows_per_pass = blockDim.x >> 3;
    for (int r0 = 0; r0 < nlo; r0 += rows_per_pass) {
      const int c = r0 + (threadIdx.x >> 3);
      double s = 0.0;
      const int row = c < nlo ? row_of(c) : 0;
      if (c < nlo) {
        const double *a = A.stage_rows ? rows + (size_t)c * A.ncr : cinv + (size_t)row * A.ncr;
        for (int j = part; j < A.ncr; j += 8) s += a[j] * bd[j];
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (c < nlo && part == 0) {
        int X, Y, Z;
        cell_xyz_rt<D>(row, q.N, &X, &Y, &Z);
        const int ti = oct_ti<D>(q.m, X - q.o[0], Y - q.o[1], Z - q.o[2]);
        q.tile[ti] = T(s);
        if (q.full)  // every CTA holds the whole level
#pragma unroll
          for (int k = 1; k < P; k++) peer(q.tile, rank ^ k)[ti] = T(s);
      }
    }
    if (q.full)
      cluster_barrier();
    else
      __syncthreads();
  }
  for (int i = ntl - 2; i >= 0; i--) {
    const Oct<T, D> F = Qs[i], C = Qs[i + 1];
    // the correction phi - old of C in place (the level is dead afterwards)
    {
      const int nc = D == 3 ? C.m * C.m * C.m : C.m * C.m;
      for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        int x, y, z;
        cell_xyz_rt<D>(c, C.m, &x, &y, &z);
        const int t = oct_ti<D>(C.m, x, y, z);
        C.tile[t] = C.tile[t] - C.old[c];
      }
    }
    if (C.full)
      __syncthreads();
    else
      cluster_barrier();
    oct_ring<T, D>(C, wneu);
    __syncthreads();
    oct_prolong<T, D>(F, C);
    __syncthreads();
    if (!F.full) {
      oct_push<T, D>(F, rank, -1);
      cluster_barrier();
    }
    for (int k = 0; k < F.L.nu; k++)
      for (int col = 0; col < 2; col++) {
        oct_smooth<T, D>(F, col, wneu);
        __syncthreads();
        if (!F.full) {
          oct_push<T, D>(F, rank, col);
          cluster_barrier();
        }
      }
  }
  {  // phi of the top level's octant back to global memory
    const Oct<T, D> &q = Qs[0];
    const int m = q.m, nc = D == 3 ? m * m * m : m * m;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      int x, y, z;
      cell_xyz_rt<D>(c, m, &x, &y, &z);
      V.phi[(q.L.poff - q.L.off) + oct_gidx(q, A.children, x, y, z)] = q.tile[oct_ti<D>(m, x, y, z)];
    }
  }
}

}  // namespace gmg
