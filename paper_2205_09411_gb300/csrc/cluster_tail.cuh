// The bottom of the V-cycle on a thread-block cluster.
//
// On the levels that hold one block per root (the root block and its
// coarsened copies), and on the level of the root's 2^D children when it is
// complete, the whole domain of one root at level l is a cube of side N_l.
// A cluster of P CTAs splits every such level into equal parts: halves along
// x and y, and halves or quarters along z in 3D (P = 4 in 2D, 8 or 16 in
// 3D).  CTA k = kx + 2 ky + 4 kz owns part (kx, ky, kz).  Each CTA keeps its
// part of every level in shared memory (phi with a one-cell ghost ring, b,
// old, the part's cut-list entries), and the levels never go to global
// memory between the load of the top level and the store of its phi at the
// end.  The sequence is that of the single-CTA tail (Sec. 2.2: N_down
// red/black sweeps, residual + restriction, FAS right-hand side, exact
// solve on the coarsest level, prolongation and N_up sweeps on the way up),
// with the same expressions.  After a half-sweep a CTA pushes the cells it
// changed that border another part into that part's ghost ring (stores to
// distributed shared memory); ghost cells beyond the cube are wall
// reflections (reading W).  A cluster barrier (release/acquire at cluster
// scope) separates dependent phases.  A half-sweep of colour c reads only
// cells of colour 1 - c across part faces, which no CTA writes during it.
// Levels of at most 8 cells a side are held whole by every CTA (`full`) and
// computed by all of them alike, with CTA barriers only.
#pragma once

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace gmg {

namespace cg = cooperative_groups;

// One level of the cube, this CTA's part.
template <typename T, int D>
struct Oct {
  T *tile;               // (m0 + 2)(m1 + 2)(m2 + 2) with the ghost ring, x fastest
  T *b, *old;            // m0 m1 m2
  unsigned short *eidx;  // m0 m1 m2: 0 regular stencil, e + 1 entry e of cf
  T *cf;                 // coefficient k of entry e at cf[k * mm + e]
  int N, mm;             // side of the cube, entries in cf
  int m[3];              // sides of the part (m[2] = 1 in 2D)
  int lg[3];             // log2 m[a] when every side is a power of two, else lg[0] = -1
  int o[3];              // first cell of the part in cube coordinates
  int bid;               // block holding the part (the root's block, or a child)
  int nblk;              // side of that block (N, or N / 2 for the children level)
  int full;              // 1: the whole cube (m = N, o = 0), computed alike by every CTA of the cluster
  LvArgs L;
};

template <typename T, int D>
__device__ __forceinline__ int oct_ti(const Oct<T, D> &Q, int x, int y, int z) {
  return (x + 1) + (Q.m[0] + 2) * ((y + 1) + (D == 3 ? (Q.m[1] + 2) * (z + 1) : 0));
}
template <typename T, int D>
__device__ __forceinline__ int oct_cells(const Oct<T, D> &Q) {
  return Q.m[0] * Q.m[1] * (D == 3 ? Q.m[2] : 1);
}
// (x, y, z) of cell c of the part (x fastest)
template <typename T, int D>
__device__ __forceinline__ void oct_xyz(const Oct<T, D> &Q, int c, int *x, int *y, int *z) {
  if (Q.lg[0] >= 0) {
    *x = c & (Q.m[0] - 1);
    const int r = c >> Q.lg[0];
    *y = r & (Q.m[1] - 1);
    *z = D == 3 ? r >> Q.lg[1] : 0;
  } else {
    *x = c % Q.m[0];
    const int r = c / Q.m[0];
    *y = r % Q.m[1];
    *z = D == 3 ? r / Q.m[1] : 0;
  }
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

// the part's side and origin along axis a (selects, so that nothing needs
// an indexed array in local memory)
template <typename T, int D>
__device__ __forceinline__ int oct_m(const Oct<T, D> &Q, int a) {
  return a == 0 ? Q.m[0] : (a == 1 ? Q.m[1] : Q.m[2]);
}
template <typename T, int D>
__device__ __forceinline__ int oct_o(const Oct<T, D> &Q, int a) {
  return a == 0 ? Q.o[0] : (a == 1 ? Q.o[1] : Q.o[2]);
}

// cells on face f = 2 axis + side of the part
template <typename T, int D>
__device__ __forceinline__ int oct_nf(const Oct<T, D> &Q, int f) {
  const int a = f >> 1;
  return D == 2 ? (a == 0 ? Q.m[1] : Q.m[0]) : (a == 0 ? Q.m[1] * Q.m[2] : (a == 1 ? Q.m[0] * Q.m[2] : Q.m[0] * Q.m[1]));
}

// Face f of the part: its ghost cell (g), the part's own cell beside it
// (in), and, across a face inside the cube, the cell of the neighbouring
// part whose ghost ring holds `in` (gn), for face cell j (the other axes
// take j's two coordinates in order).
template <typename T, int D>
__device__ __forceinline__ void face_cells(const Oct<T, D> &Q, int f, int j, int *g, int *in, int *gn) {
  const int a = f >> 1, side = f & 1;
  const int ma = oct_m(Q, a);
  const int mt0 = a == 0 ? Q.m[1] : Q.m[0];
  const int u = j % mt0, v = D == 3 ? j / mt0 : 0;
  const int ag = side ? ma : -1, ai = side ? ma - 1 : 0, an = side ? -1 : ma;
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

// Does face f of the part lie on the cube's boundary (a wall)?
template <typename T, int D>
__device__ __forceinline__ bool face_is_wall(const Oct<T, D> &Q, int f) {
  const int a = f >> 1, side = f & 1;
  const int oa = oct_o(Q, a);
  return side ? oa + oct_m(Q, a) >= Q.N : oa == 0;
}

// the CTA that owns the part across face f (inside the cube)
__device__ __forceinline__ int face_rank(int rank, int f) {
  const int a = f >> 1, side = f & 1;
  return a == 0 ? rank ^ 1 : (a == 1 ? rank ^ 2 : (side ? rank + 4 : rank - 4));
}

// Pushes the part's cells of colour `color` (-1: every colour) beside the
// faces inside the cube into the neighbouring parts' ghost rings.  The
// stores need no reply; the cluster barrier that follows makes them visible.
template <typename T, int D>
__device__ __forceinline__ void oct_push(const Oct<T, D> &Q, int rank, int color) {
  const int osum = Q.o[0] + Q.o[1] + Q.o[2];
#pragma unroll
  for (int f = 0; f < 2 * D; f++) {
    if (face_is_wall(Q, f)) continue;
    T *rt = peer(Q.tile, face_rank(rank, f));
    const int nf = oct_nf(Q, f);
    for (int j = threadIdx.x; j < nf; j += blockDim.x) {
      int g[3], in[3], gn[3];
      face_cells(Q, f, j, g, in, gn);
      if (color >= 0 && ((osum + in[0] + in[1] + in[2]) & 1) != color) continue;
      rt[oct_ti(Q, gn[0], gn[1], gn[2])] = Q.tile[oct_ti(Q, in[0], in[1], in[2])];
    }
  }
}

// Ghost cells on the faces that are walls of the cube: the wall sign times
// the adjacent cell (reading W), for the kernels that read the whole ring.
template <typename T, int D>
__device__ __forceinline__ void oct_walls(const Oct<T, D> &Q, int wneu) {
#pragma unroll
  for (int f = 0; f < 2 * D; f++) {
    if (!face_is_wall(Q, f)) continue;
    const int nf = oct_nf(Q, f);
    const T sg = wall_sign<T>(wneu, f);
    for (int j = threadIdx.x; j < nf; j += blockDim.x) {
      int g[3], in[3], gn[3];
      face_cells(Q, f, j, g, in, gn);
      Q.tile[oct_ti(Q, g[0], g[1], g[2])] = sg * Q.tile[oct_ti(Q, in[0], in[1], in[2])];
    }
  }
}

// The whole ghost ring (faces, edges, corners) of the part from the cube: a
// position beyond the cube is clamped to the cube on each axis it leaves,
// with the product of the walls' signs (reading P); the value comes from the
// part that owns the clamped cell.  Each thread issues the reads of up to
// kRingBatch positions before it stores any, so that their latencies overlap.
constexpr int kRingBatch = 4;
template <typename T, int D>
__device__ __forceinline__ void oct_ring(const Oct<T, D> &Q, int wneu) {
  const int R0 = Q.m[0] + 2, R1 = Q.m[1] + 2, tot = R0 * R1 * (D == 3 ? Q.m[2] + 2 : 1);
  for (int base = threadIdx.x; base < tot; base += kRingBatch * blockDim.x) {
    T val[kRingBatch];
    int at[kRingBatch];
#pragma unroll
    for (int u = 0; u < kRingBatch; u++) {
      const int i = base + u * blockDim.x;
      at[u] = -1;
      if (i >= tot) continue;
      const int p[3] = {i % R0 - 1, (i / R0) % R1 - 1, D == 3 ? i / (R0 * R1) - 1 : 0};
      bool ring = false;
#pragma unroll
      for (int d = 0; d < D; d++) ring = ring || p[d] < 0 || p[d] >= Q.m[d];
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
        const int k = P / Q.m[d];  // the owning part along axis d
        own += k << d;             // kx + 2 ky + 4 kz
        q[d] = P - k * Q.m[d];
      }
      const T *src = Q.full ? Q.tile : peer(Q.tile, own);
      val[u] = sg * src[oct_ti(Q, q[0], q[1], q[2])];
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

// One half-sweep of colour `color` (global cube parity) on the part.
// Across a face inside the cube the neighbour comes from the ghost ring
// (pushed after the neighbouring part's last update of that colour); across
// a wall it is the wall sign times the cell itself (reading W).
template <typename T, int D>
__device__ __forceinline__ void oct_smooth(const Oct<T, D> &Q, int color, int wneu) {
  const int m0 = Q.m[0], m1 = Q.m[1], m2 = D == 3 ? Q.m[2] : 1;
  const int R = m0 + 2, sz = R * (m1 + 2), hx = m0 / 2;
  const T h2 = T(Q.L.h2), inv2d = T(1.0 / (2 * D));
  const int lc = (color + Q.o[0] + Q.o[1] + Q.o[2]) & 1;  // colour in part coordinates
  const int nc = m0 * m1 * m2;
  int wl = 0;  // bit f: face f is a wall of the cube
#pragma unroll
  for (int f = 0; f < 2 * D; f++) wl |= face_is_wall(Q, f) ? 1 << f : 0;
  const bool p2 = Q.lg[0] >= 1;
  for (int j = threadIdx.x; j < nc / 2; j += blockDim.x) {
    const int rest = p2 ? j >> (Q.lg[0] - 1) : j / hx;
    const int y = p2 ? rest & (m1 - 1) : rest % m1;
    const int z = D == 3 ? (p2 ? rest >> Q.lg[1] : rest / m1) : 0;
    const int x = 2 * (j - rest * hx) + ((y + z + lc) & 1);
    const int c = x + m0 * (y + m1 * z);
    const int t = oct_ti(Q, x, y, z);
    const T own = Q.tile[t];
    // a wall ghost is +-own: the sign is exact, so a negation replaces the product
    const int at = (x == 0 ? 1 : 0) | (x == m0 - 1 ? 2 : 0) | (y == 0 ? 4 : 0) | (y == m1 - 1 ? 8 : 0) |
                   (D == 3 && z == 0 ? 16 : 0) | (D == 3 && z == m2 - 1 ? 32 : 0);
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
// (the children of a coarse cell of this part lie in this part).  F's ghost
// ring must be current.  FP32: one thread per fine cell, the 2^D children
// of a coarse cell on 2^D consecutive lanes (child d = dx + 2 dy + 4 dz),
// the group's first lane summing them in the order of d, as the block
// kernels do (FP64: one thread per coarse cell, the same order).  When C is a full level and F is split, the coarse cells go to the
// part's place in C, in this CTA's copy and in every other CTA's (P CTAs,
// rank: this CTA; the group's lanes share the remote stores), so that each
// CTA holds all of C.
template <typename T, int D>
__device__ __forceinline__ void oct_resid_restrict(const Oct<T, D> &F, const Oct<T, D> &C, int rank, int P) {
  constexpr int G = 1 << D;
  const int m0 = F.m[0], m1 = F.m[1];
  const int R = m0 + 2, sz = R * (m1 + 2);
  const int h0 = m0 / 2, h1 = m1 / 2, h2 = D == 3 ? F.m[2] / 2 : 1;
  const T inv_h2 = T(F.L.ih2), w = T(1.0 / (1 << D));
  const int nc = h0 * h1 * h2;
  const bool bcast = C.full && !F.full;
  const int co[3] = {bcast ? F.o[0] / 2 : 0, bcast ? F.o[1] / 2 : 0, bcast ? F.o[2] / 2 : 0};
  const bool p2 = F.lg[0] >= 1;
  if constexpr (sizeof(T) == 8) {
    // FP64: one thread per coarse cell.  A warp's FP64 instruction costs the
    // pipe the same however few of its lanes are on, so summing on one lane
    // of eight would multiply the adds' cost by eight.
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
      const int r = p2 ? j >> (F.lg[0] - 1) : j / h0;
      const int qx = j - r * h0;
      const int qy = p2 ? r & (h1 - 1) : r % h1;
      const int qz = D == 3 ? (p2 ? r >> (F.lg[1] - 1) : r / h1) : 0;
      T sp = T(0), sr = T(0);
#pragma unroll
      for (int d = 0; d < G; d++) {
        const int x = 2 * qx + (d & 1), y = 2 * qy + ((d >> 1) & 1), z = 2 * qz + (D == 3 ? d >> 2 : 0);
        const int c = x + m0 * (y + m1 * z);
        const int t = oct_ti(F, x, y, z);
        sp = sp + F.tile[t];
        int e;
        const bool cut = oct_cut(F, c, &e);
        sr = sr + resid_cell<T, D>(F.cf, cut ? 0 : -1, F.tile, t, R, sz, F.mm, e, inv_h2, F.b[c]);
      }
      const int X = co[0] + qx, Y = co[1] + qy, Z = co[2] + qz;
      const int ti = oct_ti(C, X, Y, Z), ci = X + C.m[0] * (Y + C.m[1] * Z);
      C.tile[ti] = sp * w;
      C.b[ci] = sr * w;
      if (bcast)
        for (int k = 1; k < P; k++) {
          const int rk = rank ^ k;
          peer(C.tile, rk)[ti] = sp * w;
          peer(C.b, rk)[ci] = sr * w;
        }
    }
    return;
  }
  const int lane = threadIdx.x & 31, d = lane & (G - 1), lead = lane & ~(G - 1);
  const int dx = d & 1, dy = (d >> 1) & 1, dz = D == 3 ? d >> 2 : 0;
  for (int base = 0; base < nc * G; base += blockDim.x) {  // the same trip count in every thread
    const int i = base + (int)threadIdx.x;
    const bool on = i < nc * G;
    const int j = on ? i >> D : 0;
    const int r = p2 ? j >> (F.lg[0] - 1) : j / h0;
    const int qx = j - r * h0;
    const int qy = p2 ? r & (h1 - 1) : r % h1;
    const int qz = D == 3 ? (p2 ? r >> (F.lg[1] - 1) : r / h1) : 0;
    T vp = T(0), vr = T(0);
    if (on) {
      const int x = 2 * qx + dx, y = 2 * qy + dy, z = 2 * qz + dz;
      const int c = x + m0 * (y + m1 * z);
      const int t = oct_ti(F, x, y, z);
      vp = F.tile[t];
      int e;
      const bool cut = oct_cut(F, c, &e);
      vr = resid_cell<T, D>(F.cf, cut ? 0 : -1, F.tile, t, R, sz, F.mm, e, inv_h2, F.b[c]);
    }
    // the group's first lane sums, then hands the means back to the group
    T sp = T(0), sr = T(0);
#pragma unroll
    for (int k = 0; k < G; k++) {
      const T tp = __shfl_sync(0xffffffffu, vp, lead + k), tr = __shfl_sync(0xffffffffu, vr, lead + k);
      if (d == 0) {
        sp = sp + tp;
        sr = sr + tr;
      }
    }
    const T cpv = __shfl_sync(0xffffffffu, sp * w, lead), crv = __shfl_sync(0xffffffffu, sr * w, lead);
    if (!on) continue;
    const int X = co[0] + qx, Y = co[1] + qy, Z = co[2] + qz;
    const int ti = oct_ti(C, X, Y, Z), ci = X + C.m[0] * (Y + C.m[1] * Z);
    if (d == 0) {
      C.tile[ti] = cpv;
      C.b[ci] = crv;
    }
    if (bcast)
      for (int k = 1 + d; k < P; k += G) {
        const int rk = rank ^ k;
        peer(C.tile, rk)[ti] = cpv;
        peer(C.b, rk)[ci] = crv;
      }
  }
}

// FAS right-hand side b <- A phi + b, old <- phi (face ghosts filled).
template <typename T, int D>
__device__ __forceinline__ void oct_fas(const Oct<T, D> &Q) {
  const int R = Q.m[0] + 2, sz = R * (Q.m[1] + 2);
  const T inv_h2 = T(Q.L.ih2);
  const int nc = oct_cells(Q);
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    int x, y, z;
    oct_xyz(Q, c, &x, &y, &z);
    const int t = oct_ti(Q, x, y, z);
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
  // a full C holds the whole cube: F's part sits at F.o / 2 in it
  const bool off = C.full && !F.full;
  const int cofs[3] = {off ? F.o[0] / 2 : 0, off ? F.o[1] / 2 : 0, off ? F.o[2] / 2 : 0};
  const int nc = oct_cells(F);
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    int x, y, z;
    oct_xyz(F, c, &x, &y, &z);
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
          v = v + wgt * C.tile[oct_ti(C, u[0] + sx * o[0], u[1] + sy * o[1], D == 3 ? u[2] + sz * o[2] : 0)];
        }
    F.tile[oct_ti(F, x, y, z)] += v;
  }
}

// global-memory index of part cell (x, y, z) of level Q (b / old fields;
// phi adds L.poff - L.off): its block's run, colour-split
template <typename T, int D>
__device__ __forceinline__ long long oct_gidx(const Oct<T, D> &Q, int x, int y, int z) {
  const long long base = Q.L.off + (long long)(Q.bid - Q.L.first) * Q.L.ncell;
  const int n = Q.nblk;
  // cube coordinates run below 2n: the place in the block is X or X - n
  const int X = Q.o[0] + x, Y = Q.o[1] + y, Z = D == 3 ? Q.o[2] + z : 0;
  return base + cs_pos_xyz(X >= n ? X - n : X, Y >= n ? Y - n : Y, Z >= n ? Z - n : Z, n, Q.L.ncell);
}

// nsweeps red/black sweeps of level F.  Each half-sweep of a split level
// pushes the cells it updated that border another part; the ring then holds
// both colours' current values.  A full level needs no exchange: CTA
// barriers only.
template <typename T, int D>
__device__ __forceinline__ void oct_sweeps(const Oct<T, D> &F, int nsweeps, int rank, int wneu) {
  for (int k = 0; k < nsweeps; k++)
    for (int col = 0; col < 2; col++) {
      oct_smooth<T, D>(F, col, wneu);
      __syncthreads();
      if (!F.full) {
        oct_push<T, D>(F, rank, col);
        cluster_barrier();
      }
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(kClusterThreads, 1) k_cycle_cluster(GmgView<T> V0, const LvArgs *lvtab, int lmin,
                                                                       ClusterArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int pz = D == 3 ? A.pz : 1;  // parts along z
  const int P = 4 * pz;              // CTAs of the cluster
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
    q.nblk = q.L.n;
    q.full = i >= A.full_from ? 1 : 0;
    const int kp[3] = {rank & 1, (rank >> 1) & 1, rank >> 2};
    const int np[3] = {2, 2, pz};
    int child = 0;  // which child of the root holds the part
    bool p2 = true;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      q.m[d] = d < D ? (q.full ? q.N : q.N / np[d]) : 1;
      q.o[d] = (d < D && !q.full) ? kp[d] * q.m[d] : 0;
      if (ch) child += (q.o[d] / q.nblk) << d;
      p2 = p2 && (q.m[d] & (q.m[d] - 1)) == 0;
    }
#pragma unroll
    for (int d = 0; d < 3; d++) q.lg[d] = p2 ? __ffs(q.m[d]) - 1 : -1;
    q.bid = q.L.first + (ch ? (1 << D) * root + child : root);
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
  {  // phi and b of the top level's part, in flight during the set-up
    const Oct<T, D> &q = Qs[0];
    const int nc = oct_cells(q);
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      int x, y, z;
      oct_xyz(q, c, &x, &y, &z);
      const long long g = oct_gidx(q, x, y, z);
      cp_async_elem(q.tile + oct_ti(q, x, y, z), V.phi + (q.L.poff - q.L.off) + g);
      cp_async_elem(q.b + c, V.b + g);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  // this CTA's rows of the coarse inverse (its part's cells of l_lo)
  const Oct<T, D> Qlo = Qs[ntl - 1];
  const double *cinv = A.cinv + (size_t)root * A.ncr * A.ncr;
  // rows of the coarse solve this CTA computes: its part's cells, or on a
  // full coarsest level the cells rank, rank + P, ...
  const int nlo = Qlo.full ? (A.ncr - rank + P - 1) / P : oct_cells(Qlo);
  auto row_of = [&](int c) {
    if (Qlo.full) return rank + P * c;
    int x, y, z;
    oct_xyz(Qlo, c, &x, &y, &z);
    return (Qlo.o[0] + x) + Qlo.N * ((Qlo.o[1] + y) + (D == 3 ? Qlo.N * (Qlo.o[2] + z) : 0));
  };
  // cut lists: per cell of the part its entry, and the blocks' coefficients
  for (int i = 0; i < ntl; i++) {
    const Oct<T, D> &q = Qs[i];
    if (!q.mm) continue;
    const int nc = oct_cells(q);
    for (int c = threadIdx.x; c < nc; c += blockDim.x) q.eidx[c] = 0;
  }
  __syncthreads();
  const int ne = s_ecum[ntl];  // entries of every level
  auto entry = [&](int k, int *lvl, int *e) {
    int i = 0;
    while (k >= s_ecum[i + 1]) i++;
    *lvl = i;
    *e = k - s_ecum[i];
  };
  // the coefficients: copies all in flight together
  for (int k = threadIdx.x; k < ne; k += blockDim.x) {
    int i, e;
    entry(k, &i, &e);
    const Oct<T, D> &q = Qs[i];
    const int ge = s_e0[i] + e;
#pragma unroll
    for (int kk = 0; kk < 2 * D + 1; kk++) cp_async_elem(q.cf + kk * q.mm + e, V.cut_coef + (size_t)kk * V.n_cut + ge);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  if (A.stage_rows) {
    double *rows = reinterpret_cast<double *>(smem_raw + A.off_rows);
    for (int i = threadIdx.x; i < nlo * A.ncr; i += blockDim.x) {
      const int c = i / A.ncr, j = i - c * A.ncr;
      cp_async_elem(rows + i, cinv + (size_t)row_of(c) * A.ncr + j);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  // the entries' cells, kEntryBatch a thread at a time (their reads overlap)
  constexpr int kEntryBatch = 4;
  for (int k0 = threadIdx.x; k0 < ne; k0 += kEntryBatch * blockDim.x) {
    int cells[kEntryBatch];
#pragma unroll
    for (int u = 0; u < kEntryBatch; u++) {
      const int k = k0 + u * (int)blockDim.x;
      int i = 0, e = 0;
      if (k < ne) entry(k, &i, &e);
      cells[u] = k < ne ? V.cut_cell[s_e0[i] + e] : -1;
    }
#pragma unroll
    for (int u = 0; u < kEntryBatch; u++) {
      const int k = k0 + u * (int)blockDim.x;
      if (k >= ne) continue;
      int i, e;
      entry(k, &i, &e);
      const Oct<T, D> &q = Qs[i];
      // the entry's cell in cube coordinates (the block's origin plus its
      // place in the block); is it in this part?
      int X, Y, Z;
      cell_xyz_rt<D>(cells[u], q.nblk, &X, &Y, &Z);
      const int x = X + (q.o[0] / q.nblk) * q.nblk - q.o[0];
      const int y = Y + (q.o[1] / q.nblk) * q.nblk - q.o[1];
      const int z = D == 3 ? Z + (q.o[2] / q.nblk) * q.nblk - q.o[2] : 0;
      if (x >= 0 && x < q.m[0] && y >= 0 && y < q.m[1] && z >= 0 && z < q.m[2])
        q.eidx[x + q.m[0] * (y + q.m[1] * z)] = (unsigned short)(e + 1);
    }
  }
  if (A.stage_rows)
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  else
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  // every CTA of the cluster is running and its top level is in place
  cluster_barrier();
  const int wneu = V.wneu;
  oct_push<T, D>(Qs[0], rank, -1);  // the top level's ghosts across the part faces
  cluster_barrier();
  for (int i = 0; i + 1 < ntl; i++) {
    const Oct<T, D> F = Qs[i], C = Qs[i + 1];
    oct_sweeps<T, D>(F, F.L.nd, rank, wneu);
    oct_walls<T, D>(F, wneu);
    __syncthreads();
    oct_resid_restrict<T, D>(F, C, rank, P);
    __syncthreads();
    if (!C.full) {
      oct_push<T, D>(C, rank, -1);
      cluster_barrier();
    } else if (!F.full) {
      cluster_barrier();  // every part's share of C has arrived
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
        const int kx = X / q.m[0], ky = Y / q.m[1], kz = D == 3 ? Z / q.m[2] : 0;
        const int x = X - kx * q.m[0], y = Y - ky * q.m[1], z = D == 3 ? Z - kz * q.m[2] : 0;
        bd[j] = (double)peer(q.b, kx + 2 * ky + 4 * kz)[x + q.m[0] * (y + q.m[1] * z)];
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
        const int ti = oct_ti(q, X - q.o[0], Y - q.o[1], Z - q.o[2]);
        q.tile[ti] = T(s);
        if (q.full)  // every CTA holds the whole level
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
      const int nc = oct_cells(C);
      for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        int x, y, z;
        oct_xyz(C, c, &x, &y, &z);
        const int t = oct_ti(C, x, y, z);
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
    oct_sweeps<T, D>(F, F.L.nu, rank, wneu);
  }
  {  // phi of the top level's part back to global memory
    const Oct<T, D> &q = Qs[0];
    const int nc = oct_cells(q);
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      int x, y, z;
      oct_xyz(q, c, &x, &y, &z);
      V.phi[(q.L.poff - q.L.off) + oct_gidx(q, x, y, z)] = q.tile[oct_ti(q, x, y, z)];
    }
  }
}

}  // namespace gmg
