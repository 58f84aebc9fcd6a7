// Half-sweeps on several right-hand-side slots of one block per CTA.
//
// With many slots (batched right-hand sides, serving sessions), one CTA can
// stage and update SG slots of the same block: the block's neighbour ids,
// flags and stencil flags are read once, and the index arithmetic of the
// tile staging and of the colour loop is done once for all SG slots, while
// SG tiles are in flight at the same time.  The arithmetic of every cell is
// that of smooth_block (Sec. 2.2, readings S and SW), so results do not
// depend on SG.
#pragma once

#include "kernels.cuh"

namespace gmg {

// Shared memory of k_smooth_sg: SG tiles, SG dense b arrays, the flags.
template <typename T>
__host__ __device__ inline size_t sg_smem_bytes(int D, int n, int SG) {
  const int tile = D == 3 ? TileGeo<T, 3>(n).size : TileGeo<T, 2>(n).size;
  const int nc = D == 3 ? n * n * n : n * n;
  return sizeof(T) * (size_t)SG * (tile + nc) + (size_t)((nc + 15) / 16 * 16);
}

// load_tile for the slots slot[0..SG) of block bid (slot < 0: skipped):
// slot s's tile at tiles + s * G.size, its b at bs + s * ncell; mid() runs
// once the neighbour ids have arrived.
template <typename T, int D, int NT, int SG, typename Mid>
__device__ __forceinline__ void load_tiles(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid,
                                           const int *slot, T *tiles, T *bs, unsigned char *sflag, long long sb,
                                           Mid mid) {
  static_assert(NT != 0, "slot groups need a compile-time block size");
  __shared__ int s_nb[6];
  __shared__ int s_fl;
  constexpr int n = NT, ncell = D == 3 ? NT * NT * NT : NT * NT, nf = D == 3 ? NT * NT : NT;
  constexpr int VEC = 16 / sizeof(T);
  static_assert(NT % VEC == 0, "rows of whole 16-byte chunks");
  const TileGeo<T, D> G(n);
  if (threadIdx.x < 2 * D) {
    const int a = threadIdx.x >> 1, side = threadIdx.x & 1;
    const int o[3] = {a == 0 ? 2 * side - 1 : 0, a == 1 ? 2 * side - 1 : 0, a == 2 ? 2 * side - 1 : 0};
    s_nb[threadIdx.x] = V.nbr[(size_t)bid * kNbr + nbr_slot(o[0], o[1], o[2])];
  }
  if (threadIdx.x == 0) s_fl = V.flags[bid];
  const long long base = L.off + (long long)(bid - L.first) * ncell;
  const long long pbase = L.poff + (long long)(bid - L.first) * ncell;
  for (int i = threadIdx.x; i < ncell / VEC; i += blockDim.x) {
    const int c = i * VEC;
    const int t = G.idx(c % n, (c / n) % n, D == 3 ? c / (n * n) : 0);
#pragma unroll
    for (int s = 0; s < SG; s++)
      if (slot[s] >= 0) {
        cp_async16(tiles + s * G.size + t, V.phi + slot[s] * V.rs_phi + pbase + c);
        cp_async16(bs + s * ncell + c, V.b + slot[s] * V.rs_f + base + c);
      }
  }
  if (sb >= 0) {
    const unsigned char *src = V.spec + sb / (2 * D + 1);
    if (ncell % 16 == 0 && ((size_t)src & 15) == 0) {
      for (int i = threadIdx.x; i < ncell / 16; i += blockDim.x) cp_async16(sflag + 16 * i, src + 16 * i);
    } else {
      for (int c = threadIdx.x; c < ncell; c += blockDim.x) sflag[c] = src[c];
    }
  }
  __syncthreads();
  mid();
  const int fl = s_fl;
  // x faces cell by cell
  for (int i = threadIdx.x; i < 2 * nf; i += blockDim.x) {
    const int f = i / nf, j = i - f * nf, side = f & 1;
    const int id = s_nb[f];
    if ((fl & wall_bit(0, side)) || id < 0) continue;
    const int u = j % n, v = D == 3 ? j / n : 0;
    const int t = G.idx(side ? n : -1, u, v);
    const long long q = L.poff + (long long)(id - L.first) * ncell + (side ? 0 : n - 1) + n * (u + n * v);
#pragma unroll
    for (int s = 0; s < SG; s++)
      if (slot[s] >= 0) cp_async_elem(tiles + s * G.size + t, V.phi + slot[s] * V.rs_phi + q);
  }
  // y and z faces as rows of 16-byte chunks
  constexpr int cpr = NT / VEC, rows = D == 3 ? NT : 1;
  for (int i = threadIdx.x; i < (2 * D - 2) * rows * cpr; i += blockDim.x) {
    const int f = 2 + i / (rows * cpr), rem = i - (f - 2) * rows * cpr;
    const int row = rem / cpr, x0 = (rem - row * cpr) * VEC;
    const int a = f >> 1, side = f & 1;
    const int id = s_nb[f];
    if ((fl & wall_bit(a, side)) || id < 0) continue;
    const int gn = side ? n : -1, sn = side ? 0 : n - 1;
    const int gy = a == 1 ? gn : row, gz = a == 2 ? gn : (D == 3 ? row : 0);
    const int qy = a == 1 ? sn : row, qz = a == 2 ? sn : (D == 3 ? row : 0);
    const int t = G.idx(x0, gy, gz);
    const long long q = L.poff + (long long)(id - L.first) * ncell + x0 + n * (qy + (D == 3 ? n * qz : 0));
#pragma unroll
    for (int s = 0; s < SG; s++)
      if (slot[s] >= 0) cp_async16(tiles + s * G.size + t, V.phi + slot[s] * V.rs_phi + q);
  }
  cp_async_wait_all();
  __syncthreads();
  bool special = false;
#pragma unroll
  for (int f = 0; f < 2 * D; f++) special = special || (fl & wall_bit(f >> 1, f & 1)) || s_nb[f] < 0;
  if (!special) return;
  for (int i = threadIdx.x; i < 2 * D * nf; i += blockDim.x) {
    const int f = i / nf, j = i - f * nf;
    const int a = f >> 1, side = f & 1;
    const bool wall = (fl & wall_bit(a, side)) != 0;
    if (!wall && s_nb[f] >= 0) continue;
    const int u = j % n, v = D == 3 ? j / n : 0;
    const int gn = side ? n : -1, mn = side ? n - 1 : 0;
    const int gx = a == 0 ? gn : u, gy = a == 1 ? gn : (a == 0 ? u : v), gz = a == 2 ? gn : v;
    const int mx = a == 0 ? mn : u, my = a == 1 ? mn : (a == 0 ? u : v), mz = a == 2 ? mn : v;
    const int g[3] = {gx, gy, gz};
#pragma unroll
    for (int s = 0; s < SG; s++) {
      if (slot[s] < 0) continue;
      T *tile = tiles + s * G.size;
      T val;
      if (wall) {
        val = (((V.wneu >> f) & 1) ? T(1) : T(-1)) * tile[G.idx(mx, my, mz)];
      } else {
        const T *phi = V.phi + slot[s] * V.rs_phi;
        val = refine_ghost<T, D>(phi, V.nbr, V.flags, V.parent, V.pofs, V.wneu, L, Lp, bid, g, a, phi + pbase);
      }
      tile[G.idx(gx, gy, gz)] = val;
    }
  }
  __syncthreads();
}

// One red (color 0) or black (color 1) half-sweep of a level on SG slots of
// each block per CTA: the grid holds count x ceil(nrhs / SG) CTAs, slot
// groups fastest.
template <typename T, int D, int NT, int SG>
__global__ void __launch_bounds__(kThreads) k_smooth_sg(GmgView<T> V, LvArgs L, LvArgs Lp, int color) {
  pdl_start();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ngrp = (V.nrhs + SG - 1) / SG;
  const int grp = (int)(blockIdx.x % (unsigned)ngrp), bid = L.first + (int)(blockIdx.x / (unsigned)ngrp);
  int slot[SG];
  bool any = false;
#pragma unroll
  for (int s = 0; s < SG; s++) {
    const int r = grp * SG + s;
    slot[s] = (r < V.nrhs && V.active[unit_of(V, r, bid)]) ? r : -1;
    any = any || slot[s] >= 0;
  }
  if (!any) return;  // every slot of the group frozen (same answer in every thread)
  constexpr int n = NT, hn = NT / 2, ncell = D == 3 ? NT * NT * NT : NT * NT;
  const TileGeo<T, D> G(n);
  T *tiles = reinterpret_cast<T *>(smem_raw);
  T *bs = tiles + SG * G.size;
  unsigned char *sfl = reinterpret_cast<unsigned char *>(bs + SG * ncell);
  const long long pbase = L.poff + (long long)(bid - L.first) * ncell;
  const long long sb = V.st_base[bid];
  const int4 cl = V.cut_list[bid];
  const int e0 = cl.x + (color ? cl.y : 0), m = color ? cl.z : cl.y;
  CutCell<T, D> q;
  load_tiles<T, D, NT, SG>(V, L, Lp, bid, slot, tiles, bs, sfl, sb, [&] {
    if ((int)threadIdx.x < m) q.fetch(V, e0 + threadIdx.x);
  });
  const T h2 = T(L.h2), inv2d = T(1.0 / (2 * D));
  for (int j = threadIdx.x; j < ncell / 2; j += blockDim.x) {
    const int rest = j / hn;
    const int y = rest % n, z = D == 3 ? rest / n : 0;
    const int x = 2 * (j % hn) + ((y + z + color) & 1);
    const int c = x + n * (y + n * z);
    if (sb >= 0 && sfl[c]) continue;  // a listed cell
    const int t = G.idx(x, y, z);
#pragma unroll
    for (int s = 0; s < SG; s++) {
      if (slot[s] < 0) continue;
      const T *tile = tiles + s * G.size;
      V.phi[slot[s] * V.rs_phi + pbase + c] = (nb_sum<T, D>(tile, t, G.sy, G.sz) - h2 * bs[s * ncell + c]) * inv2d;
    }
  }
  // the colour's listed cells, one stencil for all SG slots
  auto upd = [&](const CutCell<T, D> &u) {
    int x, y, z;
    cell_xyz<D>(u.c, n, &x, &y, &z);
    const int t = G.idx(x, y, z);
#pragma unroll
    for (int s = 0; s < SG; s++) {
      if (slot[s] < 0) continue;
      const T *tile = tiles + s * G.size;
      V.phi[slot[s] * V.rs_phi + pbase + u.c] = (bs[s * ncell + u.c] - offdiag_of<T, D>(u.a, tile, t, G.sy, G.sz)) / u.a[0];
    }
  };
  if ((int)threadIdx.x < m) upd(q);
  for (int i = threadIdx.x + blockDim.x; i < m; i += blockDim.x) {
    CutCell<T, D> u;
    u.fetch(V, e0 + i);
    upd(u);
  }
}

}  // namespace gmg
