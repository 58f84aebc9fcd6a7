// K red/black half-sweeps of one level in one pass (temporal blocking).
//
// A CTA stages its block together with a K-cell halo from the 26 same-level
// neighbours (phi and b), then runs the K half-sweeps of Sec. 2.2 on shrinking
// regions: half-sweep j updates the cells within K-1-j of the block, which
// only needs values that were valid after half-sweep j-1.  Every cell's update
// therefore reads exactly the inputs it reads in K separate half-sweep
// launches, so the result is the same; the level is read once instead of K
// times and K-1 launches disappear.  Walls: the first layer beyond a wall is
// refreshed from its mirror cell before each half-sweep (reading W); cells
// beyond a wall are never updated.  Used on levels whose blocks all have their
// 26 neighbours on the same level or outside the domain (uniform levels).
// Neighbouring CTAs read each other's halo, so the result goes to the other
// phi buffer.
#pragma once

#include "kernels.cuh"

namespace gmg {

template <typename T, int D, int NT, int K>
struct FusedGeo {
  static constexpr int VEC = 16 / sizeof(T);
  static constexpr int XH = ((K + VEC - 1) / VEC) * VEC;  // x halo rounded to 16 bytes
  static constexpr int RX = NT + 2 * XH, RY = NT + 2 * K, RZ = D == 3 ? NT + 2 * K : 1;
  static constexpr int SY = RX, SZ = RX * RY, TS = RX * RY * RZ;
  static constexpr int NC = D == 3 ? NT * NT * NT : NT * NT;
  static __host__ __device__ int idx(int x, int y, int z) { return (x + XH) + SY * (y + K) + (D == 3 ? SZ * (z + K) : 0); }
  static constexpr size_t smem_bytes() { return sizeof(T) * (size_t)(2 * TS); }
};

template <typename T, int D, int NT, int K>
__global__ void __launch_bounds__(kThreads) k_smooth_tb(GmgView<T> V0, LvArgs L, long long out_poff) {
  pdl_start();
  using F = FusedGeo<T, D, NT, K>;
  constexpr int n = NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_nb[kNbr];
  __shared__ long long s_stb[kNbr];
  T *tp = reinterpret_cast<T *>(smem_raw);
  T *tb = tp + F::TS;
  int bid;
  GmgView<T> V;
  if (!slot_item(V0, L, &bid, &V)) return;
  if (threadIdx.x < kNbr) {
    const int id = V.nbr[(size_t)bid * kNbr + threadIdx.x];
    s_nb[threadIdx.x] = id;
    s_stb[threadIdx.x] = id >= 0 ? V.st_base[id] : -1;
  }
  __syncthreads();
  // stage phi and b of the block and its neighbours cell by cell (the
  // fields' colour-split layout puts a row's cells in two runs)
  constexpr int CX = F::RX, ROWS = F::RY * F::RZ;
  for (int i = threadIdx.x; i < CX * ROWS; i += blockDim.x) {
    const int cx = i % CX, row = i / CX;
    const int x = cx - F::XH, y = row % F::RY - K, z = D == 3 ? row / F::RY - K : 0;
    if (x < -K || x >= n + K) continue;  // beyond the halo (x rounded to 16 bytes)
    const int ox = x < 0 ? -1 : (x >= n ? 1 : 0), oy = y < 0 ? -1 : (y >= n ? 1 : 0);
    const int oz = D == 3 ? (z < 0 ? -1 : (z >= n ? 1 : 0)) : 0;
    const int id = s_nb[nbr_slot(ox, oy, oz)];
    if (id < 0) continue;  // outside the domain
    const long long c = (long long)(id - L.first) * F::NC +
                        cs_pos_xyz(x - ox * n, y - oy * n, D == 3 ? z - oz * n : 0, n, F::NC);
    cp_async_elem(tp + F::idx(x, y, z), V.phi + L.poff + c);
    cp_async_elem(tb + F::idx(x, y, z), V.b + L.off + c);
  }
  cp_async_wait_all();
  __syncthreads();
  bool wlo[3] = {false, false, false}, whi[3] = {false, false, false};
#pragma unroll
  for (int a = 0; a < D; a++) {
    wlo[a] = s_nb[nbr_slot(a == 0 ? -1 : 0, a == 1 ? -1 : 0, a == 2 ? -1 : 0)] == -2;
    whi[a] = s_nb[nbr_slot(a == 0 ? 1 : 0, a == 1 ? 1 : 0, a == 2 ? 1 : 0)] == -2;
  }
  const bool anywall = wlo[0] || whi[0] || wlo[1] || whi[1] || wlo[2] || whi[2];
  // any cut block among the 27?  If not, every cell takes the regular stencil
  bool cut_near = false;
  for (int k = 0; k < kNbr; k++) cut_near = cut_near || s_stb[k] >= 0;
  const T h2 = T(L.h2), inv2d = T(1.0 / (2 * D));
  for (int j = 0; j < K; j++) {
    const int color = j & 1;
    if (anywall) {
      // first layer beyond each wall <- sign * mirror cell (homogeneous ghosts)
#pragma unroll
      for (int a = 0; a < D; a++)
#pragma unroll
        for (int side = 0; side < 2; side++) {
          if (!(side ? whi[a] : wlo[a])) continue;
          const T sg = ((V.wneu >> (2 * a + side)) & 1) ? T(1) : T(-1);
          // the plane spans the tile in the other axes
          const int e1 = a == 0 ? F::RY : F::RX;
          const int e2 = a == 2 ? F::RY : F::RZ;
          for (int i = threadIdx.x; i < e1 * e2; i += blockDim.x) {
            const int u = i % e1, v = i / e1;
            int x, y, z;
            if (a == 0) {
              y = u - K;
              z = D == 3 ? v - K : 0;
              x = side ? n : -1;
              tp[F::idx(x, y, z)] = sg * tp[F::idx(side ? n - 1 : 0, y, z)];
            } else if (a == 1) {
              x = u - F::XH;
              z = D == 3 ? v - K : 0;
              y = side ? n : -1;
              tp[F::idx(x, y, z)] = sg * tp[F::idx(x, side ? n - 1 : 0, z)];
            } else {
              x = u - F::XH;
              y = v - K;
              z = side ? n : -1;
              tp[F::idx(x, y, z)] = sg * tp[F::idx(x, y, side ? n - 1 : 0)];
            }
          }
        }
      __syncthreads();
    }
    const int r = K - 1 - j;
    const int lx = wlo[0] ? 0 : -r, hx = whi[0] ? n : n + r;
    const int ly = wlo[1] ? 0 : -r, hy = whi[1] ? n : n + r;
    const int lz = D == 3 ? (wlo[2] ? 0 : -r) : 0, hz = D == 3 ? (whi[2] ? n : n + r) : 1;
    const int exh = (hx - lx + 1) / 2, ey = hy - ly;
    // a thread's (x-pair, y) positions in a plane, computed once per half-sweep
    constexpr int PL = ((NT + 2 * K) / 2 * (NT + 2 * K) + kThreads - 1) / kThreads;
    int pxi[PL], py[PL];
#pragma unroll
    for (int k = 0; k < PL; k++) {
      const int q = threadIdx.x + k * kThreads;
      pxi[k] = q < exh * ey ? q % exh : -1;
      py[k] = ly + q / exh;
    }
    for (int z = lz; z < hz; z++) {
#pragma unroll
      for (int k = 0; k < PL; k++) {
        if (pxi[k] < 0) continue;
        const int y = py[k];
        const int x = lx + 2 * pxi[k] + ((lx + y + z + color) & 1);
        if (x >= hx) continue;
        const int t = F::idx(x, y, z);
        T nv;
        if (!cut_near) {
          nv = (nb_sum<T, D>(tp, t, F::SY, F::SZ) - h2 * tb[t]) * inv2d;
        } else {
          const int ox = x < 0 ? -1 : (x >= n ? 1 : 0), oy = y < 0 ? -1 : (y >= n ? 1 : 0);
          const int oz = D == 3 ? (z < 0 ? -1 : (z >= n ? 1 : 0)) : 0;
          const long long stb = s_stb[nbr_slot(ox, oy, oz)];
          const int c = (x - ox * n) + n * ((y - oy * n) + (D == 3 ? n * (z - oz * n) : 0));
          if (stb < 0 || !V.spec[stb / (2 * D + 1) + c]) {
            nv = (nb_sum<T, D>(tp, t, F::SY, F::SZ) - h2 * tb[t]) * inv2d;
          } else {
            T diag;
            const T sum = offdiag_st<T, D>(V.st + stb, tp, t, F::SY, F::SZ, F::NC, c, &diag);
            nv = (tb[t] - sum) / diag;
          }
        }
        tp[t] = nv;
      }
    }
    __syncthreads();
  }
  T *out = V.phi + out_poff + (long long)(bid - L.first) * F::NC;
  for (int q = threadIdx.x; q < F::NC; q += blockDim.x) {  // the colour-split run in order
    int x, y, z;
    cs_xyz(q, n, F::NC, D, &x, &y, &z);
    out[q] = tp[F::idx(x, y, z)];
  }
}

}  // namespace gmg
