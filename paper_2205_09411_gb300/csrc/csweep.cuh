// Red/black half-sweep on the colour-split block layout (Sec. 2.2,
// readings S and SW; Eqs. (lpl-1d-lsf) for listed cells).
//
// A cell of colour c has only cells of colour 1 - c as neighbours.  With the
// fields stored per block as the red half then the black half (cs_pos), a
// half-sweep of colour c stages in shared memory only the other colour's
// half of the block and of its face neighbours, plus its own colour's b,
// and writes its own colour's half back as one contiguous run: about 1.5
// values a cell move instead of 3 for the interleaved layout, in whole
// sectors.
//
// The other colour is kept in rows: row (y, z) holds, at k = 0 .. n/2 - 1,
// the other colour's cells x = 2k + q' of that row of the block (q' = (y +
// z + 1 - c) mod 2), and at k = -1 and k = n/2 the x ghosts.  An own cell x
// = 2k + q (q = 1 - q') then finds its x neighbours at k - 1 + q and k + q
// of its row and its y and z neighbours at k of the adjacent rows.  Rows
// outside the block (y or z = -1 or n) hold the face ghosts: a same-level
// neighbour's boundary run, the wall reflection of the own cell beside it
// (reading W), or the refinement-boundary value (reading G).
#pragma once

#include "kernels.cuh"

namespace gmg {

template <typename T, int D, int NT>
struct CsGeo {
  static constexpr int H = (D == 3 ? NT * NT * NT : NT * NT) / 2;  // cells of one colour
  static constexpr int HN = NT / 2;                                 // a row's cells of one colour
  static constexpr int X0 = 16 / (int)sizeof(T);                    // k = 0 on a 16-byte boundary
  static constexpr int RO = HN + 2 * X0;                            // row stride
  static constexpr int NR = D == 3 ? (NT + 2) * (NT + 2) : NT + 2;  // rows, ghost rows included
  static constexpr int OS = NR * RO;                                // other-colour tile
  // the tile's row of cells (y, z) of the block (each in -1 .. NT)
  static __device__ __forceinline__ int row(int y, int z) { return (y + 1) + (D == 3 ? (NT + 2) * (z + 1) : 0); }
  static __device__ __forceinline__ int at(int r, int k) { return r * RO + X0 + k; }
  // shared memory of SG slots: the other-colour tiles, the own colour's b,
  // the block's stencil flags
  static constexpr size_t smem_bytes(int sg) {
    return sizeof(T) * (size_t)sg * (OS + H) + (size_t)((2 * H + 15) / 16 * 16);
  }
};

// BF: the other colour's tile holds BF16 values (the finest level of
// GMG_MIXED_BF16); b stays T.
template <typename T, int D, int NT, bool BF = false>
inline size_t cs_smem_bytes(int sg) {
  if (!BF) return CsGeo<T, D, NT>::smem_bytes(sg);
  using G = CsGeo<bf16s, D, NT>;
  static_assert((sizeof(bf16s) * G::OS) % 16 == 0, "b must start on a 16-byte boundary");
  return sizeof(bf16s) * (size_t)sg * G::OS + sizeof(T) * (size_t)sg * G::H + (size_t)((2 * G::H + 15) / 16 * 16);
}

// BF16 values a piece of a colour run is copied in: 8 (16 bytes), 4 or 2
// (a run of a row holds NT / 2 cells, an even number on the BF16 levels)
template <int HN>
struct BfPiece {
  static_assert(HN % 2 == 0, "BF16 levels have even runs");
  static constexpr int value = HN % 8 == 0 ? 8 : (HN % 4 == 0 ? 4 : 2);
};

// Two adjacent tile entries (the first at an even index) as floats, and a
// paired store of two results (rounded to BF16 for a BF16 level).
__device__ __forceinline__ void ld_pair(const float *p, float *v) {
  const float2 w = *reinterpret_cast<const float2 *>(p);
  v[0] = w.x;
  v[1] = w.y;
}
__device__ __forceinline__ void ld_pair(const bf16s *p, float *v) {
  const unsigned w = *reinterpret_cast<const unsigned *>(p);
  v[0] = __uint_as_float(w << 16);
  v[1] = __uint_as_float(w & 0xffff0000u);
}
__device__ __forceinline__ void st_pair(float *p, float v0, float v1) {
  *reinterpret_cast<float2 *>(p) = make_float2(v0, v1);
}
__device__ __forceinline__ void st_pair(bf16s *p, float v0, float v1) {
  *reinterpret_cast<unsigned *>(p) = (unsigned)st_val<bf16s>(v0) | ((unsigned)st_val<bf16s>(v1) << 16);
}

// cs_stage_interior for BF16 phi: slot base rs_h in hphi (level-local
// offsets); b as T.
template <typename T, int D, int NT>
__device__ __forceinline__ void cs_stage_interior_bf(const GmgView<T> &V, const LvArgs &L, int bid, int c,
                                                     long long rs_h, long long rs_f, bf16s *O, T *B) {
  using G = CsGeo<bf16s, D, NT>;
  constexpr int PW = BfPiece<G::HN>::value;
  constexpr int VB = 16 / sizeof(T);
  const long long pbase = rs_h + L.poff + (long long)(bid - L.first) * (2 * G::H);
  const long long base = rs_f + L.off + (long long)(bid - L.first) * (2 * G::H);
  const bf16s *oth = V.hphi + pbase + (1 - c) * G::H;
  const T *bown = V.b + base + c * G::H;
  for (int i = threadIdx.x; i < G::H / PW; i += blockDim.x) {
    const int j = i * PW, r = j / G::HN, k = j - r * G::HN;
    cp_async_bytes<2 * PW>(O + G::at(G::row(r % NT, D == 3 ? r / NT : 0), k), oth + j);
  }
  if (G::H % VB == 0) {
    for (int i = threadIdx.x; i < G::H / VB; i += blockDim.x) cp_async16(B + i * VB, bown + i * VB);
  } else {
    for (int j = threadIdx.x; j < G::H; j += blockDim.x) cp_async_elem(B + j, bown + j);
  }
}

// cs_stage_faces for BF16 phi.  The y and z face runs come in pieces as in
// cs_stage_interior_bf.  An x ghost from a same-level neighbour comes as an
// aligned 4-byte pair: the neighbour's cells 0 and 1 of the run to k = HN,
// HN + 1 (ghost x = NT), or its cells HN - 2 and HN - 1 to k = -2, -1
// (ghost x = -1); k = HN + 1 and -2 are row padding, never read.  At a wall
// the own cell is staged by a plain load (a pair there would overwrite the
// block's own first or last cell).
template <typename T, int D, int NT>
__device__ __forceinline__ void cs_stage_faces_bf(const GmgView<T> &V, const LvArgs &L, int bid, int c,
                                                  const int *s_nb, int fl, long long rs_h, bf16s *O) {
  using G = CsGeo<bf16s, D, NT>;
  constexpr int PW = BfPiece<G::HN>::value;
  const long long pown = rs_h + L.poff + (long long)(bid - L.first) * (2 * G::H) + c * G::H;  // own colour
  constexpr int FR = D == 3 ? NT : 1;
  constexpr int PR = G::HN / PW;
  for (int i = threadIdx.x; i < (2 * D - 2) * FR * PR; i += blockDim.x) {
    const int f = 2 + i / (FR * PR), rem = i - (f - 2) * FR * PR;
    const int u = rem / PR, k = (rem - u * PR) * PW;
    const int a = f >> 1, side = f & 1;
    const int id = s_nb[f];
    const bool wall = (fl & wall_bit(a, side)) != 0;
    if (!wall && id < 0) continue;
    const int yg = a == 1 ? (side ? NT : -1) : u, zg = a == 2 ? (side ? NT : -1) : u;
    const bf16s *src;
    if (wall) {
      const int yi = a == 1 ? (side ? NT - 1 : 0) : u, zi = a == 2 ? (side ? NT - 1 : 0) : u;
      src = V.hphi + pown + G::HN * (yi + (D == 3 ? NT * zi : 0));
    } else {
      const int ys = a == 1 ? (side ? 0 : NT - 1) : u, zs = a == 2 ? (side ? 0 : NT - 1) : u;
      src = V.hphi + rs_h + L.poff + (long long)(id - L.first) * (2 * G::H) + (1 - c) * G::H +
            G::HN * (ys + (D == 3 ? NT * zs : 0));
    }
    cp_async_bytes<2 * PW>(O + G::at(G::row(yg, D == 3 ? zg : 0), k), src + k);
  }
  for (int r = threadIdx.x; r < G::H / G::HN; r += blockDim.x) {
    const int y = r % NT, z = D == 3 ? r / NT : 0;
    const int qo = (y + z + 1 - c) & 1;
    const int side = qo ? 0 : 1;
    const int id = s_nb[side];
    const bool wall = (fl & wall_bit(0, side)) != 0;
    if (!wall && id < 0) continue;
    if (wall) {
      O[G::at(G::row(y, z), side ? G::HN : -1)] = V.hphi[pown + G::HN * (y + NT * z) + (side ? G::HN - 1 : 0)];
    } else {
      const long long rowb =
          rs_h + L.poff + (long long)(id - L.first) * (2 * G::H) + (1 - c) * G::H + G::HN * (y + NT * z);
      if (side)
        cp_async_bytes<4>(O + G::at(G::row(y, z), G::HN), V.hphi + rowb);
      else
        cp_async_bytes<4>(O + G::at(G::row(y, z), -2), V.hphi + rowb + G::HN - 2);
    }
  }
}

// Stages slot s's other-colour half and own-colour b for a half-sweep of
// colour c of block bid (cp.async; nothing here depends on the neighbour
// table, so the copies start before it is read).
template <typename T, int D, int NT>
__device__ __forceinline__ void cs_stage_interior(const GmgView<T> &V, const LvArgs &L, int bid, int c,
                                                  long long rs_phi, long long rs_f, T *O, T *B) {
  using G = CsGeo<T, D, NT>;
  constexpr int VEC = 16 / sizeof(T);
  constexpr bool kChunks = (G::HN % VEC) == 0;
  const long long pbase = rs_phi + L.poff + (long long)(bid - L.first) * (2 * G::H);
  const long long base = rs_f + L.off + (long long)(bid - L.first) * (2 * G::H);
  const T *oth = V.phi + pbase + (1 - c) * G::H;
  const T *bown = V.b + base + c * G::H;
  // the block's other colour, rows (y, z) of the block, and its own b
  if (kChunks) {
    for (int i = threadIdx.x; i < G::H / VEC; i += blockDim.x) {
      const int j = i * VEC, r = j / G::HN, k = j - r * G::HN;
      cp_async16(O + G::at(G::row(r % NT, D == 3 ? r / NT : 0), k), oth + j);
      cp_async16(B + j, bown + j);
    }
  } else {
    for (int j = threadIdx.x; j < G::H; j += blockDim.x) {
      const int r = j / G::HN, k = j - r * G::HN;
      cp_async_elem(O + G::at(G::row(r % NT, D == 3 ? r / NT : 0), k), oth + j);
      cp_async_elem(B + j, bown + j);
    }
  }
}

// Stages slot s's face ghosts that come from same-level blocks, and on a
// wall face the block's own cells beside the wall (cp.async); the wall
// sign and the refinement ghosts need the copies done and are applied by
// cs_special_ghosts.  A wall ghost reflects the own-colour cell beside it
// (reading W), which sits at the same position k of its row's own-colour
// run as the ghost in the ghost row: the run is copied whole.
template <typename T, int D, int NT>
__device__ __forceinline__ void cs_stage_faces(const GmgView<T> &V, const LvArgs &L, int bid, int c, const int *s_nb,
                                               int fl, long long rs_phi, T *O) {
  using G = CsGeo<T, D, NT>;
  constexpr int VEC = 16 / sizeof(T);
  constexpr bool kChunks = (G::HN % VEC) == 0;
  const long long pown = rs_phi + L.poff + (long long)(bid - L.first) * (2 * G::H) + c * G::H;  // own colour
  // y and z faces toward same-level neighbours: the neighbour's boundary
  // row of the other colour, one contiguous run of HN cells per row (in
  // 16-byte pieces when the run is whole vectors); toward a wall, the own
  // colour's row beside it
  constexpr int FR = D == 3 ? NT : 1;  // rows per face
  constexpr int PW = kChunks ? VEC : 1;  // cells per piece
  constexpr int PR = G::HN / PW;         // pieces per row
  for (int i = threadIdx.x; i < (2 * D - 2) * FR * PR; i += blockDim.x) {
    const int f = 2 + i / (FR * PR), rem = i - (f - 2) * FR * PR;
    const int u = rem / PR, k = (rem - u * PR) * PW;  // u: the face's row, k: first cell of the piece
    const int a = f >> 1, side = f & 1;
    const int id = s_nb[f];
    const bool wall = (fl & wall_bit(a, side)) != 0;
    if (!wall && id < 0) continue;  // a refinement boundary
    const int yg = a == 1 ? (side ? NT : -1) : u, zg = a == 2 ? (side ? NT : -1) : u;
    const T *src;
    if (wall) {
      const int yi = a == 1 ? (side ? NT - 1 : 0) : u, zi = a == 2 ? (side ? NT - 1 : 0) : u;
      src = V.phi + pown + G::HN * (yi + (D == 3 ? NT * zi : 0));
    } else {
      const int ys = a == 1 ? (side ? 0 : NT - 1) : u, zs = a == 2 ? (side ? 0 : NT - 1) : u;
      src = V.phi + rs_phi + L.poff + (long long)(id - L.first) * (2 * G::H) + (1 - c) * G::H +
            G::HN * (ys + (D == 3 ? NT * zs : 0));
    }
    T *dst = O + G::at(G::row(yg, D == 3 ? zg : 0), k);
    if (kChunks)
      cp_async16(dst, src + k);
    else
      cp_async_elem(dst, src + k);
  }
  // x faces: in a row whose other-colour parity is 1 the ghost x = -1 is
  // read (at k = -1), in the other rows the ghost x = NT (at k = HN)
  for (int r = threadIdx.x; r < G::H / G::HN; r += blockDim.x) {
    const int y = r % NT, z = D == 3 ? r / NT : 0;
    const int qo = (y + z + 1 - c) & 1;
    const int side = qo ? 0 : 1;
    const int id = s_nb[side];
    const bool wall = (fl & wall_bit(0, side)) != 0;
    if (!wall && id < 0) continue;
    // the neighbour's cell (NT - 1, y, z) or (0, y, z): both of colour 1 -
    // c; at a wall the own cell (0, y, z) or (NT - 1, y, z) of colour c,
    // first or last of its row's own-colour run
    const long long q = wall ? pown + G::HN * (y + NT * z) + (side ? G::HN - 1 : 0)
                             : rs_phi + L.poff + (long long)(id - L.first) * (2 * G::H) + (1 - c) * G::H +
                                   G::HN * (y + NT * z) + (side ? 0 : G::HN - 1);
    cp_async_elem(O + G::at(G::row(y, z), side ? G::HN : -1), V.phi + q);
  }
}

// Wall and refinement-boundary ghosts of the other colour (after the
// staged copies have landed): a wall ghost is the sign times the own cell
// beside it (staged in the ghost's place by cs_stage_faces), a refinement
// ghost follows reading G (refine_ghost, on the slot's own block).
// S is the tile's type: T, or bf16s for a BF16 level (phi: the slot's T
// fields, for the coarse level; own: the block's own run, of type S).
template <typename T, int D, int NT, typename S = T>
__device__ __forceinline__ void cs_special_ghosts(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid,
                                                  int c, const int *s_nb, int fl, const T *phi, const S *own, S *O) {
  using G = CsGeo<S, D, NT>;
  constexpr int FR = D == 3 ? NT : 1;
  // y and z faces: ghost (x, -1 or NT, z) / (x, y, -1 or NT) with x = 2k + qg
  for (int i = threadIdx.x; i < (2 * D - 2) * FR * G::HN; i += blockDim.x) {
    const int f = 2 + i / (FR * G::HN), rem = i - (f - 2) * FR * G::HN;
    const int u = rem / G::HN, k = rem - u * G::HN;
    const int a = f >> 1, side = f & 1;
    const bool wall = (fl & wall_bit(a, side)) != 0;
    if (!wall && s_nb[f] >= 0) continue;
    const int yg = a == 1 ? (side ? NT : -1) : u, zg = a == 2 ? (side ? NT : -1) : (D == 3 ? u : 0);
    const int qg = (yg + zg + 1 - c) & 1;  // the ghost row's other-colour parity
    const int x = 2 * k + qg;
    S *dst = O + G::at(G::row(yg, zg), k);
    if (wall) {
      *dst = wall_reflect(*dst, (V.wneu >> f) & 1);
    } else {
      const int g[3] = {x, yg, zg};
      *dst = st_val<S>(refine_ghost<T, D>(phi, V.nbr, V.flags, V.parent, V.pofs, V.wneu, L, Lp, bid, g, a, own));
    }
  }
  for (int r = threadIdx.x; r < G::H / G::HN; r += blockDim.x) {
    const int y = r % NT, z = D == 3 ? r / NT : 0;
    const int side = ((y + z + 1 - c) & 1) ? 0 : 1;
    const bool wall = (fl & wall_bit(0, side)) != 0;
    if (!wall && s_nb[side] >= 0) continue;
    const int xg = side ? NT : -1;
    S *dst = O + G::at(G::row(y, z), side ? G::HN : -1);
    if (wall) {
      *dst = wall_reflect(*dst, (V.wneu >> side) & 1);
    } else {
      const int g[3] = {xg, y, z};
      *dst = st_val<S>(refine_ghost<T, D>(phi, V.nbr, V.flags, V.parent, V.pofs, V.wneu, L, Lp, bid, g, 0, own));
    }
  }
}

// One half-sweep of colour `color` on block bid for the slots slot[0 ..
// SG - 1] (-1: skipped); shared memory as CsGeo::smem_bytes(SG).  Used by
// the per-level kernel below and by the cooperative coarse cycle.
// BF: the level's phi is stored as BF16 (the finest level of
// GMG_MIXED_BF16): tiles of BF16 values, arithmetic in T, each result
// rounded to BF16 when written.
template <typename T, int D, int NT, int SG, bool BF = false>
__device__ __forceinline__ void smooth_cs_block(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid,
                                                const int *slot, int color, unsigned char *smem_raw) {
  using S = typename std::conditional<BF, bf16s, T>::type;
  using G = CsGeo<S, D, NT>;
  __shared__ int s_nb[6];
  __shared__ int s_fl;
  S *O = reinterpret_cast<S *>(smem_raw);
  T *B = reinterpret_cast<T *>(O + SG * G::OS);
  S *Pf;  // the level's phi (slot 0)
  long long rsP;
  if constexpr (BF) {
    Pf = V.hphi;
    rsP = V.rs_h;
  } else {
    Pf = V.phi;
    rsP = V.rs_phi;
  }
  unsigned char *sfl = reinterpret_cast<unsigned char *>(B + SG * G::H);
  const long long sb = V.st_base[bid];
  // this colour's cut list: entry e0 + i goes to thread i (fetched while the
  // tile loads)
  const int4 cl = V.cut_list[bid];
  const int e0 = cl.x + (color ? cl.y : 0), m = color ? cl.z : cl.y;
  CutCell<T, D> cq;
  if ((int)threadIdx.x < m) cq.fetch(V, e0 + threadIdx.x);
  if (threadIdx.x < 2 * D) {
    const int a = threadIdx.x >> 1, side = threadIdx.x & 1;
    const int o[3] = {a == 0 ? 2 * side - 1 : 0, a == 1 ? 2 * side - 1 : 0, a == 2 ? 2 * side - 1 : 0};
    s_nb[threadIdx.x] = V.nbr[(size_t)bid * kNbr + nbr_slot(o[0], o[1], o[2])];
  }
  if (threadIdx.x == 0) s_fl = V.flags[bid];
  if (sb >= 0) {  // which cells of a cut block have a listed stencil
    const unsigned char *src = V.spec + sb / (2 * D + 1);
    if ((2 * G::H) % 16 == 0 && ((size_t)src & 15) == 0) {
      for (int i = threadIdx.x; i < 2 * G::H / 16; i += blockDim.x) cp_async16(sfl + 16 * i, src + 16 * i);
    } else {
      for (int i = threadIdx.x; i < 2 * G::H; i += blockDim.x) sfl[i] = src[i];
    }
  }
  // the block's own halves are in flight while the neighbour table is read
#pragma unroll
  for (int s = 0; s < SG; s++)
    if (slot[s] >= 0) {
      if constexpr (BF)
        cs_stage_interior_bf<T, D, NT>(V, L, bid, color, slot[s] * V.rs_h, slot[s] * V.rs_f, O + s * G::OS,
                                       B + s * G::H);
      else
        cs_stage_interior<T, D, NT>(V, L, bid, color, slot[s] * V.rs_phi, slot[s] * V.rs_f, O + s * G::OS,
                                    B + s * G::H);
    }
  __syncthreads();
  const int fl = s_fl;
#pragma unroll
  for (int s = 0; s < SG; s++)
    if (slot[s] >= 0) {
      if constexpr (BF)
        cs_stage_faces_bf<T, D, NT>(V, L, bid, color, s_nb, fl, slot[s] * V.rs_h, O + s * G::OS);
      else
        cs_stage_faces<T, D, NT>(V, L, bid, color, s_nb, fl, slot[s] * V.rs_phi, O + s * G::OS);
    }
  cp_async_wait_all();
  __syncthreads();
  bool special = false;
#pragma unroll
  for (int f = 0; f < 2 * D; f++) special = special || (fl & wall_bit(f >> 1, f & 1)) || s_nb[f] < 0;
  if (special) {
#pragma unroll
    for (int s = 0; s < SG; s++)
      if (slot[s] >= 0)
        cs_special_ghosts<T, D, NT, S>(V, L, Lp, bid, color, s_nb, fl, V.phi + slot[s] * V.rs_phi,
                                       Pf + slot[s] * rsP + L.poff + (long long)(bid - L.first) * (2 * G::H),
                                       O + s * G::OS);
    __syncthreads();
  }
  const T h2 = T(L.h2), inv2d = T(1.0 / (2 * D));
  const long long pown = L.poff + (long long)(bid - L.first) * (2 * G::H) + color * G::H;
  // the six neighbours of own cell j (row r, position k) in the tile
  auto nbrs = [&](int j, int *t) {
    const int r = j / G::HN, k = j - r * G::HN;
    const int y = r % NT, z = D == 3 ? r / NT : 0;
    const int q = (y + z + color) & 1;
    const int rr = G::row(y, z);
    t[0] = G::at(rr, k - 1 + q);
    t[1] = G::at(rr, k + q);
    t[2] = G::at(G::row(y - 1, z), k);
    t[3] = G::at(G::row(y + 1, z), k);
    t[4] = D == 3 ? G::at(G::row(y, z - 1), k) : 0;
    t[5] = D == 3 ? G::at(G::row(y, z + 1), k) : 0;
    return 2 * k + q + NT * (y + NT * z);  // natural index of the cell
  };
  if constexpr (std::is_same<T, float>::value) {
    // FP32 arithmetic: two cells of a row at a time, k and k + 1 (k even).
    // Their x neighbours are three consecutive tile entries, their y and z
    // neighbours and their b adjacent pairs (one 8-byte, or for BF16 one
    // 4-byte, shared load each), their results one paired store.  Each
    // cell's sum is the single-cell loop's, term for term and in the same
    // order.
    static_assert(G::RO % 2 == 0 && G::X0 % 2 == 0 && G::HN % 2 == 0, "pairs start on even tile entries");
    for (int jp = threadIdx.x; jp < G::H / 2; jp += blockDim.x) {
      const int j = 2 * jp;
      const int r = j / G::HN, k = j - r * G::HN;
      const int y = r % NT, z = D == 3 ? r / NT : 0;
      const int q = (y + z + color) & 1;
      const int cn = 2 * k + q + NT * (y + NT * z);  // natural index of the first cell
      const bool l0 = sb >= 0 && sfl[cn], l1 = sb >= 0 && sfl[cn + 2];  // listed cells
      if (l0 && l1) continue;
      const int xa = G::at(G::row(y, z), k - 1 + q);
      const int ym = G::at(G::row(y - 1, z), k), yp = G::at(G::row(y + 1, z), k);
      const int zm = D == 3 ? G::at(G::row(y, z - 1), k) : 0, zp = D == 3 ? G::at(G::row(y, z + 1), k) : 0;
#pragma unroll
      for (int s = 0; s < SG; s++) {
        if (slot[s] < 0) continue;
        const S *o = O + s * G::OS;
        const float x0 = ld_val(o[xa]), x1 = ld_val(o[xa + 1]), x2 = ld_val(o[xa + 2]);
        float a[2], b[2], c[2] = {0.f, 0.f}, d[2] = {0.f, 0.f};
        ld_pair(o + ym, a);
        ld_pair(o + yp, b);
        if (D == 3) {
          ld_pair(o + zm, c);
          ld_pair(o + zp, d);
        }
        float s0 = (x0 + x1) + (a[0] + b[0]);
        float s1 = (x1 + x2) + (a[1] + b[1]);
        if (D == 3) {
          s0 += c[0] + d[0];
          s1 += c[1] + d[1];
        }
        const float2 bb = *reinterpret_cast<const float2 *>(B + s * G::H + j);
        const float v0 = (s0 - h2 * bb.x) * inv2d, v1 = (s1 - h2 * bb.y) * inv2d;
        S *dst = Pf + slot[s] * rsP + pown + j;
        if (!l0 && !l1 && ((size_t)dst & (2 * sizeof(S) - 1)) == 0) {
          st_pair(dst, v0, v1);
        } else {
          if (!l0) dst[0] = st_val<S>(v0);
          if (!l1) dst[1] = st_val<S>(v1);
        }
      }
    }
  } else {
    for (int j = threadIdx.x; j < G::H; j += blockDim.x) {
      int t[6];
      const int cn = nbrs(j, t);
      if (sb >= 0 && sfl[cn]) continue;  // a listed cell
#pragma unroll
      for (int s = 0; s < SG; s++) {
        if (slot[s] < 0) continue;
        const S *o = O + s * G::OS;
        T sum = (ld_val(o[t[0]]) + ld_val(o[t[1]])) + (ld_val(o[t[2]]) + ld_val(o[t[3]]));
        if (D == 3) sum += ld_val(o[t[4]]) + ld_val(o[t[5]]);
        Pf[slot[s] * rsP + pown + j] = st_val<S>((sum - h2 * B[s * G::H + j]) * inv2d);
      }
    }
  }
  auto upd = [&](const CutCell<T, D> &u) {
    const int j = u.c >> 1;  // within its colour: the row pair's index
    int t[6];
    nbrs(j, t);
#pragma unroll
    for (int s = 0; s < SG; s++) {
      if (slot[s] < 0) continue;
      const S *o = O + s * G::OS;
      T sum = u.a[1] * ld_val(o[t[0]]) + u.a[2] * ld_val(o[t[1]]) + u.a[3] * ld_val(o[t[2]]) +
              u.a[4] * ld_val(o[t[3]]);
      if (D == 3) sum += u.a[5] * ld_val(o[t[4]]) + u.a[6] * ld_val(o[t[5]]);
      Pf[slot[s] * rsP + pown + j] = st_val<S>((B[s * G::H + j] - sum) / u.a[0]);
    }
  };
  if ((int)threadIdx.x < m) upd(cq);
  for (int i = threadIdx.x + blockDim.x; i < m; i += blockDim.x) {  // lists longer than the CTA
    CutCell<T, D> u;
    u.fetch(V, e0 + i);
    upd(u);
  }
}

// The half-sweep kernel: one CTA per (block, group of SG slots); the grid
// holds count x ceil(nrhs / SG) CTAs, slot groups fastest.  Frozen units
// are skipped per slot.  FP32 16^3 blocks ask for five CTAs of 256 threads
// per SM (at most 51 registers a thread; the paired loop would otherwise
// take 58 and leave four).
template <typename T, int D, int NT, int SG, bool BF = false>
__global__ void __launch_bounds__(kThreads, (NT == 16 && sizeof(T) == 4) ? 5 : 0)
    k_smooth_cs(GmgView<T> V, LvArgs L, LvArgs Lp, int color) {
  pdl_start();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ngrp = (V.nrhs + SG - 1) / SG;
  const int grp = (int)(blockIdx.x % (unsigned)ngrp);
  const int bid = L.first + (int)(blockIdx.x / (unsigned)ngrp);
  int slot[SG];
  bool any = false;
#pragma unroll
  for (int s = 0; s < SG; s++) {
    const int r = grp * SG + s;
    slot[s] = (r < V.nrhs && V.active[unit_of(V, r, bid)]) ? r : -1;
    any = any || slot[s] >= 0;
  }
  if (!any) return;
  smooth_cs_block<T, D, NT, SG, BF>(V, L, Lp, bid, slot, color, smem_raw);
}

}  // namespace gmg
