// Level kernels of the FAS V-cycle (Sec. 2.2, 3.3, 3.4).  One CTA handles
// one block: it stages the block and its ghost layer in shared memory
// (same-level neighbours, wall reflections, refinement-boundary ghosts),
// then updates the block's cells.  T is the storage/arithmetic type of the
// V-cycle (double for the FP64 path, float inside the mixed path).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gmg_internal.h"

namespace gmg {

constexpr int kThreads = 256;      // threads per CTA of the per-level kernels (at most; see cta_threads)
constexpr int kCoopThreads = 512;  // threads per CTA of the cooperative coarse cycle
constexpr int kResThreads = 256;   // threads per CTA of the residual-norm kernel (at most)

// cells of a block of side n (compile-time when n is)
#define NCELL (D == 3 ? n * n * n : n * n)

// Programmatic dependent launch: a solve-step kernel launched with the
// attribute is dispatched as soon as the previous kernel's CTAs have all
// exited, and waits here until that grid has finished and its writes are
// visible (a no-op without the attribute).  Every kernel of a solve step
// starts with this, before it reads any field.  No kernel triggers its
// dependents early: CTAs dispatched early would sit resident while they
// wait, and measured slower (2.20 ms against 2.14 ms per 128^3 solve).
__device__ __forceinline__ void pdl_start() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

// Conversions between double and float with integer operations.  A
// hardware conversion of a double runs on the FP64 pipe, which the FP64
// residual keeps busy (it is that kernel's bound on this GPU); the integer
// pipes are idle there.  Both give the IEEE 754 results bit for bit.
//
// double -> float rounded to nearest, ties to even (IEEE 754
// roundTiesToEven): for a result in float's normal range, the float keeps
// the sign, the exponent rebased from bias 1023 to bias 127 and the top 23
// of the 52 fraction bits; the 29 bits dropped round it up when they exceed
// half a unit in the last place, or equal it with the kept fraction odd (a
// carry out of the fraction raises the exponent, to infinity past the
// largest float).  Zeros keep their sign; results that are subnormal,
// infinite or NaN take the hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned int hi = (unsigned int)(u >> 32), lo = (unsigned int)u;
  const unsigned int e = (hi >> 20) & 0x7ffu, sign = hi & 0x80000000u;
  if (e - 897u > 253u) {  // float exponent e - 896 outside [1, 254]
    if ((hi & 0x7fffffffu) == 0u && lo == 0u) return __uint_as_float(sign);
    return __double2float_rn(v);
  }
  const unsigned int frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned int rest = lo & 0x1fffffffu;
  const unsigned int up = (rest > 0x10000000u || (rest == 0x10000000u && (frac & 1u))) ? 1u : 0u;
  return __uint_as_float(sign | ((((e - 896u) << 23) | frac) + up));
}

// float -> double (exact): the exponent rebased from bias 127 to bias 1023,
// the 23 fraction bits placed at the top of the 52.  Zeros keep their
// sign; subnormal, infinite and NaN inputs take the hardware conversion.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int e = (b >> 23) & 0xffu, sign = b & 0x80000000u;
  if (e - 1u > 253u) {  // not a normal float
    if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)sign, 0);
    return (double)f;
  }
  return __hiloint2double((int)(sign | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)), (int)(b << 29));
}

// The wall reflection of v (reading W): v itself for a Neumann wall, -v
// for a Dirichlet wall, by flipping the sign bit on the integer pipes (a
// double multiply by -1 would queue on the FP64 pipe); exact either way.
__device__ __forceinline__ float wall_reflect(float v, bool neumann) {
  return neumann ? v : __int_as_float(__float_as_int(v) ^ (int)0x80000000u);
}
__device__ __forceinline__ double wall_reflect(double v, bool neumann) {
  return neumann ? v : __hiloint2double(__double2hiint(v) ^ (int)0x80000000u, __double2loint(v));
}

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return f64_to_f32_rn(v); }

// BF16 storage of the FP32 correction's state on the finest level
// (GMG_MIXED_BF16): a value is kept as the top 16 bits of its float (sign,
// 8 exponent bits, 7 fraction bits), held as unsigned short.  Widening is
// exact (the low 16 bits become zero); narrowing rounds to nearest, ties to
// even (__float2bfloat16_rn).  ld_val / st_val are the identity for float
// and double, so kernels written with them compile to the same code for
// those types.
using bf16s = unsigned short;
__device__ __forceinline__ float ld_val(float v) { return v; }
__device__ __forceinline__ double ld_val(double v) { return v; }
__device__ __forceinline__ float ld_val(bf16s u) { return __uint_as_float((unsigned)u << 16); }
template <typename S>
__device__ __forceinline__ S st_val(float v) { return v; }
template <typename S>
__device__ __forceinline__ S st_val(double v) { return v; }
template <>
__device__ __forceinline__ bf16s st_val<bf16s>(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
// the wall reflection of a BF16 value: its sign bit flipped (Dirichlet)
__device__ __forceinline__ bf16s wall_reflect(bf16s v, bool neumann) { return neumann ? v : (bf16s)(v ^ 0x8000u); }

// Position of cell j of a run of whole blocks of level L (the coarsest
// level's unknowns of one root: blocks one after the other, natural cell
// order inside each, as the coarse inverse numbers them) in the fields'
// colour-split layout.
__host__ __device__ __forceinline__ int coarse_pos(int j, const LvArgs &L) {
  const int jb = j / L.ncell, jc = j - jb * L.ncell;
  const int D = L.ncell == L.n * L.n ? 2 : 3;
  return jb * L.ncell + cs_pos(jc, L.n, L.ncell, D);
}

__device__ __forceinline__ int nbr_slot(int ox, int oy, int oz) { return (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1); }

// Local coordinate p (each component in [-1, n]) of block `bid` on level L:
// axes leaving the domain are reflected with the homogeneous wall sign,
// other axes leaving the block go to the same-level neighbour.  Returns
// false when that neighbour does not exist on this level.
template <int D>
__device__ __forceinline__ bool resolve(const int *__restrict__ nbr, const int *__restrict__ flags, int wneu,
                                        const LvArgs &L, int bid, const int *pin, long long *idx, float *sign) {
  const int n = L.n;
  int p[3] = {pin[0], pin[1], pin[2]}, o[3] = {0, 0, 0};
  float sg = 1.f;
  const int fl = flags[bid];
#pragma unroll
  for (int d = 0; d < D; d++) {
    if (p[d] < 0) {
      if (fl & wall_bit(d, 0)) {
        p[d] = -1 - p[d];
        sg *= ((wneu >> (2 * d)) & 1) ? 1.f : -1.f;
      } else {
        o[d] = -1;
        p[d] += n;
      }
    } else if (p[d] >= n) {
      if (fl & wall_bit(d, 1)) {
        p[d] = 2 * n - 1 - p[d];
        sg *= ((wneu >> (2 * d + 1)) & 1) ? 1.f : -1.f;
      } else {
        o[d] = 1;
        p[d] -= n;
      }
    }
  }
  int id = bid;
  if (o[0] | o[1] | o[2]) {
    id = nbr[(size_t)bid * kNbr + nbr_slot(o[0], o[1], o[2])];
    if (id < 0) return false;
  }
  *idx = L.off + (long long)(id - L.first) * L.ncell + cs_pos_xyz(p[0], p[1], D == 3 ? p[2] : 0, n, L.ncell);
  *sign = sg;
  return true;
}

// resolve() with the block's 27 same-level neighbours already in shared
// memory (-2 marks a neighbour position outside the domain).
template <int D>
__device__ __forceinline__ bool resolve_s(const int *s_nb, int bid, const LvArgs &L, int wneu,
                                          const int *pin, long long *idx, float *sign) {
  const int n = L.n;
  int p[3] = {pin[0], pin[1], pin[2]}, o[3] = {0, 0, 0};
  float sg = 1.f;
#pragma unroll
  for (int d = 0; d < D; d++) {
    const int lo = nbr_slot(d == 0 ? -1 : 0, d == 1 ? -1 : 0, d == 2 ? -1 : 0);
    const int hi = nbr_slot(d == 0 ? 1 : 0, d == 1 ? 1 : 0, d == 2 ? 1 : 0);
    if (p[d] < 0) {
      if (s_nb[lo] == -2) {
        p[d] = -1 - p[d];
        sg *= ((wneu >> (2 * d)) & 1) ? 1.f : -1.f;
      } else {
        o[d] = -1;
        p[d] += n;
      }
    } else if (p[d] >= n) {
      if (s_nb[hi] == -2) {
        p[d] = 2 * n - 1 - p[d];
        sg *= ((wneu >> (2 * d + 1)) & 1) ? 1.f : -1.f;
      } else {
        o[d] = 1;
        p[d] -= n;
      }
    }
  }
  const int id = (o[0] | o[1] | o[2]) ? s_nb[nbr_slot(o[0], o[1], o[2])] : bid;
  if (id < 0) return false;
  *idx = L.off + (long long)(id - L.first) * L.ncell + cs_pos_xyz(p[0], p[1], D == 3 ? p[2] : 0, n, L.ncell);
  *sign = sg;
  return true;
}

// Refinement-boundary ghost (reading G): g = f/3 + 2/3 c_hat, with f the
// adjacent fine cell and c_hat the coarse cell containing the ghost centre
// shifted by central tangential slopes (+-1/4 coarse cell).
// `own` holds the block's own cells (phi, or old for a covered block in the
// FAS kernel).  The tables come as plain arguments (not the view), so that
// callers can keep a per-slot view in registers.
// `own` may be stored as BF16 (S = bf16s, the finest level of
// GMG_MIXED_BF16); the coarse level's phi is always of type T.
template <typename T, int D, typename S = T>
__device__ __noinline__ T refine_ghost(const T *phi, const int *nbr, const int *flags, const int *parent,
                                       const int *pofs_t, int wneu, const LvArgs &L, const LvArgs &Lp, int bid,
                                       const int *p, int a, const S *own) {
  const int n = L.n;
  int q[3] = {p[0], p[1], p[2]};
  q[a] = p[a] < 0 ? 0 : n - 1;
  const T f = ld_val(own[cs_pos_xyz(q[0], q[1], D == 3 ? q[2] : 0, n, L.ncell)]);
  const long long dp = Lp.poff - Lp.off;  // phi of the coarse level may live in the second buffer
  const int P = parent[bid], po = pofs_t[bid];
  const int pofs[3] = {po & 1023, (po >> 10) & 1023, (po >> 20) & 1023};
  int cq[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < D; d++) cq[d] = pofs[d] + (p[d] >> 1);
  long long ix;
  float sg;
  if (!resolve<D>(nbr, flags, wneu, Lp, P, cq, &ix, &sg)) return T(NAN);
  const T c = phi[ix + dp];
  T chat = c;
#pragma unroll
  for (int t = 0; t < D; t++) {
    if (t == a) continue;
    const T o = (p[t] & 1) ? T(0.25) : T(-0.25);
    int qp[3] = {cq[0], cq[1], cq[2]}, qm[3] = {cq[0], cq[1], cq[2]};
    qp[t] += 1;
    qm[t] -= 1;
    long long ip, im;
    float sp, sm;
    if (!resolve<D>(nbr, flags, wneu, Lp, P, qp, &ip, &sp)) return T(NAN);
    if (!resolve<D>(nbr, flags, wneu, Lp, P, qm, &im, &sm)) return T(NAN);
    const T cp = T(sp) * phi[ip + dp], cm = T(sm) * phi[im + dp];
    chat = chat + o * (T(0.5) * (cp - cm));
  }
  return f / T(3) + T(2) * chat / T(3);
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};

// Asynchronous global -> shared copies (cp.async): they take no registers,
// so a CTA can keep all of its block's loads in flight at once.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
// cp.async of NB = 4, 8 or 16 bytes (both addresses NB-aligned)
template <int NB>
__device__ __forceinline__ void cp_async_bytes(void *smem, const void *gmem) {
  static_assert(NB == 4 || NB == 8 || NB == 16, "cp.async copies 4, 8 or 16 bytes");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (NB == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
  else if (NB == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Tile of one block in shared memory: its cells plus one ghost layer.  Rows
// along x are [.. ghost x=-1 | x = 0..n-1 | ghost x=n ..] with the first cell
// at X0 = 16 / sizeof(T), so every row of cells starts on a 16-byte boundary
// (16-byte cp.async); rows are R = n + 2 X0 (+ pad) long, y and z carry one
// ghost.  FP32 rows of 8 cells get 4 more words, so that the 8 rows a warp
// touches in a half-sweep (4 cells of one colour per row) fall on 32
// different banks (row stride 20 words instead of 16).
template <typename T, int D>
struct TileGeo {
  int n, X0, R, sy, sz, size;
  static __host__ __device__ int row(int n) {
    return n + 2 * (16 / (int)sizeof(T)) + ((sizeof(T) == 4 && n == 8) ? 4 : 0);
  }
  __host__ __device__ explicit TileGeo(int n_)
      : n(n_),
        X0(16 / (int)sizeof(T)),
        R(row(n_)),
        sy(row(n_)),
        sz(row(n_) * (n_ + 2)),
        size(D == 3 ? row(n_) * (n_ + 2) * (n_ + 2) : row(n_) * (n_ + 2)) {}
  __host__ __device__ int idx(int x, int y, int z) const { return (x + X0) + sy * (y + 1) + (D == 3 ? sz * (z + 1) : 0); }
};

// Shared memory of the level kernels: the tile, the block's dense b and the
// per-cell flags of a cut block (1 = the cell's stencil differs from the
// regular one).
template <typename T>
__host__ __device__ inline size_t level_smem_bytes(int D, int n) {
  const int tile = D == 3 ? TileGeo<T, 3>(n).size : TileGeo<T, 2>(n).size;
  const int nc = D == 3 ? n * n * n : n * n;
  return sizeof(T) * (size_t)(tile + nc) + (size_t)((nc + 15) / 16 * 16);
}

// Shared memory of the residual-norm kernel: the tile and the per-cell
// flags of a cut block (b is read from global memory, once per cell).
template <typename T>
__host__ __device__ inline size_t resnorm_smem_bytes(int D, int n) {
  const int tile = D == 3 ? TileGeo<T, 3>(n).size : TileGeo<T, 2>(n).size;
  const int nc = D == 3 ? n * n * n : n * n;
  return sizeof(T) * (size_t)tile + (size_t)((nc + 15) / 16 * 16);
}

// The flags of a cut block follow its dense b in shared memory.
template <typename T>
__device__ __forceinline__ unsigned char *level_flags(T *sbv, int ncell) {
  return reinterpret_cast<unsigned char *>(sbv + ncell);
}

// Stage phi of block `bid` with its face ghosts into the tile and, if
// sbv != nullptr, the block's b into the dense array sbv[n^D], in the
// fields' colour-split order (sbv[cs_pos(c)] is cell c's).  The cells come
// as 16-byte vectors of one colour scattered into the tile, b as 16-byte
// cp.async, while the face neighbours' ids are read; the neighbours' faces
// follow as element cp.async; wall ghosts (reflection
// of the adjacent cell, homogeneous sign) and refinement-boundary ghosts
// (reading G) are filled once the copies have landed.  Ends with a barrier.
// FAS: the tile of a covered block for the FAS kernel, whose phi (and that
// of covered neighbours) the restriction left in `old` (see
// resid_restrict_block); leaf neighbours' phi is read from phi.
struct NoMid {
  __device__ void operator()() const {}
};

template <typename T, int D, int NT, bool FAS = false, typename Mid = NoMid>
__device__ __forceinline__ void load_tile(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid, T *tile,
                                          T *sbv = nullptr, unsigned char *sflag = nullptr, long long sb = -1,
                                          Mid mid = Mid()) {
  __shared__ int s_nb[6];
  __shared__ int s_fl;
  const int n = NT ? NT : L.n;
  const TileGeo<T, D> G(n);
  const int ncell = D == 3 ? n * n * n : n * n;
  if (threadIdx.x < 2 * D) {
    const int a = threadIdx.x >> 1, side = threadIdx.x & 1;
    const int o[3] = {a == 0 ? 2 * side - 1 : 0, a == 1 ? 2 * side - 1 : 0, a == 2 ? 2 * side - 1 : 0};
    s_nb[threadIdx.x] = V.nbr[(size_t)bid * kNbr + nbr_slot(o[0], o[1], o[2])];
  }
  if (threadIdx.x == 0) s_fl = V.flags[bid];
  const long long base = L.off + (long long)(bid - L.first) * ncell;   // b
  const long long pbase = L.poff + (long long)(bid - L.first) * ncell; // phi
  const T *own = FAS ? V.old + base : V.phi + pbase;  // the block's own cells
  constexpr int VEC = 16 / sizeof(T);
  // the block's run in the colour-split layout, read in order: 16-byte
  // vectors of one colour (cells x0, x0 + 2, ... of one row) scattered to
  // the tile; b kept in the run's order (the dense b is indexed by cs_pos)
  if (n % (2 * VEC) == 0) {
    using VT = typename Vec16<T>::type;
    const VT *ownv = reinterpret_cast<const VT *>(own);
    for (int i = threadIdx.x; i < ncell / VEC; i += blockDim.x) {
      if (sbv) cp_async16(sbv + i * VEC, V.b + base + i * VEC);
      const VT v = __ldcg(ownv + i);
      int x, y, z;
      cs_xyz(i * VEC, n, ncell, D, &x, &y, &z);
      const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
      for (int q = 0; q < VEC; q++) tile[G.idx(x + 2 * q, y, z)] = e[q];
    }
  } else {  // rows narrower than two vectors (coarse sub-levels)
    for (int q = threadIdx.x; q < ncell; q += blockDim.x) {
      int x, y, z;
      cs_xyz(q, n, ncell, D, &x, &y, &z);
      cp_async_elem(tile + G.idx(x, y, z), own + q);
      if (sbv) cp_async_elem(sbv + q, V.b + base + q);
    }
  }
  if (sflag && sb >= 0) {  // which cells of a cut block have a non-regular stencil
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
  const int nf = D == 3 ? n * n : n;
  // face f = 2 axis + side: ghost cell (gx,gy,gz) from the cell (qx,qy,qz) of
  // the same-level neighbour.  x faces cell by cell; the y and z faces are
  // rows along x whose two colours are each a contiguous run of n/2 cells
  // in the neighbour's block: 16-byte vectors of one colour scattered to
  // every other cell of the tile row, when a run is whole vectors.
  constexpr bool kRows = NT != 0 && NT % (2 * VEC) == 0;
  const int nfx = kRows ? 2 * nf : 2 * D * nf;
  for (int i = threadIdx.x; i < nfx; i += blockDim.x) {
    const int f = i / nf, j = i - f * nf;
    const int a = f >> 1, side = f & 1;
    const int id = s_nb[f];
    if ((fl & wall_bit(a, side)) || id < 0) continue;
    const int u = j % n, v = D == 3 ? j / n : 0;
    const int gn = side ? n : -1, sn = side ? 0 : n - 1;
    const int gx = a == 0 ? gn : u, gy = a == 1 ? gn : (a == 0 ? u : v), gz = a == 2 ? gn : v;
    const int qx = a == 0 ? sn : u, qy = a == 1 ? sn : (a == 0 ? u : v), qz = a == 2 ? sn : v;
    const T *src = (FAS && (fl & face_covered_bit(f))) ? V.old + L.off : V.phi + L.poff;
    cp_async_elem(tile + G.idx(gx, gy, gz), src + (long long)(id - L.first) * ncell + cs_pos_xyz(qx, qy, qz, n, ncell));
  }
  if (kRows) {
    using VT = typename Vec16<T>::type;
    constexpr int hn = kRows ? NT / 2 : 2;      // a row's cells of one colour
    constexpr int vpr = kRows ? hn / VEC : 1;  // vectors per colour run
    const int rows = D == 3 ? n : 1;           // rows per face
    for (int i = threadIdx.x; i < (2 * D - 2) * rows * 2 * vpr; i += blockDim.x) {
      const int f = 2 + i / (rows * 2 * vpr), rem = i - (f - 2) * rows * 2 * vpr;
      const int row = rem / (2 * vpr), cv = rem - row * 2 * vpr;
      const int col = cv / vpr, k0 = (cv - col * vpr) * VEC;  // colour of the run, first cell in it
      const int a = f >> 1, side = f & 1;
      const int id = s_nb[f];
      if ((fl & wall_bit(a, side)) || id < 0) continue;
      const int gn = side ? n : -1, sn = side ? 0 : n - 1;
      const int gy = a == 1 ? gn : row, gz = a == 2 ? gn : (D == 3 ? row : 0);
      const int qy = a == 1 ? sn : row, qz = a == 2 ? sn : (D == 3 ? row : 0);
      const T *src = (FAS && (fl & face_covered_bit(f))) ? V.old + L.off : V.phi + L.poff;
      const VT w = __ldcg(reinterpret_cast<const VT *>(src + (long long)(id - L.first) * ncell + col * (ncell / 2) +
                                                        hn * (qy + (D == 3 ? n * qz : 0)) + k0));
      const int x0 = 2 * k0 + ((qy + qz + col) & 1);  // x of the run's first cell (same x in the ghost row)
      const T *e = reinterpret_cast<const T *>(&w);
#pragma unroll
      for (int q = 0; q < VEC; q++) tile[G.idx(x0 + 2 * q, gy, gz)] = e[q];
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // faces with a wall or a refinement boundary (same list in every thread)
  // (face ids packed 4 bits each, so that the list stays in a register)
  unsigned sf = 0;
  int nsf = 0;
#pragma unroll
  for (int f = 0; f < 2 * D; f++)
    if ((fl & wall_bit(f >> 1, f & 1)) || s_nb[f] < 0) sf |= (unsigned)f << (4 * nsf++);
  if (nsf == 0) return;  // every ghost came from a same-level neighbour
  for (int i = threadIdx.x; i < nsf * nf; i += blockDim.x) {
    const int k = i / nf, j = i - k * nf;
    const int f = (int)((sf >> (4 * k)) & 15u);
    const int a = f >> 1, side = f & 1;
    const bool wall = (fl & wall_bit(a, side)) != 0;
    const int u = j % n, v = D == 3 ? j / n : 0;
    const int gn = side ? n : -1, mn = side ? n - 1 : 0;
    const int gx = a == 0 ? gn : u, gy = a == 1 ? gn : (a == 0 ? u : v), gz = a == 2 ? gn : v;
    T val;
    if (wall) {
      const int mx = a == 0 ? mn : u, my = a == 1 ? mn : (a == 0 ? u : v), mz = a == 2 ? mn : v;
      val = wall_reflect(tile[G.idx(mx, my, mz)], (V.wneu >> f) & 1);
    } else {
      const int g[3] = {gx, gy, gz};
      val = refine_ghost<T, D>(V.phi, V.nbr, V.flags, V.parent, V.pofs, V.wneu, L, Lp, bid, g, a, own);
    }
    tile[G.idx(gx, gy, gz)] = val;
  }
  __syncthreads();
}

// PW BF16 values in one load (16, 8, 4 or 2 bytes)
template <int PW>
struct BfVec;
template <>
struct BfVec<8> {
  using type = uint4;
};
template <>
struct BfVec<4> {
  using type = uint2;
};
template <>
struct BfVec<2> {
  using type = unsigned int;
};
template <>
struct BfVec<1> {
  using type = unsigned short;
};

// load_tile for a level whose phi is stored as BF16 (the finest level of
// GMG_MIXED_BF16; compiled block sides only): the same tile of T values,
// widened on the way in.  The block's run is read in pieces of PW cells of
// one colour of one row (16 bytes when a row's colour half allows), b as
// 16-byte cp.async in the run's order, the face ghosts by plain loads, then
// wall and refinement-boundary ghosts as in load_tile.  Ends with a barrier.
template <typename T, int D, int NT, typename Mid = NoMid>
__device__ __forceinline__ void load_tile_h(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid, T *tile,
                                            T *sbv, unsigned char *sflag, long long sb, Mid mid = Mid()) {
  static_assert(NT != 0, "BF16 levels have a compiled block side");
  __shared__ int s_nb[6];
  __shared__ int s_fl;
  constexpr int n = NT, HN = NT / 2;
  constexpr int ncell = D == 3 ? n * n * n : n * n;
  constexpr int PW = HN % 8 == 0 ? 8 : (HN % 4 == 0 ? 4 : (HN % 2 == 0 ? 2 : 1));
  const TileGeo<T, D> G(n);
  if (threadIdx.x < 2 * D) {
    const int a = threadIdx.x >> 1, side = threadIdx.x & 1;
    const int o[3] = {a == 0 ? 2 * side - 1 : 0, a == 1 ? 2 * side - 1 : 0, a == 2 ? 2 * side - 1 : 0};
    s_nb[threadIdx.x] = V.nbr[(size_t)bid * kNbr + nbr_slot(o[0], o[1], o[2])];
  }
  if (threadIdx.x == 0) s_fl = V.flags[bid];
  const long long base = L.off + (long long)(bid - L.first) * ncell;    // b
  const long long pbase = L.poff + (long long)(bid - L.first) * ncell;  // phi, level-local
  const bf16s *own = V.hphi + pbase;
  constexpr int VEC = 16 / sizeof(T);
  if (ncell % VEC == 0) {
    for (int i = threadIdx.x; i < ncell / VEC; i += blockDim.x) cp_async16(sbv + i * VEC, V.b + base + i * VEC);
  } else {
    for (int q = threadIdx.x; q < ncell; q += blockDim.x) cp_async_elem(sbv + q, V.b + base + q);
  }
  using PV = typename BfVec<PW>::type;
  for (int i = threadIdx.x; i < ncell / PW; i += blockDim.x) {
    const PV v = __ldcg(reinterpret_cast<const PV *>(own) + i);
    int x, y, z;
    cs_xyz(i * PW, n, ncell, D, &x, &y, &z);
    const bf16s *e = reinterpret_cast<const bf16s *>(&v);
#pragma unroll
    for (int q = 0; q < PW; q++) tile[G.idx(x + 2 * q, y, z)] = ld_val(e[q]);
  }
  if (sflag && sb >= 0) {  // which cells of a cut block have a non-regular stencil
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
  constexpr int nf = D == 3 ? n * n : n;
  for (int i = threadIdx.x; i < 2 * D * nf; i += blockDim.x) {
    const int f = i / nf, j = i - f * nf;
    const int a = f >> 1, side = f & 1;
    const int id = s_nb[f];
    if ((fl & wall_bit(a, side)) || id < 0) continue;
    const int u = j % n, v = D == 3 ? j / n : 0;
    const int gn = side ? n : -1, sn = side ? 0 : n - 1;
    const int gx = a == 0 ? gn : u, gy = a == 1 ? gn : (a == 0 ? u : v), gz = a == 2 ? gn : v;
    const int qx = a == 0 ? sn : u, qy = a == 1 ? sn : (a == 0 ? u : v), qz = a == 2 ? sn : v;
    tile[G.idx(gx, gy, gz)] =
        ld_val(V.hphi[L.poff + (long long)(id - L.first) * ncell + cs_pos_xyz(qx, qy, qz, n, ncell)]);
  }
  cp_async_wait_all();
  __syncthreads();
  unsigned sf = 0;
  int nsf = 0;
#pragma unroll
  for (int f = 0; f < 2 * D; f++)
    if ((fl & wall_bit(f >> 1, f & 1)) || s_nb[f] < 0) sf |= (unsigned)f << (4 * nsf++);
  if (nsf == 0) return;
  for (int i = threadIdx.x; i < nsf * nf; i += blockDim.x) {
    const int k = i / nf, j = i - k * nf;
    const int f = (int)((sf >> (4 * k)) & 15u);
    const int a = f >> 1, side = f & 1;
    const bool wall = (fl & wall_bit(a, side)) != 0;
    const int u = j % n, v = D == 3 ? j / n : 0;
    const int gn = side ? n : -1, mn = side ? n - 1 : 0;
    const int gx = a == 0 ? gn : u, gy = a == 1 ? gn : (a == 0 ? u : v), gz = a == 2 ? gn : v;
    T val;
    if (wall) {
      const int mx = a == 0 ? mn : u, my = a == 1 ? mn : (a == 0 ? u : v), mz = a == 2 ? mn : v;
      val = wall_reflect(tile[G.idx(mx, my, mz)], (V.wneu >> f) & 1);
    } else {
      const int g[3] = {gx, gy, gz};
      val = refine_ghost<T, D>(V.phi, V.nbr, V.flags, V.parent, V.pofs, V.wneu, L, Lp, bid, g, a, own);
    }
    tile[G.idx(gx, gy, gz)] = val;
  }
  __syncthreads();
}

template <typename T, int D>
__device__ __forceinline__ T nb_sum(const T *tile, int t, int sy, int sz) {
  T s = (tile[t - 1] + tile[t + 1]) + (tile[t - sy] + tile[t + sy]);
  if (D == 3) s += tile[t - sz] + tile[t + sz];
  return s;
}

// Off-diagonal sum of a stored stencil a[0 .. 2D] (diagonal first, then the
// faces -x, +x, -y, +y, -z, +z) at tile index t.
template <typename T, int D>
__device__ __forceinline__ T offdiag_of(const T *a, const T *tile, int t, int sy, int sz) {
  T s = a[1] * tile[t - 1] + a[2] * tile[t + 1] + a[3] * tile[t - sy] + a[4] * tile[t + sy];
  if (D == 3) s += a[5] * tile[t - sz] + a[6] * tile[t + sz];
  return s;
}

// Off-diagonal sum and diagonal of cell c from a stencil array with
// coefficient k at st[k * ncell + c].
template <typename T, int D>
__device__ __forceinline__ T offdiag_st(const T *__restrict__ st, const T *tile, int t, int sy, int sz, int ncell,
                                        int c, T *diag) {
  T cf[2 * D + 1];
#pragma unroll
  for (int k = 0; k < 2 * D + 1; k++) cf[k] = st[k * ncell + c];
  *diag = cf[0];
  return offdiag_of<T, D>(cf, tile, t, sy, sz);
}

// One entry of a cut list in registers: the cell (index in its block) and
// its 2D + 1 coefficients.  A CTA fetches its block's entries while the
// tile loads, so that no cell waits on a stencil read.
template <typename T, int D>
struct CutCell {
  int c;
  T a[2 * D + 1];
  __device__ __forceinline__ void fetch(const GmgView<T> &V, long long e) {
    c = V.cut_cell[e];
#pragma unroll
    for (int k = 0; k < 2 * D + 1; k++) a[k] = V.cut_coef[k * V.n_cut + e];
  }
};

// r = b - A phi at cell c (tile index t); the regular 5/7-point form costs
// 2D - 1 adds and two fused multiply-adds (FP64 throughput bounds that path).
template <typename T, int D>
__device__ __forceinline__ T resid_cell(const T *__restrict__ st, long long sb, const T *tile, int t, int sy, int sz,
                                        int ncell, int c, T inv_h2, T b) {
  if (sb < 0) return b - inv_h2 * (nb_sum<T, D>(tile, t, sy, sz) - T(2 * D) * tile[t]);
  T diag;
  const T s = offdiag_st<T, D>(st + sb, tile, t, sy, sz, ncell, c, &diag);
  return b - (diag * tile[t] + s);
}

template <int D>
__device__ __forceinline__ void cell_xyz(int c, int n, int *x, int *y, int *z) {
  *x = c % n;
  *y = (c / n) % n;
  *z = D == 3 ? c / (n * n) : 0;
}

// (x, y, z) of cell c of a block of side n: shifts and masks when n is a
// power of two, divisions otherwise
template <int D>
__device__ __forceinline__ void cell_xyz_rt(int c, int n, int *x, int *y, int *z) {
  if ((n & (n - 1)) == 0) {
    const int lg = __ffs(n) - 1;
    *x = c & (n - 1);
    *y = (c >> lg) & (n - 1);
    *z = D == 3 ? c >> (2 * lg) : 0;
  } else {
    cell_xyz<D>(c, n, x, y, z);
  }
}

// the j-th cell of colour `color` ((x + y + z) mod 2) of a block of side n
template <int D>
__device__ __forceinline__ void colour_xyz(int j, int n, int color, int *x, int *y, int *z) {
  const int hn = n / 2;
  int xp;
  if ((n & (n - 1)) == 0) {
    const int lh = __ffs(hn) - 1;
    xp = j & (hn - 1);
    const int rest = j >> lh;
    *y = rest & (n - 1);
    *z = D == 3 ? rest >> (lh + 1) : 0;
  } else {
    xp = j % hn;
    const int rest = j / hn;
    *y = rest % n;
    *z = D == 3 ? rest / n : 0;
  }
  *x = 2 * xp + ((*y + *z + color) & 1);
}

// Work item of a per-level launch: the grid holds count x nrhs CTAs with the
// slot index fastest, so that the slots of one block run side by side and
// share its tables and stencil through L2.  Returns false for a frozen unit
// (slot, or slot and tree of a forest).
template <typename T>
__device__ __forceinline__ bool slot_item(const GmgView<T> &V, const LvArgs &L, int *bid, GmgView<T> *W) {
  const int r = (int)(blockIdx.x % (unsigned)V.nrhs);
  *bid = L.first + (int)(blockIdx.x / (unsigned)V.nrhs);
  if (!V.active[unit_of(V, r, *bid)]) return false;
  *W = slot_view(V, r);
  return true;
}

// One red (color 0) or black (color 1) half-sweep of Gauss-Seidel on every
// block of a level (Sec. 2.2, readings S and SW):
// phi_i <- (b_i - sum_j c_ij phi_j) / c_ii on the cells of one colour.
template <typename T, int D, int NT>
__device__ void smooth_block(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid, int color, unsigned char *smem_raw) {
  const int n = NT ? NT : L.n, hn = n / 2;
  const TileGeo<T, D> G(n);
  T *tile = reinterpret_cast<T *>(smem_raw);
  T *sbv = tile + G.size;
  unsigned char *sfl = level_flags(sbv, NCELL);
  const long long pbase = L.poff + (long long)(bid - L.first) * NCELL;
  const long long sb = V.st_base[bid];
  // this colour's cut list: entry e0 + i goes to thread i (prefetched)
  const int4 cl = V.cut_list[bid];
  const int e0 = cl.x + (color ? cl.y : 0), m = color ? cl.z : cl.y;
  CutCell<T, D> q;
  load_tile<T, D, NT>(V, L, Lp, bid, tile, sbv, sfl, sb, [&] {
    if ((int)threadIdx.x < m) q.fetch(V, e0 + threadIdx.x);
  });
  const T h2 = T(L.h2), inv2d = T(1.0 / (2 * D));
  const int nhalf = NCELL / 2;
  for (int j = threadIdx.x; j < nhalf; j += blockDim.x) {
    const int rest = j / hn;
    const int y = rest % n, z = D == 3 ? rest / n : 0;
    const int x = 2 * (j % hn) + ((y + z + color) & 1);
    const int c = x + n * (y + n * z);
    if (sb >= 0 && sfl[c]) continue;  // a listed cell
    const int q = cs_pos_xyz(x, y, z, n, NCELL);
    V.phi[pbase + q] = (nb_sum<T, D>(tile, G.idx(x, y, z), G.sy, G.sz) - h2 * sbv[q]) * inv2d;
  }
  auto upd = [&](const CutCell<T, D> &u) {
    int x, y, z;
    cell_xyz<D>(u.c, n, &x, &y, &z);
    const int t = G.idx(x, y, z);
    const int q = cs_pos_xyz(x, y, z, n, NCELL);
    V.phi[pbase + q] = (sbv[q] - offdiag_of<T, D>(u.a, tile, t, G.sy, G.sz)) / u.a[0];
  };
  if ((int)threadIdx.x < m) upd(q);
  for (int i = threadIdx.x + blockDim.x; i < m; i += blockDim.x) {  // lists longer than the CTA
    CutCell<T, D> u;
    u.fetch(V, e0 + i);
    upd(u);
  }
}

template <typename T, int D, int NT>
__global__ void __launch_bounds__(kThreads) k_smooth(GmgView<T> V, LvArgs L, LvArgs Lp, int color) {
  pdl_start();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int bid;
  GmgView<T> W;
  if (!slot_item(V, L, &bid, &W)) return;
  smooth_block<T, D, NT>(W, L, Lp, bid, color, smem_raw);
}

// Residuals of a block's listed cells (both colours) in place of their b
// in shared memory: sbv[c] <- b_c - (diag phi_c + off-diagonal sum), the
// stencil branch of resid_cell.  Entry i of thread i arrives prefetched in
// q; longer lists are fetched here.  Ends with a barrier when the block has
// a list (m is the same in every thread).
template <typename T, int D>
__device__ __forceinline__ void cut_residuals(const GmgView<T> &V, const TileGeo<T, D> &G, int n, const T *tile,
                                              T *sbv, int4 cl, const CutCell<T, D> &q) {
  const int m = cl.y + cl.z;
  if (m == 0) return;
  auto res = [&](const CutCell<T, D> &u) {
    int x, y, z;
    cell_xyz<D>(u.c, n, &x, &y, &z);
    const int t = G.idx(x, y, z);
    const int q = cs_pos_xyz(x, y, z, n, D == 3 ? n * n * n : n * n);
    sbv[q] = sbv[q] - (u.a[0] * tile[t] + offdiag_of<T, D>(u.a, tile, t, G.sy, G.sz));
  };
  const int i = threadIdx.x, bd = blockDim.x;
  if (i < m) res(q);
  for (int k = i + bd; k < m; k += bd) {
    CutCell<T, D> u;
    u.fetch(V, cl.x + k);
    res(u);
  }
  __syncthreads();
}

// Residual r = b - A phi (Eq. (residual)) of every cell, restricted to the
// parent as the mean of the 2^D children, together with phi (Sec. 2.2):
// parent phi <- mean phi, parent b <- mean r (the FAS kernel adds A phi).
// The restricted phi goes to the parent level's `old` field (dead until the
// FAS kernel sets it): other CTAs of this launch may still read the parent
// level's phi for their refinement-boundary ghosts, and must see the values
// from before the restriction, as the sequential order has it.
// H: the level's phi is stored as BF16 (load_tile_h).
template <typename T, int D, int NT, bool H = false>
__device__ void resid_restrict_block(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid, unsigned char *smem_raw) {
  const int n = NT ? NT : L.n, hn = n / 2;
  const TileGeo<T, D> G(n);
  T *tile = reinterpret_cast<T *>(smem_raw);
  T *sbv = tile + G.size;
  unsigned char *sfl = level_flags(sbv, NCELL);
  const long long sb = V.st_base[bid];
  const int P = V.parent[bid], po = V.pofs[bid];
  const int4 cl = V.cut_list[bid];
  const int m = cl.y + cl.z;
  CutCell<T, D> q;
  auto prefetch = [&] {
    if ((int)threadIdx.x < m) q.fetch(V, cl.x + threadIdx.x);
  };
  if constexpr (H)
    load_tile_h<T, D, NT>(V, L, Lp, bid, tile, sbv, sfl, sb, prefetch);
  else
    load_tile<T, D, NT>(V, L, Lp, bid, tile, sbv, sfl, sb, prefetch);
  cut_residuals<T, D>(V, G, n, tile, sbv, cl, q);
  const T inv_h2 = T(L.ih2);
  const int pofs[3] = {po & 1023, (po >> 10) & 1023, (po >> 20) & 1023};
  const long long pbase = Lp.off + (long long)(P - Lp.first) * Lp.ncell;
  const int pn = Lp.n;
  const int ncq = D == 3 ? hn * hn * hn : hn * hn;
  const T w = T(1.0 / (1 << D));
  for (int j = threadIdx.x; j < ncq; j += blockDim.x) {
    const int qx = j % hn, qy = (j / hn) % hn, qz = D == 3 ? j / (hn * hn) : 0;
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
          sp = sp + tile[t];
          const int p = cs_pos_xyz(x, y, z, n, NCELL);
          sr = sr + ((sb >= 0 && sfl[c]) ? sbv[p]  // a listed cell: its residual
                                         : resid_cell<T, D>(nullptr, -1, tile, t, G.sy, G.sz, NCELL, c, inv_h2, sbv[p]));
        }
    const long long pc = pbase + cs_pos_xyz(pofs[0] + qx, pofs[1] + qy, D == 3 ? pofs[2] + qz : 0, pn, Lp.ncell);
    V.old[pc] = sp * w;
    V.b[pc] = sr * w;
  }
}

template <typename T, int D, int NT, bool H = false>
__global__ void __launch_bounds__(kThreads) k_resid_restrict(GmgView<T> V, LvArgs L, LvArgs Lp) {
  pdl_start();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int bid;
  GmgView<T> W;
  if (!slot_item(V, L, &bid, &W)) return;
  resid_restrict_block<T, D, NT, H>(W, L, Lp, bid, smem_raw);
}

// FAS coarse right-hand side on covered cells: b <- A phi + (restricted r);
// old <- phi on every cell of the level (start of the coarse visit).  A
// covered block's restricted phi arrives in old (resid_restrict_block) and
// is copied to phi here; covered neighbours' ghosts are read from old too.
template <typename T, int D, int NT>
__device__ void fas_block(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid, unsigned char *smem_raw) {
  const int n = NT ? NT : L.n;
  const TileGeo<T, D> G(n);
  const long long base = L.off + (long long)(bid - L.first) * NCELL;
  if (!(V.flags[bid] & kHasChildren)) {
    constexpr int VEC = 16 / sizeof(T);
    using VT = typename Vec16<T>::type;
    const VT *src = reinterpret_cast<const VT *>(V.phi + (L.poff - L.off) + base);
    VT *dst = reinterpret_cast<VT *>(V.old + base);
    for (int i = threadIdx.x; i < NCELL / VEC; i += blockDim.x) dst[i] = src[i];
    return;
  }
  T *tile = reinterpret_cast<T *>(smem_raw);
  T *sbv = tile + G.size;
  unsigned char *sfl = level_flags(sbv, NCELL);
  const long long sb = V.st_base[bid];
  const int4 cl = V.cut_list[bid];
  const int m = cl.y + cl.z;
  CutCell<T, D> q;
  load_tile<T, D, NT, true>(V, L, Lp, bid, tile, sbv, sfl, sb, [&] {
    if ((int)threadIdx.x < m) q.fetch(V, cl.x + threadIdx.x);
  });
  if (m) {  // listed cells: sbv[c] <- A phi + sbv[c] with the stored stencil
    auto fas = [&](const CutCell<T, D> &u) {
      int x, y, z;
      cell_xyz<D>(u.c, n, &x, &y, &z);
      const int t = G.idx(x, y, z);
      const int q = cs_pos_xyz(x, y, z, n, NCELL);
      sbv[q] = (u.a[0] * tile[t] + offdiag_of<T, D>(u.a, tile, t, G.sy, G.sz)) + sbv[q];
    };
    const int i = threadIdx.x, bd = blockDim.x;
    if (i < m) fas(q);
    for (int k = i + bd; k < m; k += bd) {
      CutCell<T, D> u;
      u.fetch(V, cl.x + k);
      fas(u);
    }
    __syncthreads();
  }
  const T inv_h2 = T(L.ih2);
  const long long pbase = L.poff + (long long)(bid - L.first) * NCELL;
  for (int c = threadIdx.x; c < NCELL; c += blockDim.x) {
    int x, y, z;
    cell_xyz<D>(c, n, &x, &y, &z);
    const int t = G.idx(x, y, z);
    const T ph = tile[t];
    const int q = cs_pos_xyz(x, y, z, n, NCELL);
    V.b[base + q] = (sb >= 0 && sfl[c]) ? sbv[q] : inv_h2 * (nb_sum<T, D>(tile, t, G.sy, G.sz) - T(2 * D) * ph) + sbv[q];
    V.phi[pbase + q] = ph;  // old already holds ph
  }
}

template <typename T, int D, int NT>
__global__ void __launch_bounds__(kThreads) k_fas(GmgView<T> V, LvArgs L, LvArgs Lp) {
  pdl_start();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int bid;
  GmgView<T> W;
  if (!slot_item(V, L, &bid, &W)) return;
  fas_block<T, D, NT>(W, L, Lp, bid, smem_raw);
}

// Coarsest level: phi = A^-1 b with the FP64 inverse of each root's
// operator (block-diagonal over the nroot independent roots), one warp per
// row and slot.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_coarse(GmgView<T> V, LvArgs Lc, const double *__restrict__ Ainv,
                                                     int ncr, int nroot) {
  pdl_start();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long item = (long long)blockIdx.x * (kThreads / 32) + warp;
  const int M = ncr * nroot;
  if (item >= (long long)M * V.nrhs) return;
  const int r = (int)(item / M), row = (int)(item % M);
  const int k = row / ncr, i = row - k * ncr;
  if (!V.active[V.ntree > 1 ? r * V.ntree + k : r]) return;  // root k = tree k of a forest
  const double *a = Ainv + ((size_t)k * ncr + i) * ncr;
  const T *b = V.b + r * V.rs_f + Lc.off + (size_t)k * ncr;
  double s = 0.0;
  for (int j = lane; j < ncr; j += 32) s += a[j] * (double)b[coarse_pos(j, Lc)];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) V.phi[r * V.rs_phi + Lc.poff + (size_t)k * ncr + coarse_pos(i, Lc)] = T(s);
}

// (Bi/tri)linear prolongation of the coarse correction phi - old
// (Sec. 2.2, 3.4): weights 3/4 and 1/4 per dimension from the parent cell
// and its neighbours toward the fine cell (reading P).  The block's own
// cells are held in registers, sized for CTAs of at least PT threads.
// H: the fine level's phi is stored as BF16 (read, corrected in T, rounded
// back).
template <typename T, int D, int NT, int PT = kThreads, bool H = false>
__device__ void prolong_block(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid, unsigned char *smem_raw) {
  __shared__ int s_nb[kNbr];
  T *tile = reinterpret_cast<T *>(smem_raw);
  const int n = NT ? NT : L.n, hn = n / 2, m = hn + 2;
  // the parent's 27 same-level neighbours (precomputed per block), -2 outside
  if (threadIdx.x < kNbr) s_nb[threadIdx.x] = V.pnb[(size_t)bid * kNbr + threadIdx.x];
  const int P = V.parent[bid], po = V.pofs[bid];
  // the block's own phi, loaded while the coarse correction is staged
  constexpr int VEC = 16 / sizeof(T);
  using VT = typename Vec16<T>::type;
  const long long base = L.poff + (long long)(bid - L.first) * NCELL;
  VT *__restrict__ fine = reinterpret_cast<VT *>(V.phi + base);
  uint2 *__restrict__ fineh = H ? reinterpret_cast<uint2 *>(V.hphi + base) : nullptr;  // 4 BF16 a vector
  static_assert(!H || VEC == 4, "BF16 levels are FP32 levels");
  // vectors in pairs: vector i of the red half and vector i of the black
  // half hold the two colours of the same 2 VEC consecutive cells of a row
  // (when a row's colour half is whole vectors)
  constexpr bool kPairs = NT != 0 && NT % (2 * VEC) == 0;
  constexpr int HV = NT ? (D == 3 ? NT * NT * NT : NT * NT) / 2 / VEC : 1;  // vectors of one colour
  constexpr int IV = kPairs ? (HV + PT - 1) / PT : 1;
  VT rv[IV], rw[IV];
  if (kPairs) {
#pragma unroll
    for (int k = 0; k < IV; k++) {
      const int i = threadIdx.x + k * blockDim.x;
      if (i < HV) {
        if constexpr (H) {
          const uint2 a = fineh[i], b = fineh[HV + i];
          rv[k] = make_float4(ld_val((bf16s)(a.x & 0xffffu)), ld_val((bf16s)(a.x >> 16)),
                              ld_val((bf16s)(a.y & 0xffffu)), ld_val((bf16s)(a.y >> 16)));
          rw[k] = make_float4(ld_val((bf16s)(b.x & 0xffffu)), ld_val((bf16s)(b.x >> 16)),
                              ld_val((bf16s)(b.y & 0xffffu)), ld_val((bf16s)(b.y >> 16)));
        } else {
          rv[k] = fine[i];
          rw[k] = fine[HV + i];
        }
      }
    }
  }
  __syncthreads();
  const int pofs[3] = {po & 1023, (po >> 10) & 1023, (po >> 20) & 1023};
  const int tsize = D == 3 ? m * m * m : m * m;
  for (int t = threadIdx.x; t < tsize; t += blockDim.x) {
    int q[3] = {pofs[0] - 1 + t % m, pofs[1] - 1 + (t / m) % m, D == 3 ? pofs[2] - 1 + t / (m * m) : 0};
    long long ix;
    float sg;
    T v = T(NAN);
    if (resolve_s<D>(s_nb, P, Lp, V.wneu, q, &ix, &sg)) v = T(sg) * (V.phi[ix + (Lp.poff - Lp.off)] - V.old[ix]);
    tile[t] = v;
  }
  __syncthreads();
  // fine cell (x,y,z): parent cell u = (x/2,...) + 1 in tile coordinates,
  // the interpolation partner on the side of the fine cell's centre
  auto interp = [&](int x, int y, int z) {
    const int u[3] = {(x >> 1) + 1, (y >> 1) + 1, (z >> 1) + 1};
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
          const int tx = u[0] + sx * o[0], ty = u[1] + sy * o[1], tz = D == 3 ? u[2] + sz * o[2] : 0;
          v = v + wgt * tile[tx + m * (ty + (D == 3 ? m * tz : 0))];
        }
    return v;
  };
  if (kPairs) {
#pragma unroll
    for (int k = 0; k < IV; k++) {
      const int i = threadIdx.x + k * blockDim.x;
      if (i < HV) {
        T *e0 = reinterpret_cast<T *>(&rv[k]);  // red cells x0 + 2q (x0 = first red x)
        T *e1 = reinterpret_cast<T *>(&rw[k]);  // black cells x0 + 1 - 2 (x0 & 1) + 2q
        int x, y, z;
        cs_xyz(i * VEC, n, NCELL, D, &x, &y, &z);
        const int xe = x & ~1;                  // the pair's even cell
#pragma unroll
        for (int q = 0; q < VEC; q++) {         // cells xe + 2q and xe + 2q + 1, in x order
          const T a = interp(xe + 2 * q, y, z), b = interp(xe + 2 * q + 1, y, z);
          if (x & 1) {
            e1[q] += a;
            e0[q] += b;
          } else {
            e0[q] += a;
            e1[q] += b;
          }
        }
        if constexpr (H) {
          auto pack = [](float lo, float hi) {
            return (unsigned)st_val<bf16s>(lo) | ((unsigned)st_val<bf16s>(hi) << 16);
          };
          fineh[i] = make_uint2(pack(rv[k].x, rv[k].y), pack(rv[k].z, rv[k].w));
          fineh[HV + i] = make_uint2(pack(rw[k].x, rw[k].y), pack(rw[k].z, rw[k].w));
        } else {
          fine[i] = rv[k];
          fine[HV + i] = rw[k];
        }
      }
    }
  } else {
    for (int q = threadIdx.x; q < NCELL; q += blockDim.x) {
      int x, y, z;
      cs_xyz(q, n, NCELL, D, &x, &y, &z);
      if constexpr (H)
        V.hphi[base + q] = st_val<bf16s>(ld_val(V.hphi[base + q]) + interp(x, y, z));
      else
        V.phi[base + q] += interp(x, y, z);
    }
  }
}

template <typename T, int D, int NT, int PT, bool H = false>
__global__ void __launch_bounds__(PT) k_prolong(GmgView<T> V, LvArgs L, LvArgs Lp) {
  pdl_start();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int bid;
  GmgView<T> W;
  if (!slot_item(V, L, &bid, &W)) return;
  prolong_block<T, D, NT, PT, H>(W, L, Lp, bid, smem_raw);
}

// phi of covered cells <- mean of the children (composite consistency).
// H: the fine level's phi is stored as BF16.
template <typename T, int D, int NT, bool H = false>
__global__ void __launch_bounds__(kThreads) k_restrict_phi(GmgView<T> V0, LvArgs L, LvArgs Lp) {
  pdl_start();
  int bid;
  GmgView<T> V;
  if (!slot_item(V0, L, &bid, &V)) return;
  const int n = NT ? NT : L.n, hn = n / 2;
  const long long base = L.poff + (long long)(bid - L.first) * NCELL;
  const int P = V.parent[bid], po = V.pofs[bid];
  const int pofs[3] = {po & 1023, (po >> 10) & 1023, (po >> 20) & 1023};
  const long long pbase = Lp.poff + (long long)(P - Lp.first) * Lp.ncell;
  const int pn = Lp.n;
  const int ncq = D == 3 ? hn * hn * hn : hn * hn;
  const T w = T(1.0 / (1 << D));
  for (int j = threadIdx.x; j < ncq; j += blockDim.x) {
    const int qx = j % hn, qy = (j / hn) % hn, qz = D == 3 ? j / (hn * hn) : 0;
    T sp = T(0);
    for (int dz = 0; dz < (D == 3 ? 2 : 1); dz++)
      for (int dy = 0; dy < 2; dy++)
        for (int dx = 0; dx < 2; dx++) {
          const long long f = base + cs_pos_xyz(2 * qx + dx, 2 * qy + dy, 2 * qz + dz, n, NCELL);
          if constexpr (H)
            sp = sp + ld_val(V.hphi[f]);
          else
            sp = sp + V.phi[f];
        }
    V.phi[pbase + cs_pos_xyz(pofs[0] + qx, pofs[1] + qy, D == 3 ? pofs[2] + qz : 0, pn, Lp.ncell)] = sp * w;
  }
}

// Block reduction of (sum r^2, max |r|, sum b^2) into out[0..2] (CTAs of
// up to kResThreads threads).
__device__ __forceinline__ void block_reduce3(double s2, double mx, double b2, double *out) {
  __shared__ double red[3][kResThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    b2 += __shfl_xor_sync(0xffffffffu, b2, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    red[0][warp] = s2;
    red[1][warp] = mx;
    red[2][warp] = b2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); i++) {
      a += red[0][i];
      b = fmax(b, red[1][i]);
      c += red[2][i];
    }
    out[0] = a;
    out[1] = b;
    out[2] = c;
  }
}

// The final norm reduction folded into the residual launch (when it is the
// step's only residual launch, with kResThreads threads a CTA): each CTA
// counts itself in after writing its partials, and the last one reduces
// every unit's partials exactly as k_reduce_partials does (same threads,
// same order: the same bits), then re-arms the counter.
struct ResFold {
  unsigned int *counter;  // 0 between launches
  double *out;            // [units][4]: sum r^2, max |r|, sum b^2, barrier error
  const int *tree_blocks, *tree_boff;
  const int *err;         // the coarse cycle's barrier error word
  int ntree, units, on;
};

__device__ __forceinline__ void fold_norms(const ResFold &F, const double *partials0, int nbt) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's partials before its arrival
    s_last = atomicAdd(F.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int u = 0; u < F.units; u++) {
    const int r = u / F.ntree, tr = u % F.ntree;
    const double *p = partials0 + (size_t)r * nbt * 3;
    const int b0 = F.tree_boff[tr], b1 = F.tree_boff[tr + 1];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = b0 + threadIdx.x; k < b1; k += blockDim.x) {
      const size_t i = (size_t)F.tree_blocks[k];
      a += __ldcg(p + i * 3);
      b = fmax(b, __ldcg(p + i * 3 + 1));
      c += __ldcg(p + i * 3 + 2);
    }
    block_reduce3(a, b, c, F.out + (size_t)u * 4);
    if (threadIdx.x == 0) F.out[(size_t)u * 4 + 3] = F.err ? (double)*F.err : 0.0;
    __syncthreads();  // block_reduce3's shared words serve the next unit
  }
  if (threadIdx.x == 0) *F.counter = 0u;
}

// Residual norms over the leaf blocks of a level (reading R); with `rout`
// the residual itself is written as float (right-hand side of the FP32
// correction V-cycle in the mixed path).  With F.on, the final reduction
// follows in the last CTA (fold_norms).
template <typename T, int D, int NT>
__device__ __forceinline__ void resnorm_block(const GmgView<T> &V0, const LvArgs &L, const LvArgs &Lp,
                                              double *partials, float *rout, int nbt, unsigned char *smem_raw) {
  int bid;
  GmgView<T> V;
  const int slot = (int)(blockIdx.x % (unsigned)V0.nrhs);
  if (!slot_item(V0, L, &bid, &V)) return;  // a frozen slot keeps its last partials
  partials += ((size_t)slot * nbt + bid) * 3;
  if (V.flags[bid] & kHasChildren) {
    if (threadIdx.x == 0) partials[0] = partials[1] = partials[2] = 0.0;  // one writer, as block_reduce3
    return;
  }
  if (rout) rout += slot * V0.rs_f;
  const int n = NT ? NT : L.n;
  const TileGeo<T, D> G(n);
  // the tile and a cut block's flags only: up to four CTAs of 16^3 FP64
  // blocks per SM, so that one CTA's staging overlaps another's arithmetic
  T *tile = reinterpret_cast<T *>(smem_raw);
  unsigned char *sfl = reinterpret_cast<unsigned char *>(tile + G.size);
  const long long base = L.off + (long long)(bid - L.first) * NCELL;
  const T *bg = V.b + base;  // the block's b, colour-split (read once per cell)
  const long long sb = V.st_base[bid];
  const int4 cl = V.cut_list[bid];
  const int m = cl.y + cl.z;
  CutCell<T, D> q;
  load_tile<T, D, NT>(V, L, Lp, bid, tile, nullptr, sfl, sb, [&] {
    if ((int)threadIdx.x < m) q.fetch(V, cl.x + threadIdx.x);
  });
  const T inv_h2 = T(L.ih2);
  // the norms only steer the stopping test: squares and maxima of the
  // rounded residual are accumulated in FP32 per thread, then in FP64
  float s2f = 0.f, mxf = 0.f, b2f = 0.f;
  auto acc = [&](int c, float r, T bb) {
    if (rout) rout[base + cs_pos(c, n, NCELL, D)] = r;
    s2f = fmaf(r, r, s2f);
    mxf = fmaxf(mxf, fabsf(r));
    const float bf = to_f32(bb);
    b2f = fmaf(bf, bf, b2f);
  };
  {  // listed cells first (stored stencils)
    auto res = [&](const CutCell<T, D> &u) {
      int x, y, z;
      cell_xyz<D>(u.c, n, &x, &y, &z);
      const int t = G.idx(x, y, z);
      const T bb = __ldg(bg + cs_pos_xyz(x, y, z, n, NCELL));
      acc(u.c, to_f32(bb - (u.a[0] * tile[t] + offdiag_of<T, D>(u.a, tile, t, G.sy, G.sz))), bb);
    };
    const int i = threadIdx.x, bd = blockDim.x;
    if (i < m) res(q);
    for (int k = i + bd; k < m; k += bd) {
      CutCell<T, D> u;
      u.fetch(V, cl.x + k);
      res(u);
    }
  }
  for (int c = threadIdx.x; c < NCELL; c += blockDim.x) {
    if (sb >= 0 && sfl[c]) continue;
    int x, y, z;
    cell_xyz<D>(c, n, &x, &y, &z);
    const T bb = __ldg(bg + cs_pos_xyz(x, y, z, n, NCELL));
    acc(c, to_f32(resid_cell<T, D>(nullptr, -1, tile, G.idx(x, y, z), G.sy, G.sz, NCELL, c, inv_h2, bb)), bb);
  }
  block_reduce3((double)s2f, (double)mxf, (double)b2f, partials);
}

template <typename T, int D, int NT>
__global__ void __launch_bounds__(kResThreads, 4) k_resnorm(GmgView<T> V0, LvArgs L, LvArgs Lp, double *partials,
                                                      float *rout, int nbt, ResFold F) {
  pdl_start();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  resnorm_block<T, D, NT>(V0, L, Lp, partials, rout, nbt, smem_raw);
  if (F.on) fold_norms(F, partials, nbt);
}

// Deterministic final reduction of the per-block partials (fixed order),
// one CTA per unit (slot, tree).
__global__ void __launch_bounds__(kResThreads) k_reduce_partials(const double *partials, int nb, const int *tree_blocks,
                                                                 const int *tree_boff, int ntree, double *out,
                                                                 const GridBar *bar);

}  // namespace gmg
