// The coarse part of the V-cycle in one cooperative launch.
//
// The levels with few blocks (the root grid and the first refinement levels)
// hold little data, so one kernel launch per phase would cost far more than
// the work.  This kernel runs, for levels l_hi .. l_lo, the same sequence as
// the per-level kernels (Sec. 2.2: N_down red/black sweeps, residual +
// restriction, FAS right-hand side; exact solve on l_lo; prolongation and
// N_up sweeps on the way up) with a grid-wide barrier between dependent
// phases.  Each CTA works through the blocks b = blockIdx.x, +gridDim.x, ...
// of a phase, so the arithmetic is exactly that of the per-level kernels.
#pragma once

#include "kernels.cuh"

namespace gmg {

struct GridBar {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

constexpr long long kSpinLimit = 1LL << 24;  // ~1.7 s of 100 ns sleeps

// Grid-wide barrier of a cooperative launch (all CTAs co-resident).  Thread
// 0 of each CTA arrives on the counter; the last arrival resets it and
// advances the generation; the others poll the generation with a bounded
// number of sleeps and record GMG_ERR_TIMEOUT when it runs out, so a barrier
// that can never complete ends the kernel instead of hanging it.  Returns
// the same verdict to every thread of the CTA: false once any CTA has
// recorded an error.
__device__ __forceinline__ bool grid_sync(GridBar *bar, unsigned int nctas, long long spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *vgen = &bar->gen;
    volatile int *verr = &bar->err;
    const unsigned int g = *vgen;
    __threadfence();
    if (atomicAdd(&bar->count, 1u) == nctas - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g && *verr == 0) {
        if (++spins > spin_limit) {
          atomicCAS(&bar->err, 0, GMG_ERR_TIMEOUT);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = *verr == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

struct LevelSet {
  LvArgs lv[kMaxLevels];
  int lmin;
};

struct CycleArgs {
  int l_lo, l_hi, n_down, n_up, nc;
  const double *cinv;
  GridBar *bar;
  long long spin_limit;
  int l_one;  // levels l_lo .. l_one hold one block each and run on CTA 0 alone (-1 << 20: none)
};

// Block operations with the compile-time side NT for levels >= 1 and the
// runtime side for the coarse sub-levels inside the root blocks.
template <typename T, int D, int NT>
__device__ __forceinline__ void smooth_any(const GmgView<T> &V, const LvArgs &L, const LvArgs &Lp, int bid, int c,
                                           unsigned char *sm) {
  if (NT && L.n == NT)
    smooth_block<T, D, NT>(V, L, Lp, bid, c, sm);
  else
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

// Exact solve on level Lc by warps w0, w0 + nw, ... : phi = A^-1 b, one warp
// per row, FP64 accumulation.
template <typename T>
__device__ __forceinline__ void coarse_rows(const GmgView<T> &V, const LvArgs &Lc, const double *cinv, int nc, int w0,
                                            int nw) {
  const int lane = threadIdx.x & 31;
  for (int row = w0; row < nc; row += nw) {
    const double *a = cinv + (size_t)row * nc;
    double s = 0.0;
    for (int j = lane; j < nc; j += 32) s += a[j] * (double)V.b[Lc.off + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) V.phi[Lc.poff + row] = T(s);
  }
}

template <typename T, int D, int NT>
__global__ void __launch_bounds__(kThreads) k_cycle_coop(GmgView<T> V, LevelSet LS, CycleArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned int G = gridDim.x;
#define GMG_LV(l) LS.lv[(l)-LS.lmin]
  // levels l_hi .. l_one + 1: every CTA, grid barrier between phases
  for (int l = A.l_hi; l > A.l_lo && l > A.l_one; l--) {
    const LvArgs L = GMG_LV(l), Lp = GMG_LV(l - 1);
    for (int k = 0; k < A.n_down; k++)
      for (int c = 0; c < 2; c++) {
        for (int b = blockIdx.x; b < L.count; b += G) {
          smooth_any<T, D, NT>(V, L, Lp, L.first + b, c, smem_raw);
          __syncthreads();
        }
        if (!grid_sync(A.bar, G, A.spin_limit)) return;
      }
    for (int b = blockIdx.x; b < L.count; b += G) {
      resid_restrict_any<T, D, NT>(V, L, Lp, L.first + b, smem_raw);
      __syncthreads();
    }
    if (!grid_sync(A.bar, G, A.spin_limit)) return;
    const LvArgs Lpp = l - 2 >= LS.lmin ? GMG_LV(l - 2) : Lp;
    for (int b = blockIdx.x; b < Lp.count; b += G) {
      fas_any<T, D, NT>(V, Lp, Lpp, Lp.first + b, smem_raw);
      __syncthreads();
    }
    if (!grid_sync(A.bar, G, A.spin_limit)) return;
  }
  if (A.l_one >= A.l_lo) {
    // single-block levels l_one .. l_lo: CTA 0 runs the bottom of the cycle
    // (sweeps, restriction, FAS, coarse solve, prolongation, sweeps) with
    // block-level barriers only
    if (blockIdx.x == 0) {
      const int top = A.l_one < A.l_hi ? A.l_one : A.l_hi;
      for (int l = top; l > A.l_lo; l--) {
        const LvArgs L = GMG_LV(l), Lp = GMG_LV(l - 1);
        for (int k = 0; k < A.n_down; k++)
          for (int c = 0; c < 2; c++) {
            smooth_any<T, D, NT>(V, L, Lp, L.first, c, smem_raw);
            __syncthreads();
          }
        resid_restrict_any<T, D, NT>(V, L, Lp, L.first, smem_raw);
        __syncthreads();
        const LvArgs Lpp = l - 2 >= LS.lmin ? GMG_LV(l - 2) : Lp;
        fas_any<T, D, NT>(V, Lp, Lpp, Lp.first, smem_raw);
        __syncthreads();
      }
      coarse_rows<T>(V, GMG_LV(A.l_lo), A.cinv, A.nc, threadIdx.x >> 5, kThreads / 32);
      __syncthreads();
      for (int l = A.l_lo + 1; l <= top; l++) {
        const LvArgs L = GMG_LV(l), Lp = GMG_LV(l - 1);
        prolong_any<T, D, NT>(V, L, Lp, L.first, smem_raw);
        __syncthreads();
        for (int k = 0; k < A.n_up; k++)
          for (int c = 0; c < 2; c++) {
            smooth_any<T, D, NT>(V, L, Lp, L.first, c, smem_raw);
            __syncthreads();
          }
      }
    }
  } else {
    coarse_rows<T>(V, GMG_LV(A.l_lo), A.cinv, A.nc, blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5),
                   (int)G * (kThreads / 32));
  }
  if (A.l_hi > A.l_one && !grid_sync(A.bar, G, A.spin_limit)) return;
  for (int l = (A.l_one >= A.l_lo ? A.l_one : A.l_lo) + 1; l <= A.l_hi; l++) {
    const LvArgs L = GMG_LV(l), Lp = GMG_LV(l - 1);
    for (int b = blockIdx.x; b < L.count; b += G) {
      prolong_any<T, D, NT>(V, L, Lp, L.first + b, smem_raw);
      __syncthreads();
    }
    if (!grid_sync(A.bar, G, A.spin_limit)) return;
    for (int k = 0; k < A.n_up; k++)
      for (int c = 0; c < 2; c++) {
        for (int b = blockIdx.x; b < L.count; b += G) {
          smooth_any<T, D, NT>(V, L, Lp, L.first + b, c, smem_raw);
          __syncthreads();
        }
        // the last sweep of the range needs no barrier: the kernel ends
        if (!(l == A.l_hi && k == A.n_up - 1 && c == 1) && !grid_sync(A.bar, G, A.spin_limit)) return;
      }
  }
#undef GMG_LV
}

// A cooperative kernel whose barrier waits for one CTA more than it has:
// the wait must run out and record GMG_ERR_TIMEOUT (failure-detection test).
__global__ void k_barrier_selftest(GridBar *bar, long long spin_limit) {
  grid_sync(bar, gridDim.x + 1, spin_limit);
}

}  // namespace gmg
