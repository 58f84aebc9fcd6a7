// Field evaluation E = -grad(phi) on cell faces (Sec. 4.4, two-electrode
// example): the components of grad(phi) on a staggered grid, taking the
// stored boundary distances into account.  For every leaf cell i and axis k
// the gradient on its upper face i + 1/2:
//   (phi_b - phi_i) / (d dx)        if the level set's boundary lies between
//                                   i and i + e_k at relative distance d < 1,
//   2 (phi_w - phi_i) / dx          at a Dirichlet domain wall (value phi_w
//                                   at the face centre), 0 at a Neumann wall,
//   (phi_{i+e_k} - phi_i) / dx      otherwise, with phi_{i+e_k} the same
//                                   ghost the operator uses (same-level
//                                   neighbour or refinement-boundary ghost),
// and E = 0 in cells whose centre lies inside the object.
#pragma once

#include "kernels.cuh"

namespace gmg {

struct EfieldArgs {
  const unsigned char *cellflag;  // per block and cell: bit 1 = centre inside the object
  const long long *mask_base;     // [nb] offset of the block's flags
  const double *dist, *bphib;     // cut blocks: ncell x 2D distances and boundary values
  const long long *dist_base;     // [nb] offset, -1 for blocks without a cut
  const double *wallv;            // blocks on an upper wall: D x n^(D-1) face values
  const long long *wallv_base;    // [nb] offset, -1 for none
  const int *leafpos;             // [nb] first leaf cell of the block / ncell, -1 for covered blocks
  double *out;                    // [nrhs][n_leaf][D]
  long long nleaf;
  int dirichlet_upper;            // bit k: the upper wall of axis k is Dirichlet
};

template <int D, int NT>
__global__ void __launch_bounds__(kThreads) k_efield(GmgView<double> V0, LvArgs L, LvArgs Lp, EfieldArgs E) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int bid;
  GmgView<double> V;
  const int slot = (int)(blockIdx.x % (unsigned)V0.nrhs);
  if (!slot_item(V0, L, &bid, &V)) return;
  const int lp = E.leafpos[bid];
  if (lp < 0) return;  // covered block: no leaf cells
  const int n = NT ? NT : L.n;
  const int ncell = D == 3 ? n * n * n : n * n, nf = D == 3 ? n * n : n;
  const TileGeo<double, D> G(n);
  double *tile = reinterpret_cast<double *>(smem_raw);
  load_tile<double, D, NT>(V, L, Lp, bid, tile);
  const double h = L.h;
  const long long db = E.dist_base[bid], wb = E.wallv_base[bid];
  const unsigned char *fl = E.cellflag + E.mask_base[bid];
  double *out = E.out + ((long long)slot * E.nleaf + (long long)lp * ncell) * D;
  const int st[3] = {1, G.sy, G.sz};
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    int p[3];
    cell_xyz<D>(c, n, &p[0], &p[1], &p[2]);
    const int t = G.idx(p[0], p[1], p[2]);
    const double ph = tile[t];
    const bool inside = (fl[c] & 2) != 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
      double g;
      const double d = db >= 0 ? E.dist[db + (long long)c * 2 * D + 2 * k + 1] : 1.0;
      if (inside) {
        g = 0.0;
      } else if (d < 1.0) {
        g = (E.bphib[db + (long long)c * 2 * D + 2 * k + 1] - ph) / (d * h);
      } else if (p[k] == n - 1 && wb >= 0 && (V.flags[bid] & wall_bit(k, 1))) {
        const int j = k == 0 ? p[1] + n * p[2] : (k == 1 ? p[0] + n * p[2] : p[0] + n * p[1]);
        g = ((E.dirichlet_upper >> k) & 1) ? 2.0 * (E.wallv[wb + (long long)k * nf + (D == 3 ? j : (k == 0 ? p[1] : p[0]))] - ph) / h
                                           : 0.0;
      } else {
        g = (tile[t + st[k]] - ph) / h;
      }
      out[(long long)c * D + k] = -g;
    }
  }
}

}  // namespace gmg
