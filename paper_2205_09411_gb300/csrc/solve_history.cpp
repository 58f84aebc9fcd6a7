// Solve with the residual history: the loop of gmg_solve (Sec. 2.2: a
// residual, then cycles each followed by the residual, until every unit's
// relative residual reaches the tolerance), run step by step through
// gmg_iterate, keeping every unit's relative residual after every step (the
// convergence curves of Sec. 4).  Same stopping and failure rules as
// gmg_solve, and the same device work per step.
#include <cmath>
#include <vector>

#include "gmg_internal.h"

extern "C" int gmg_solve_history(gmg_tree *t, int precision, double rel_tol, int max_cycles, double *history,
                                 gmg_stats *stats, void *stream) {
  using namespace gmg;
  if (!t || !history || max_cycles < 0 || !(rel_tol > 0.0)) return set_error("bad arguments"), GMG_ERR_INVALID_ARG;
  if (!t->bound) return set_error("tree not bound"), GMG_ERR_STATE;
  const int R = t->units();
  std::vector<int> act(R, 1), cyc(R, 0);
  std::vector<double> rel(R, 0.0), linf(R, 0.0), prev(R, INFINITY);
  for (size_t i = 0; i < (size_t)(max_cycles + 1) * R; i++) history[i] = NAN;
  int rc = gmg_iterate(t, precision, act.data(), 1, rel.data(), linf.data(), stream);
  if (rc) return rc;
  int cycles = 0;
  for (;;) {
    for (int r = 0; r < R; r++) history[(size_t)cycles * R + r] = rel[r];
    int left = 0;
    for (int r = 0; r < R; r++) {
      if (!act[r]) continue;
      if (!std::isfinite(rel[r]) || (cyc[r] > 2 && rel[r] > 1e3 * prev[r])) {
        rc = GMG_ERR_NONFINITE;
        set_error("residual norm is not finite or diverges");
      }
      prev[r] = std::min(prev[r], rel[r]);
      if (rel[r] <= rel_tol) act[r] = 0;
      left += act[r];
    }
    if (rc || left == 0) break;
    if (cycles >= max_cycles) {
      rc = GMG_ERR_NOT_CONVERGED;
      set_error("tolerance not reached within max_cycles");
      break;
    }
    rc = gmg_iterate(t, precision, act.data(), 0, rel.data(), linf.data(), stream);
    if (rc) return rc;
    cycles++;
    for (int r = 0; r < R; r++) cyc[r] += act[r];
  }
  if (stats)
    for (int r = 0; r < R; r++) {
      stats[r].cycles = cyc[r];
      stats[r].rel_l2 = rel[r];
      stats[r].linf = linf[r];
      stats[r].bnorm = std::sqrt(t->h_red[4 * (size_t)r + 2]);  // the unit's last reduction (synchronised)
    }
  return rc;
}
