// Level-set functions and the line search of Sec. 3.2, usable on host and
// device.  Compiled without multiply-add contraction (host:
// -ffp-contract=off, device: --fmad=false) so that every evaluation is the
// plain IEEE sequence written here.
#pragma once

#include <math.h>

#include "gmg.h"

namespace gmg {

struct LsfSpec {
  int kind;
  double p[16];
};

// Built-in level-set functions (Sec. 3.1, Eq. (lsf-example)); negative inside.
__host__ __device__ inline double lsf_builtin(const LsfSpec &L, int D, const double *x) {
  const double *p = L.p;
  switch (L.kind) {
    case GMG_LSF_SPHERE: {
      double s = 0.0;
      for (int d = 0; d < D; d++) {
        double t = x[d] - p[d];
        s = s + t * t;
      }
      return sqrt(s) - p[3];
    }
    case GMG_LSF_CAPSULE: {
      double ab[3], ax[3], num = 0.0, den = 0.0;
      for (int d = 0; d < D; d++) {
        ab[d] = p[3 + d] - p[d];
        ax[d] = x[d] - p[d];
        num = num + ax[d] * ab[d];
        den = den + ab[d] * ab[d];
      }
      double t = num / den;
      t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
      double s = 0.0;
      for (int d = 0; d < D; d++) {
        double q = x[d] - (p[d] + t * ab[d]);
        s = s + q * q;
      }
      return sqrt(s) - p[6];
    }
    case GMG_LSF_ELLIPSOID: {
      double s = 0.0, amin = p[12];
      for (int i = 0; i < D; i++) {
        double y = 0.0;
        for (int j = 0; j < D; j++) y = y + p[3 + 3 * j + i] * (x[j] - p[j]);
        double q = y / p[12 + i];
        s = s + q * q;
        amin = p[12 + i] < amin ? p[12 + i] : amin;
      }
      return amin * (sqrt(s) - 1.0);
    }
    case GMG_LSF_SHAPE: {  // Sec. 4.3, Eqs. (spheroid) .. (astroid); reading SH for the coordinates
      double u, v;
      if (p[1] != 0.0) {
        u = 4.0 * (sqrt(x[0] * x[0] + x[1] * x[1]) - 0.5);
        v = 4.0 * (x[2] - 0.5);
      } else {
        u = 4.0 * (x[0] - 0.5);
        v = 4.0 * (x[1] - 0.5);
      }
      switch ((int)p[0]) {
        case 0: return sqrt(8.0 * u * u + v * v) - 1.0;
        case 1: return 8.0 * fabs(u) + fabs(v) - 1.5;
        case 2: {
          const double w = v - cbrt(u * u);
          return u * u + w * w - 1.0;
        }
        default: return cbrt(u * u) / 0.8 + cbrt(v * v) / 1.5 - 0.8;
      }
    }
    default:
      return 1.0;
  }
}

__host__ __device__ inline void seg_point(int D, const double *a, const double *b, double t, double *x) {
  for (int d = 0; d < 3; d++) x[d] = d < D ? a[d] + t * (b[d] - a[d]) : 0.0;
}

// Bisection on t in [0, t_hi] along a -> b, f(a) f(x(t_hi)) <= 0; halves
// while the bracket is at least eps wide and returns its midpoint.
template <typename F>
__host__ __device__ inline double bisect_root(const F &f, int D, const double *a, const double *b, double fa,
                                              double t_hi, double eps) {
  double lo = 0.0, hi = t_hi, x[3];
  while (hi - lo >= eps) {
    double mid = 0.5 * (lo + hi);
    seg_point(D, a, b, mid, x);
    if (fa * f(x) <= 0.0)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Relative distance d in [eps, 1] from a toward b (Eq. (relative-distance)):
// bisection when f(a) f(b) <= 0, otherwise a golden-section search for the
// minimum of f(a) f(x) that stops at the first sign change and then bisects;
// 1 when no sign change is found (no boundary).
template <typename F>
__host__ __device__ inline double line_search(const F &f, int D, const double *a, const double *b, double eps) {
  double x[3];
  double fa = f(a), fb = f(b);
  double t = 1.0;
  bool found = false;
  if (fa * fb <= 0.0) {
    t = bisect_root(f, D, a, b, fa, 1.0, eps);
    found = true;
  } else {
    const double gr = (sqrt(5.0) - 1.0) / 2.0;
    double lo = 0.0, hi = 1.0;
    double t1 = hi - gr * (hi - lo), t2 = lo + gr * (hi - lo);
    seg_point(D, a, b, t1, x);
    double h1 = fa * f(x);
    double h2 = 0.0;
    if (h1 <= 0.0) {
      t = bisect_root(f, D, a, b, fa, t1, eps);
      found = true;
    } else {
      seg_point(D, a, b, t2, x);
      h2 = fa * f(x);
      if (h2 <= 0.0) {
        t = bisect_root(f, D, a, b, fa, t2, eps);
        found = true;
      }
    }
    while (!found && hi - lo >= eps) {
      if (h1 < h2) {
        hi = t2;
        t2 = t1;
        h2 = h1;
        t1 = hi - gr * (hi - lo);
        seg_point(D, a, b, t1, x);
        h1 = fa * f(x);
        if (h1 <= 0.0) {
          t = bisect_root(f, D, a, b, fa, t1, eps);
          found = true;
        }
      } else {
        lo = t1;
        t1 = t2;
        h1 = h2;
        t2 = lo + gr * (hi - lo);
        seg_point(D, a, b, t2, x);
        h2 = fa * f(x);
        if (h2 <= 0.0) {
          t = bisect_root(f, D, a, b, fa, t2, eps);
          found = true;
        }
      }
    }
  }
  if (!found) return 1.0;
  if (t < eps) t = eps;
  if (t > 1.0) t = 1.0;
  return t;
}

}  // namespace gmg
