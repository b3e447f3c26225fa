// Host arithmetic of one check of the stopping test (Sec. 5.1.5) from the
// sums the device formed (no CUDA): the residual norm, the duality gap of
// the primal / dual pair of Sec. 2.2 that it gives in closed form, and f(w)
// of the model from the maintained vectors.
//   primal (method 0; x = w, v = rho = y - X^T w, n = K): gap at the dual
//     point alpha = X^T w - y is ||r||^2/(2 lambda);
//     f(w) = lambda/2 ||w||^2 + ||rho||^2/(2n)
//   dual (method 1; x = alpha, v = w = -X alpha/(lambda n), n = N): gap at w
//     is ||r||^2/(2n); D(alpha) = lambda/2 ||w||^2 + ||alpha + y||^2/(2n) and
//     f(w) = ||y||^2/(2n) - D(alpha) + gap
// sums: [0] ||r||^2; with the objective rule [1] ||v||^2, [2] ||w||^2
// (primal) or ||alpha + y||^2 (dual), [3] ||y||^2 (dual).
#pragma once

#include <cmath>

inline void check_values(int method, bool objective, double lam, long long N, long long K,
                         const double* sums, double* res, double* gap, double* fval) {
  const double r2 = sums[0];
  *res = std::sqrt(r2);
  if (method == 0) {
    *gap = r2 / (2.0 * lam);
    if (objective) *fval = 0.5 * lam * sums[2] + sums[1] / (2.0 * (double)K);
  } else {
    *gap = r2 / (2.0 * (double)N);
    if (objective) {
      const double D = 0.5 * lam * sums[1] + sums[2] / (2.0 * (double)N);
      *fval = sums[3] / (2.0 * (double)N) - D + *gap;
    }
  }
}

// Certified relative objective error of a check under the objective rule:
// f(w*) >= f(w) - gap gives (f(w) - f(w*))/f(w*) <= gap / (f(w) - gap) when
// f(w) > gap; -1 when no bound follows.
inline double certified_bound(double fval, double gap) {
  return fval > gap ? gap / (fval - gap) : -1.0;
}

// Whether a check ends the solve: the objective rule stops once
// gap <= tol (f(w) - gap), the residual rule once ||r|| <= tol ||r_0||
// (tol = 0: never).
inline bool check_stops(int objective, double tol, double res0, double res, double gap,
                        double fval) {
  if (!(tol > 0.0)) return false;
  if (objective) return gap <= tol * (fval - gap);
  return res <= tol * res0;
}
