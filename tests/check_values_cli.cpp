// Reads lines "method objective lambda N K s0 s1 s2 s3" and prints
// "res gap fval bound stop" from check_values, certified_bound and
// check_stops (paper_1612_04003_gb300/csrc/ca_check.h), the host arithmetic
// of a stopping-test check; stop is the objective rule's decision at
// tol = 1e-6 (with res0 = res).
#include <cstdio>

#include "ca_check.h"

int main() {
  int method = 0, objective = 0;
  double lam = 0, s[4] = {0, 0, 0, 0};
  long long N = 0, K = 0;
  while (std::scanf("%d %d %lf %lld %lld %lf %lf %lf %lf", &method, &objective, &lam, &N, &K,
                    &s[0], &s[1], &s[2], &s[3]) == 9) {
    double res = 0, gap = 0, fval = 0;
    check_values(method, objective != 0, lam, N, K, s, &res, &gap, &fval);
    const double bound = certified_bound(fval, gap);
    const int stop = check_stops(1, 1e-6, res, res, gap, fval) ? 1 : 0;
    std::printf("%.17g %.17g %.17g %.17g %d\n", res, gap, fval, bound, stop);
  }
  return 0;
}
