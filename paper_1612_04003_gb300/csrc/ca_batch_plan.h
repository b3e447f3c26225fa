// Work plan of a shared Gram launch over several solve instances (host only,
// no CUDA).  One outer step of instance i reads its sb_i sampled rows over
// K_i columns, in 32-column atoms (steps a2 + a3).  In a shared launch the P
// CTAs split the concatenation of every instance's atoms, each CTA taking one
// contiguous stretch of equal cost; the cost of an atom of instance i is the
// bytes it moves, sb_i * 128 (FP32 rows) + 256 (the FP32 pair of v), the
// pass being bound by HBM.  A stretch may cross instance boundaries: the CTA
// then runs one unit per instance it touches, each unit writing its own
// split-K partial slot, and the reduction of instance i sums its nslots[i]
// slots.  An atom goes to the CTA whose share of the total cost holds the
// atom's midpoint, so every CTA's cost is within one atom's cost of C / P.
//
// Instances of one launch share the Gram tile class (s*b padded to 32, 64,
// 128 or 256); the caller groups them by it.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace cabatch {

struct Instance {
  long long K;  // columns of A (> 0)
  int sb;       // sampled rows of the outer step (> 0)
};

struct Unit {
  int inst;          // instance
  long long a0, a1;  // its atoms [a0, a1)
  int slot;          // its partial slot, 0-based within the instance
};

struct Plan {
  std::vector<std::vector<Unit>> cta;  // units of each CTA, in order
  std::vector<int> nslots;             // partial slots of each instance
  std::vector<double> load;            // cost of each CTA
};

inline long long atoms_of(long long K) { return (K + 31) / 32; }
inline double atom_cost(int sb) { return (double)sb * 128.0 + 256.0; }

// Fills *out; false on invalid input (no instances, P < 1, K < 1 or sb < 1).
inline bool plan(const std::vector<Instance>& in, int P, Plan* out) {
  if (in.empty() || P < 1 || !out) return false;
  double total = 0.0;
  for (const Instance& x : in) {
    if (x.K < 1 || x.sb < 1) return false;
    total += (double)atoms_of(x.K) * atom_cost(x.sb);
  }
  out->cta.assign((size_t)P, {});
  out->nslots.assign(in.size(), 0);
  out->load.assign((size_t)P, 0.0);
  const double share = total / (double)P;
  double start = 0.0;  // cost before the instance's first atom
  for (int i = 0; i < (int)in.size(); ++i) {
    const long long na = atoms_of(in[(size_t)i].K);
    const double c = atom_cost(in[(size_t)i].sb);
    // the CTA whose share holds the midpoint of atom t (monotone in t)
    auto cta_of = [&](long long t) {
      return std::min(P - 1, (int)((start + ((double)t + 0.5) * c) / share));
    };
    long long a = 0;
    while (a < na) {
      const int p = cta_of(a);
      long long e = na;
      if (p < P - 1) {
        // atoms t < lim have their midpoint below the next share
        const double lim = ((double)(p + 1) * share - start) / c - 0.5;
        e = std::min(na, std::max(a + 1, (long long)std::ceil(std::min(lim, (double)na))));
        while (e > a + 1 && cta_of(e - 1) != p) --e;  // rounding guards
        while (e < na && cta_of(e) == p) ++e;
      }
      out->cta[(size_t)p].push_back(Unit{i, a, e, out->nslots[(size_t)i]++});
      out->load[(size_t)p] += (double)(e - a) * c;
      a = e;
    }
    start += (double)na * c;
  }
  return true;
}

}  // namespace cabatch
