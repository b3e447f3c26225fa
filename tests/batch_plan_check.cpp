// Checks of the shared-launch work plan (paper_1612_04003_gb300/csrc/
// ca_batch_plan.h) on random uneven batches: every atom of every instance in
// exactly one unit, each instance's slots 0 .. nslots-1 used once, CTAs
// taking contiguous stretches of the concatenated atoms in order, and every
// CTA's cost within one atom's cost of the mean.  Prints "ALL OK".
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "ca_batch_plan.h"

static int fails = 0;
#define CHECK(c)                                                    \
  do {                                                              \
    if (!(c)) {                                                     \
      std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c);       \
      ++fails;                                                      \
    }                                                               \
  } while (0)

static uint64_t rng_state = 0x9E3779B97F4A7C15ULL;
static uint64_t next_u64() {  // splitmix64
  uint64_t z = (rng_state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static long long uniform(long long lo, long long hi) {  // [lo, hi]
  return lo + (long long)(next_u64() % (uint64_t)(hi - lo + 1));
}

static void check_plan(const std::vector<cabatch::Instance>& in, int P) {
  cabatch::Plan pl;
  CHECK(cabatch::plan(in, P, &pl));
  CHECK((int)pl.cta.size() == P && pl.nslots.size() == in.size());
  double total = 0.0, cmax = 0.0;
  for (const auto& x : in) {
    total += (double)cabatch::atoms_of(x.K) * cabatch::atom_cost(x.sb);
    cmax = std::max(cmax, cabatch::atom_cost(x.sb));
  }
  // walk the CTAs in order: their units must continue the concatenation
  int inst = 0;
  long long at = 0;
  std::vector<std::vector<int>> slot_seen(in.size());
  for (size_t i = 0; i < in.size(); ++i) slot_seen[i].assign((size_t)pl.nslots[i], 0);
  for (int p = 0; p < P; ++p) {
    double load = 0.0;
    for (const auto& u : pl.cta[(size_t)p]) {
      while (inst < (int)in.size() && at == cabatch::atoms_of(in[(size_t)inst].K)) {
        ++inst;
        at = 0;
      }
      CHECK(u.inst == inst && u.a0 == at && u.a1 > u.a0);
      CHECK(u.a1 <= cabatch::atoms_of(in[(size_t)u.inst].K));
      CHECK(u.slot >= 0 && u.slot < pl.nslots[(size_t)u.inst]);
      if (u.slot >= 0 && u.slot < pl.nslots[(size_t)u.inst]) ++slot_seen[(size_t)u.inst][(size_t)u.slot];
      at = u.a1;
      load += (double)(u.a1 - u.a0) * cabatch::atom_cost(in[(size_t)u.inst].sb);
    }
    CHECK(std::fabs(load - pl.load[(size_t)p]) <= 1e-9 * total);
    CHECK(std::fabs(load - total / P) <= cmax * (1 + 1e-9));
  }
  CHECK(inst == (int)in.size() - 1 && at == cabatch::atoms_of(in.back().K));
  for (const auto& v : slot_seen)
    for (int c : v) CHECK(c == 1);
}

int main() {
  // one instance: the even split-K of a single solve (atom counts differ by
  // at most one between CTAs)
  {
    std::vector<cabatch::Instance> one{{262144, 128}};
    cabatch::Plan pl;
    CHECK(cabatch::plan(one, 151, &pl));
    long long mn = 1LL << 60, mx = 0;
    for (const auto& c : pl.cta) {
      CHECK(c.size() == 1);
      if (c.size() == 1) {
        mn = std::min(mn, c[0].a1 - c[0].a0);
        mx = std::max(mx, c[0].a1 - c[0].a0);
      }
    }
    CHECK(mx - mn <= 1 && pl.nslots[0] == 151);
    check_plan(one, 151);
  }
  // fewer atoms than CTAs: some CTAs stay empty, none gets two atoms
  {
    std::vector<cabatch::Instance> small{{64, 32}, {32, 8}};
    cabatch::Plan pl;
    CHECK(cabatch::plan(small, 151, &pl));
    int used = 0;
    for (const auto& c : pl.cta) {
      CHECK(c.size() <= 1);
      used += (int)c.size();
    }
    CHECK(used == 3);
    check_plan(small, 151);
  }
  // invalid input
  {
    cabatch::Plan pl;
    CHECK(!cabatch::plan({}, 4, &pl));
    CHECK(!cabatch::plan({{100, 8}}, 0, &pl));
    CHECK(!cabatch::plan({{0, 8}}, 4, &pl));
    CHECK(!cabatch::plan({{100, 0}}, 4, &pl));
  }
  // random uneven batches (the served mix: K log-uniform, sb in 4 .. 256)
  for (int trial = 0; trial < 400; ++trial) {
    const int m = (int)uniform(1, 64);
    std::vector<cabatch::Instance> in;
    for (int i = 0; i < m; ++i) {
      const double lk = std::log(1.0) + (std::log(300000.0) - std::log(1.0)) *
                                            (double)(next_u64() >> 11) / 9007199254740992.0;
      in.push_back({std::max(1LL, (long long)std::exp(lk)), (int)uniform(4, 256)});
    }
    const int Ps[] = {1, 2, 7, 151, 152, 600};
    check_plan(in, Ps[trial % 6]);
  }
  if (fails == 0) std::printf("ALL OK\n");
  return fails ? 1 : 0;
}
