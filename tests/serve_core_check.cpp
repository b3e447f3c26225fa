// CPU check of the serving scheduler (ca_serve_core.h) with a fake executor:
// the executor mirrors the arena model (a worker's arena grows to a request's
// need when it starts, a release sets it to zero) and checks, at every start,
// that the arenas of all workers fit the budget; starts must follow the
// submission order; oversized requests are rejected; every request ends.
#include <atomic>
#include <cstdio>
#include <mutex>
#include <random>
#include <vector>

#include "ca_serve_core.h"

static int fails = 0;
#define CHECK(c)                                             \
  do {                                                       \
    if (!(c)) {                                              \
      std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c); \
      ++fails;                                               \
    }                                                        \
  } while (0)

struct Fake {
  std::mutex m;
  std::vector<size_t> arena;
  std::vector<size_t> need;
  std::vector<long long> starts;
  size_t budget;
  int running = 0, peak = 0;
  bool over = false;
  std::atomic<int> releases{0};
  Fake(int workers, size_t b) : arena(workers, 0), budget(b) {}
  size_t group_need(const std::vector<long long>& ids) const {
    size_t t = 0;
    for (long long id : ids) t += need[(size_t)id];
    return t;
  }
  int run(int w, const std::vector<long long>& ids) {
    {
      std::lock_guard<std::mutex> lk(m);
      arena[w] = std::max(arena[w], group_need(ids));
      size_t tot = 0;
      for (size_t a : arena) tot += a;
      if (tot > budget) over = true;
      for (long long id : ids) starts.push_back(id);
      groups.push_back(ids);
      running += (int)ids.size();
      peak = std::max(peak, running);
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200 + (ids[0] * 7919) % 1800));
    std::lock_guard<std::mutex> lk(m);
    running -= (int)ids.size();
    return 0;
  }
  std::vector<std::vector<long long>> groups;
  void release(int w) {
    std::lock_guard<std::mutex> lk(m);
    arena[w] = 0;
    ++releases;
  }
};

static void scenario(int workers, size_t budget, int njobs, size_t lo, size_t hi, unsigned seed,
                     int max_group = 1) {
  Fake f(workers, budget);
  std::mt19937 rng(seed);
  std::uniform_int_distribution<size_t> dist(lo, hi);
  for (int i = 0; i < njobs; ++i) f.need.push_back(dist(rng));
  std::vector<long long> ids, order;
  {
    caserve::Scheduler s(
        workers, budget, [&](int w, const std::vector<long long>& g) { return f.run(w, g); },
        [&](int w) { f.release(w); });
    if (max_group > 1) s.set_grouping(max_group);
    // groups of requests with the same parity of their need
    for (int i = 0; i < njobs; ++i)
      ids.push_back(max_group > 1 ? s.submit(f.need[(size_t)i], (long long)(f.need[(size_t)i] % 2),
                                             f.need[(size_t)i])
                                  : s.submit(f.need[(size_t)i]));
    for (int i = 0; i < njobs; ++i) {
      caserve::JobState j = s.wait(ids[(size_t)i]);
      CHECK(j.done);
      if (f.need[(size_t)i] > budget) {
        CHECK(j.status == caserve::Scheduler::kRejected && j.admitted < 0);
      } else {
        CHECK(j.status == 0 && j.worker >= 0 && j.worker < workers);
        order.push_back(j.admitted);
      }
    }
    s.drain();
    caserve::Stats st = s.stats();
    long long nrej = 0;
    for (size_t v : f.need) nrej += v > budget;
    CHECK(st.submitted == njobs && st.rejected == nrej && st.completed == njobs - nrej);
    CHECK(st.p50_ms > 0 && st.p50_ms <= st.p99_ms && st.p99_ms <= st.max_ms);
    CHECK(st.peak_footprint <= budget);
    CHECK(st.peak_concurrency <= workers * max_group && st.peak_concurrency == f.peak);
  }
  CHECK(!f.over);
  // admission follows the submission order (rejected requests never start)
  for (size_t k = 0; k < order.size(); ++k) CHECK(order[k] == (long long)k);
  CHECK(f.starts.size() == order.size());
  // groups: consecutive submissions, all accepted by the grouping rule, at
  // most max_group, never more than the budget
  size_t grouped = 0;
  for (const auto& g : f.groups) {
    CHECK((int)g.size() <= max_group && !g.empty());
    for (size_t k = 1; k < g.size(); ++k) {
      CHECK(g[k] > g[k - 1]);
      CHECK(f.need[(size_t)g[k]] % 2 == f.need[(size_t)g[0]] % 2);
    }
    CHECK(f.group_need(g) <= budget);
    grouped += g.size() > 1;
  }
  if (max_group > 1) CHECK(grouped > 0);
  std::printf("scenario workers=%d budget=%zu jobs=%d: peak concurrency %d, releases %d\n", workers,
              budget, njobs, f.peak, f.releases.load());
}

// The s tuner: each class explores its candidates once, then keeps to the
// cheapest measured one; classes do not share measurements.
static void tuner_checks() {
  caserve::STuner t(256);
  CHECK((t.candidates(8) == std::vector<int>{8, 16, 4, 32, 2, 1}));
  CHECK((t.candidates(64) == std::vector<int>{4, 2, 1}));
  CHECK(t.largest(8) == 32 && t.largest(300) == 1);
  caserve::STuner::Key a{0, 1, 3, 8, 12, 18}, b{1, 1, 3, 8, 14, 11};
  // seconds per update: a prefers s = 16, b prefers s = 4
  auto cost_a = [](int s) { return 1.0 / s + 0.004 * s; };
  auto cost_b = [](int s) { return 0.2 / s + 0.02 * s; };
  std::vector<int> seen_a, seen_b;
  for (int it = 0; it < 12; ++it) {
    const int sa = t.choose(a), sb = t.choose(b);
    seen_a.push_back(sa);
    seen_b.push_back(sb);
    t.record(a, sa, cost_a(sa) * 1000, 1000);
    t.record(b, sb, cost_b(sb) * 500, 500);
  }
  CHECK((std::vector<int>(seen_a.begin(), seen_a.begin() + 6) == t.candidates(8)));
  for (int it = 6; it < 12; ++it) CHECK(seen_a[(size_t)it] == 16 && seen_b[(size_t)it] == 4);
  CHECK(t.cost(a, 16) > 0 && t.cost(a, 64) < 0);
  // concurrent use
  std::vector<std::thread> th;
  for (int k = 0; k < 8; ++k)
    th.emplace_back([&t, k] {
      caserve::STuner::Key c{0, 1, 2, 4, k, 10};
      for (int it = 0; it < 200; ++it) {
        const int s = t.choose(c);
        t.record(c, s, 1e-3 * (1.0 / s + 0.01 * s), 1);
      }
    });
  for (auto& x : th) x.join();
  caserve::STuner::Key c0{0, 1, 2, 4, 0, 10};
  CHECK(t.choose(c0) == 8);  // argmin of 1/s + 0.01 s over 1, 2, 4, ..., 64
  std::printf("tuner: class a -> %d, class b -> %d\n", seen_a.back(), seen_b.back());
}

int main() {
  tuner_checks();
  scenario(4, 100, 60, 5, 40, 1);    // several requests fit at once
  scenario(4, 100, 40, 30, 120, 2);  // large requests: releases, rejections
  scenario(1, 50, 20, 1, 50, 3);     // one worker: strictly one at a time
  scenario(8, 1000, 200, 1, 100, 4); // wide
  scenario(2, 400, 120, 1, 60, 5, 8);  // grouping: up to 8 requests per start
  scenario(3, 100, 80, 5, 40, 6, 4);   // grouping under a tight budget
  {  // a request that needs the whole budget after others grew their arenas
    Fake f(3, 90);
    f.need = {30, 30, 30, 90, 10};
    caserve::Scheduler s(
        3, 90, [&](int w, const std::vector<long long>& g) { return f.run(w, g); },
        [&](int w) { f.release(w); });
    std::vector<long long> ids;
    for (size_t v : f.need) ids.push_back(s.submit(v));
    for (size_t k = 0; k < ids.size(); ++k) CHECK(s.wait(ids[k]).admitted == (long long)k);
    s.drain();
    CHECK(!f.over);
    CHECK(f.releases.load() >= 2);
  }
  if (fails == 0) std::printf("ALL OK\n");
  return fails == 0 ? 0 : 1;
}
