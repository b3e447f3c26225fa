// Request scheduler of the serving loop (host only, no CUDA): a FIFO queue of
// solve requests, a fixed set of workers (in the server each owns a CUDA
// stream and a library context, so admitted requests run concurrently on the
// device), and admission by device-memory footprint.
//
// Footprint model: worker w keeps a scratch arena of arena_w bytes that a
// request needing `need` bytes grows to max(arena_w, need) (the library frees
// the old arena before allocating the larger one).  The queue's head may
// start on an idle worker w when
//     sum_{v != w} arena_v + max(arena_w, need) <= budget,
// on the idle worker for which that sum is smallest.  When it fits on no idle
// worker, the largest arena of an idle worker is released and admission is
// tried again; when no idle worker holds an arena, the head waits for a
// request to finish.  A request needing more than the whole budget is
// rejected at submission.  Strict FIFO: no request overtakes an earlier one.
//
// Grouping (optional, set_grouping): a request may be submitted with a group
// key >= 0 and its need inside a group; the head may then take along the
// longest run of requests queued right behind it with the head's key, up to
// max_group, as long as the group's need (the sum of its members' group
// needs) fits as above; the group starts on one worker and its requests end
// together.  Requests still start in submission order.
//
// run(worker, ids) executes the requests ids (one, or a group) on that worker
// and returns a status for all of them; release(worker) frees an idle
// worker's arena.  Both are called without the scheduler's lock held.
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <thread>
#include <vector>

namespace caserve {

using Clock = std::chrono::steady_clock;

struct JobState {
  size_t need = 0;
  long long gkey = -1;  // group key (-1: never grouped)
  size_t gneed = 0;     // need inside a group
  int status = 0;
  int worker = -1;
  long long admitted = -1;  // position in the admission order
  bool done = false;
  Clock::time_point t_submit, t_start, t_end;
};

struct Stats {
  long long submitted = 0, completed = 0, rejected = 0;
  double p50_ms = 0, p99_ms = 0, mean_ms = 0, max_ms = 0;  // submission -> end
  double wall_s = 0;            // first submission -> last end
  size_t peak_footprint = 0;    // largest sum of arenas admitted
  int peak_concurrency = 0;     // most requests running at once
};

class Scheduler {
 public:
  using RunFn = std::function<int(int worker, const std::vector<long long>& ids)>;
  using ReleaseFn = std::function<void(int worker)>;

  static constexpr int kRejected = -6;  // status of a request larger than the budget

  Scheduler(int workers, size_t budget, RunFn run, ReleaseFn release)
      : budget_(budget), run_(std::move(run)), release_(std::move(release)), ws_(workers) {
    for (int w = 0; w < workers; ++w) ws_[w].th = std::thread([this, w] { worker_loop(w); });
    disp_ = std::thread([this] { dispatch_loop(); });
  }

  ~Scheduler() {
    drain();
    {
      std::lock_guard<std::mutex> lk(m_);
      stop_ = true;
    }
    cv_disp_.notify_all();
    for (auto& w : ws_) w.cv.notify_all();
    disp_.join();
    for (auto& w : ws_) w.th.join();
  }

  Scheduler(const Scheduler&) = delete;
  Scheduler& operator=(const Scheduler&) = delete;

  // Groups of up to max_group requests (1: no grouping).
  void set_grouping(int max_group) {
    std::lock_guard<std::mutex> lk(m_);
    max_group_ = std::max(1, max_group);
  }

  // Queue a request needing `need` bytes of scratch alone (and gneed inside a
  // group of requests with the same gkey >= 0); returns its id.
  long long submit(size_t need, long long gkey = -1, size_t gneed = 0) {
    std::lock_guard<std::mutex> lk(m_);
    const long long id = (long long)jobs_.size();
    jobs_.emplace_back();
    JobState& j = jobs_.back();
    j.need = need;
    j.gkey = gkey;
    j.gneed = gneed;
    j.t_submit = Clock::now();
    if (first_ == Clock::time_point()) first_ = j.t_submit;
    if (need > budget_) {
      j.status = kRejected;
      j.done = true;
      j.t_start = j.t_end = j.t_submit;
      ++rejected_;
      cv_done_.notify_all();
    } else {
      queue_.push_back(id);
      ++gen_;
      cv_disp_.notify_one();
    }
    return id;
  }

  // Block until request id has ended; returns its state.
  JobState wait(long long id) {
    std::unique_lock<std::mutex> lk(m_);
    cv_done_.wait(lk, [&] { return jobs_[(size_t)id].done; });
    return jobs_[(size_t)id];
  }

  // Block until every submitted request has ended.
  void drain() {
    std::unique_lock<std::mutex> lk(m_);
    cv_done_.wait(lk, [&] { return queue_.empty() && running_ == 0; });
  }

  Stats stats() {
    std::lock_guard<std::mutex> lk(m_);
    Stats s;
    s.submitted = (long long)jobs_.size();
    s.rejected = rejected_;
    s.peak_footprint = peak_footprint_;
    s.peak_concurrency = peak_running_;
    std::vector<double> lat;
    Clock::time_point last = first_;
    for (const JobState& j : jobs_)
      if (j.done && j.status != kRejected) {
        lat.push_back(std::chrono::duration<double, std::milli>(j.t_end - j.t_submit).count());
        last = std::max(last, j.t_end);
      }
    s.completed = (long long)lat.size();
    if (!lat.empty()) {
      std::sort(lat.begin(), lat.end());
      auto rank = [&](double q) {  // nearest-rank percentile
        size_t k = (size_t)std::ceil(q * (double)lat.size());
        return lat[std::min(lat.size(), std::max<size_t>(k, 1)) - 1];
      };
      s.p50_ms = rank(0.50);
      s.p99_ms = rank(0.99);
      s.max_ms = lat.back();
      double sum = 0;
      for (double v : lat) sum += v;
      s.mean_ms = sum / (double)lat.size();
      s.wall_s = std::chrono::duration<double>(last - first_).count();
    }
    return s;
  }

  size_t arena_of(int w) {
    std::lock_guard<std::mutex> lk(m_);
    return ws_[w].arena;
  }

 private:
  struct Worker {
    size_t arena = 0;
    std::vector<long long> jobs;  // assigned requests (empty: none)
    bool busy = false;   // running, or being released
    std::thread th;
    std::condition_variable cv;
  };

  void dispatch_loop() {
    std::unique_lock<std::mutex> lk(m_);
    for (;;) {
      const unsigned long long seen = gen_;
      if (stop_ && queue_.empty()) return;
      if (!queue_.empty()) {
        size_t total = 0;
        for (const Worker& w : ws_) total += w.arena;
        // the idle worker on which `need` leaves the smallest sum of arenas
        auto fit = [&](size_t need, int* best, size_t* best_total) {
          *best = -1;
          for (int w = 0; w < (int)ws_.size(); ++w) {
            if (ws_[w].busy) continue;
            const size_t t = total - ws_[w].arena + std::max(ws_[w].arena, need);
            if (t <= budget_ && (*best < 0 || t < *best_total)) {
              *best = w;
              *best_total = t;
            }
          }
          return *best >= 0;
        };
        const long long head = queue_.front();
        std::vector<long long> grp{head};
        size_t gneed = jobs_[(size_t)head].need;
        int best = -1;
        size_t best_total = 0;
        if (fit(gneed, &best, &best_total)) {
          // grouping: requests right behind the head with its key
          const long long key = jobs_[(size_t)head].gkey;
          size_t gsum = jobs_[(size_t)head].gneed;
          for (size_t k = 1; k < queue_.size() && (int)grp.size() < max_group_ && key >= 0 &&
                             jobs_[(size_t)queue_[k]].gkey == key;
               ++k) {
            grp.push_back(queue_[k]);
            gsum += jobs_[(size_t)queue_[k]].gneed;
            const size_t n2 = std::max(gsum, jobs_[(size_t)head].need);
            int b2 = -1;
            size_t t2 = 0;
            if (!fit(n2, &b2, &t2)) {
              grp.pop_back();
              break;
            }
            gneed = n2;
            best = b2;
            best_total = t2;
          }
          for (size_t k = 0; k < grp.size(); ++k) queue_.pop_front();
          Worker& w = ws_[best];
          w.arena = std::max(w.arena, gneed);  // the arena the group grows it to
          w.busy = true;
          w.jobs = grp;
          for (long long id : grp) {
            JobState& j = jobs_[(size_t)id];
            j.worker = best;
            j.admitted = admitted_++;
          }
          running_ += (int)grp.size();
          peak_running_ = std::max(peak_running_, running_);
          peak_footprint_ = std::max(peak_footprint_, best_total);
          w.cv.notify_one();
          continue;
        }
        int victim = -1;  // the largest arena of an idle worker
        for (int w = 0; w < (int)ws_.size(); ++w)
          if (!ws_[w].busy && ws_[w].arena > 0 && (victim < 0 || ws_[w].arena > ws_[victim].arena))
            victim = w;
        if (victim >= 0) {
          ws_[victim].busy = true;
          lk.unlock();
          release_(victim);
          lk.lock();
          ws_[victim].arena = 0;
          ws_[victim].busy = false;
          continue;
        }
      }
      cv_disp_.wait(lk, [&] { return gen_ != seen || (stop_ && queue_.empty()); });
    }
  }

  void worker_loop(int w) {
    std::unique_lock<std::mutex> lk(m_);
    for (;;) {
      ws_[w].cv.wait(lk, [&] { return stop_ || !ws_[w].jobs.empty(); });
      if (ws_[w].jobs.empty()) return;
      const std::vector<long long> ids = ws_[w].jobs;
      const Clock::time_point t0 = Clock::now();
      for (long long id : ids) jobs_[(size_t)id].t_start = t0;
      lk.unlock();
      const int st = run_(w, ids);
      lk.lock();
      const Clock::time_point t1 = Clock::now();
      for (long long id : ids) {
        JobState& j = jobs_[(size_t)id];
        j.status = st;
        j.t_end = t1;
        j.done = true;
      }
      ws_[w].jobs.clear();
      ws_[w].busy = false;
      running_ -= (int)ids.size();
      ++gen_;
      cv_disp_.notify_one();
      cv_done_.notify_all();
    }
  }

  const size_t budget_;
  RunFn run_;
  ReleaseFn release_;
  int max_group_ = 1;
  std::mutex m_;
  std::condition_variable cv_disp_, cv_done_;
  std::deque<JobState> jobs_;  // element references stay valid as it grows
  std::deque<long long> queue_;
  std::vector<Worker> ws_;
  std::thread disp_;
  bool stop_ = false;
  unsigned long long gen_ = 0;  // bumped on every submission and completion
  int running_ = 0, peak_running_ = 0;
  long long rejected_ = 0, admitted_ = 0;
  size_t peak_footprint_ = 0;
  Clock::time_point first_{};
};

// Per-instance unrolling depth s by measured cost (the paper's b / s
// trade-off: a larger s reads Y once for more block updates but lengthens
// the dependent chain and the Gram tile).  Requests of one shape class share
// a table of measured seconds per block update for every candidate s (powers
// of two with s * b <= max_sb); a class first tries each candidate once, in
// the order 8, 16, 4, 32, 2, 1, 64, ..., then runs the candidate with the
// least mean cost so far (every run updates its running mean).
class STuner {
 public:
  struct Key {
    int method, xfmt, prec, b, lg_n, lg_k;  // lg_*: binade of N and K
    bool operator<(const Key& o) const {
      return std::tie(method, xfmt, prec, b, lg_n, lg_k) <
             std::tie(o.method, o.xfmt, o.prec, o.b, o.lg_n, o.lg_k);
    }
  };

  explicit STuner(int max_sb = 256) : max_sb_(max_sb) {}

  static int binade(long long v) {
    int e = 0;
    while (v > 1) {
      v >>= 1;
      ++e;
    }
    return e;
  }

  // candidates of a block size b, in the order they are first tried
  std::vector<int> candidates(int b) const {
    std::vector<int> out;
    for (int s : {8, 16, 4, 32, 2, 1, 64, 128, 256})
      if (b >= 1 && (long long)s * b <= max_sb_) out.push_back(s);
    if (out.empty()) out.push_back(1);
    return out;
  }

  // the largest candidate (its scratch bounds every candidate's)
  int largest(int b) const {
    int m = 1;
    for (int s : candidates(b)) m = std::max(m, s);
    return m;
  }

  int choose(const Key& k) {
    std::lock_guard<std::mutex> lk(m_);
    auto& t = table_[k];
    int best = -1;
    double best_cost = 0;
    for (int s : candidates(k.b)) {
      const auto it = t.find(s);
      if (it == t.end() || it->second.second == 0) return s;  // not measured yet
      const double c = it->second.first / (double)it->second.second;
      if (best < 0 || c < best_cost) {
        best = s;
        best_cost = c;
      }
    }
    return best;
  }

  // a run of `updates` block updates at depth s took `seconds`
  void record(const Key& k, int s, double seconds, long long updates) {
    if (updates <= 0 || !(seconds >= 0)) return;
    std::lock_guard<std::mutex> lk(m_);
    auto& e = table_[k][s];
    e.first += seconds / (double)updates;
    e.second += 1;
  }

  // mean measured seconds per block update at depth s (-1: none yet)
  double cost(const Key& k, int s) {
    std::lock_guard<std::mutex> lk(m_);
    const auto it = table_.find(k);
    if (it == table_.end()) return -1;
    const auto jt = it->second.find(s);
    if (jt == it->second.end() || jt->second.second == 0) return -1;
    return jt->second.first / (double)jt->second.second;
  }

 private:
  const int max_sb_;
  std::mutex m_;
  // per class: s -> (sum of seconds per update, runs)
  std::map<Key, std::map<int, std::pair<double, long long>>> table_;
};

}  // namespace caserve
