// Serving loop (host code): the C ABI of include/ca_serve.h over the
// scheduler of ca_serve_core.h.  Worker w owns a library context on its own
// non-blocking CUDA stream; a request runs as one synchronous ca_bcd_solve /
// ca_bdcd_solve call on its worker's host thread, so requests admitted
// together overlap on the device.  Its footprint is the scratch the solve
// takes from the context's arena (ca_solve_scratch_bytes); admission keeps
// the sum of the workers' arenas within the budget.  Requests submitted with
// opts.s = 0 get their unrolling depth from a measured-cost tuner shared by
// requests of the same shape class.
// Batching (ca_server_set_batching): the scheduler may start the queue's
// head together with the requests queued right behind it that a batched
// solve accepts (FP32 X, one tcgen05 Gram mode, b <= 16, s*b <= 128), as one
// ca_batch_solve on one worker: their outer steps share launches.
#include <cuda_runtime.h>

#include <deque>
#include <memory>
#include <mutex>
#include <vector>

#include "ca_bcd.h"
#include "ca_serve.h"
#include "ca_serve_core.h"

struct ca_server {
  int device = 0;
  size_t budget = 0;
  std::vector<cudaStream_t> streams;
  std::vector<ca_ctx*> ctxs;
  std::mutex m;                   // guards reqs and results
  std::deque<ca_request> reqs;    // by id; element references stay valid
  std::deque<ca_result> results;  // by id
  caserve::STuner tuner;           // s of requests submitted with opts.s = 0
  std::unique_ptr<caserve::Scheduler> sched;
};

namespace {

caserve::STuner::Key tuner_key(const ca_request& r) {
  const long long N = r.method == 0 ? r.d : r.n, K = r.method == 0 ? r.n : r.d;
  return {r.method, r.xfmt, r.opts.prec, r.opts.b, caserve::STuner::binade(N),
          caserve::STuner::binade(K)};
}

int run_batch(ca_server* s, int w, const std::vector<long long>& ids) {
  std::vector<ca_request> rs;
  {
    std::lock_guard<std::mutex> lk(s->m);
    for (long long id : ids) rs.push_back(s->reqs[(size_t)id]);
  }
  if (cudaSetDevice(s->device) != cudaSuccess) {
    cudaGetLastError();
    return CA_ERR_CUDA;
  }
  std::vector<ca_result> res(rs.size());
  const int st = ca_batch_solve(s->ctxs[(size_t)w], (int)rs.size(), rs.data(), CA_BATCH_GRAPH,
                                res.data());
  std::lock_guard<std::mutex> lk(s->m);
  for (size_t k = 0; k < ids.size(); ++k) {
    ca_result& out = s->results[(size_t)ids[k]];
    const size_t need = out.scratch_bytes;
    out = res[k];
    out.status = st;
    out.worker = w;
    out.scratch_bytes = need;
  }
  return st;
}

int run_request(ca_server* s, int w, long long id) {
  ca_request r;
  {
    std::lock_guard<std::mutex> lk(s->m);
    r = s->reqs[(size_t)id];
  }
  if (cudaSetDevice(s->device) != cudaSuccess) {
    cudaGetLastError();
    return CA_ERR_CUDA;
  }
  ca_ctx* ctx = s->ctxs[(size_t)w];
  const bool tuned = r.opts.s == 0;
  const caserve::STuner::Key key = tuner_key(r);
  if (tuned) r.opts.s = s->tuner.choose(key);
  const auto t0 = caserve::Clock::now();
  const int st = r.method == 0
                     ? ca_bcd_solve(ctx, r.xfmt, r.X, r.d, r.n, r.ld, r.y, &r.opts, r.x, r.aux)
                     : ca_bdcd_solve(ctx, r.xfmt, r.X, r.d, r.n, r.ld, r.y, &r.opts, r.x, r.aux);
  const double secs = std::chrono::duration<double>(caserve::Clock::now() - t0).count();
  ca_info info{};
  if (st == CA_OK) ca_solve_info(ctx, &info);
  if (tuned && st == CA_OK) s->tuner.record(key, r.opts.s, secs, info.h_done);
  std::lock_guard<std::mutex> lk(s->m);
  ca_result& out = s->results[(size_t)id];
  out.status = st;
  out.worker = w;
  out.s = r.opts.s;
  out.h_done = st == CA_OK ? info.h_done : 0;
  out.res0 = info.res0;
  out.res = info.res;
  out.gap = info.gap;
  out.fval = info.fval;
  out.bound = st == CA_OK ? info.bound : -1.0;
  return st;
}

// Memory of the server's device (or managed memory): the footprint admitted
// excludes host staging, and the solves run on that device.
bool on_device(const void* p, int device) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice && at.device == device) ||
         at.type == cudaMemoryTypeManaged;
}

void fill_times(ca_result* out, const caserve::JobState& j) {
  using ms = std::chrono::duration<double, std::milli>;
  out->queue_ms = ms(j.t_start - j.t_submit).count();
  out->run_ms = ms(j.t_end - j.t_start).count();
  out->latency_ms = ms(j.t_end - j.t_submit).count();
}

}  // namespace

extern "C" {

int ca_server_create(ca_server** out, int device, int workers, size_t budget_bytes) {
  if (!out || workers < 1 || budget_bytes < 1) return CA_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return CA_ERR_CUDA;
  }
  auto s = std::make_unique<ca_server>();
  s->device = device;
  s->budget = budget_bytes;
  for (int w = 0; w < workers; ++w) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      ca_server_destroy(s.release());
      return CA_ERR_CUDA;
    }
    s->streams.push_back(st);
    ca_ctx* ctx = nullptr;
    const int e = ca_bcd_init(&ctx, device, st, 0);
    if (e != CA_OK) {
      ca_server_destroy(s.release());
      return e;
    }
    s->ctxs.push_back(ctx);
  }
  ca_server* raw = s.get();
  s->sched = std::make_unique<caserve::Scheduler>(
      workers, budget_bytes,
      [raw](int w, const std::vector<long long>& ids) {
        return ids.size() == 1 ? run_request(raw, w, ids[0]) : run_batch(raw, w, ids);
      },
      [raw](int w) { ca_bcd_release_scratch(raw->ctxs[(size_t)w]); });
  *out = s.release();
  return CA_OK;
}

int ca_server_submit(ca_server* s, const ca_request* r, long long* id) {
  if (!s || !r || !id || !r->X || !r->y || !r->x) return CA_ERR_ARG;
  if (r->method != 0 && r->method != 1) return CA_ERR_ARG;
  if (r->method == 1 && !r->aux) return CA_ERR_ARG;
  for (const void* q : {r->X, static_cast<const void*>(r->y), static_cast<const void*>(r->x)})
    if (!on_device(q, s->device)) return CA_ERR_ARG;
  if (r->aux && !on_device(r->aux, s->device)) return CA_ERR_ARG;
  // s = 0: chosen at run time by measured cost; admit with the footprint of
  // the largest candidate, which bounds every candidate's
  ca_opts o = r->opts;
  if (o.s == 0) o.s = s->tuner.largest(o.b);
  size_t need = 0;
  const int e = ca_solve_scratch_bytes(s->ctxs[0], r->method, r->xfmt, r->d, r->n, &o, &need);
  if (e != CA_OK) return e;
  // the request's entries exist before the scheduler can start it (ids are
  // the submission order in both tables: submissions are serialised here)
  // its share of a batched solve (alone: the shared pools of one problem,
  // which bound its part of any group's pools)
  size_t bneed = 0;
  const bool bable = ca_batch_scratch_bytes(s->ctxs[0], 1, r, &bneed) == CA_OK;
  std::lock_guard<std::mutex> lk(s->m);
  s->reqs.push_back(*r);
  ca_result res{};
  res.worker = -1;
  res.scratch_bytes = need;
  if (need > s->budget) res.status = CA_ERR_OOM;  // the scheduler rejects it at once
  s->results.push_back(res);
  // batchable requests group by Gram mode (a batched solve runs one)
  *id = s->sched->submit(need, bable ? (long long)r->opts.prec : -1LL, bneed);
  return CA_OK;
}

int ca_server_set_batching(ca_server* s, int max_group) {
  if (!s || max_group < 1) return CA_ERR_ARG;
  s->sched->set_grouping(max_group);
  return CA_OK;
}

int ca_server_wait(ca_server* s, long long id, ca_result* out) {
  if (!s || !out || id < 0) return CA_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->m);
    if (id >= (long long)s->results.size()) return CA_ERR_ARG;
  }
  const caserve::JobState j = s->sched->wait(id);
  std::lock_guard<std::mutex> lk(s->m);
  *out = s->results[(size_t)id];
  if (j.status == caserve::Scheduler::kRejected) {
    out->status = CA_ERR_OOM;
    out->worker = -1;
  }
  fill_times(out, j);
  return CA_OK;
}

int ca_server_drain(ca_server* s) {
  if (!s) return CA_ERR_ARG;
  s->sched->drain();
  return CA_OK;
}

int ca_server_get_stats(ca_server* s, ca_server_stats* out) {
  if (!s || !out) return CA_ERR_ARG;
  const caserve::Stats st = s->sched->stats();
  out->submitted = st.submitted;
  out->completed = st.completed;
  out->rejected = st.rejected;
  out->p50_ms = st.p50_ms;
  out->p99_ms = st.p99_ms;
  out->mean_ms = st.mean_ms;
  out->max_ms = st.max_ms;
  out->wall_s = st.wall_s;
  out->peak_footprint = st.peak_footprint;
  out->peak_concurrency = st.peak_concurrency;
  double h = 0;
  {
    std::lock_guard<std::mutex> lk(s->m);
    for (const ca_result& r : s->results)
      if (r.status == CA_OK) h += (double)r.h_done;
  }
  out->block_updates_per_s = st.wall_s > 0 ? h / st.wall_s : 0.0;
  return CA_OK;
}

void ca_server_destroy(ca_server* s) {
  if (!s) return;
  s->sched.reset();  // drains, then joins the worker threads
  cudaSetDevice(s->device);
  for (ca_ctx* c : s->ctxs) ca_bcd_destroy(c);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
