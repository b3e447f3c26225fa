// ca_batch.cu -- ca_batch_solve: several dense ridge problems (primal CA-BCD,
// Algorithm 2, or dual CA-BDCD, Algorithm 4) of uneven sizes solved together.
//
// Each round runs one outer step of every unfinished problem in three shared
// launches:
//   * one Gram pass (steps a2+a3, with the deferred update a5 of the
//     problem's previous step fused in): the P CTAs split the concatenation
//     of all problems' 32-column atoms into stretches of equal HBM cost
//     (ca_batch_plan.h); a CTA walks the units of its stretch, one split-K
//     partial slot each;
//   * one reduction of every problem's partial slots, with the inversion of
//     its diagonal blocks (step a4);
//   * one chain CTA per problem (the s unrolled solves of eq. "recur" / its
//     dual analogue), so the dependent chains of different problems run at
//     the same time on different SMs.
// A small problem alone cannot fill the GPU (its Gram pass has fewer atoms
// than SMs, and its chain leaves all but one SM idle); in a shared round the
// problems fill each other's gaps.  Rounds whose launches differ only in
// pointers form a segment; with CA_BATCH_GRAPH a segment is captured into a
// CUDA graph once and launched as one.  Problems submitted with s = 0 get
// their unrolling depth by measured cost: trial rounds with s b = 128, 64
// and 32 rows per outer step, each timed with CUDA events, then the
// cheapest per block update (the paper's trade-off between fewer launches
// and a larger Gram, Sec. 5, measured instead of modelled).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ca_batch_plan.h"
#include "ca_bcd.h"
#include "ca_check.h"
#include "ca_internal.h"
#include "ca_kernels.cuh"
#include "ca_serve.h"

namespace {

using namespace caint;

constexpr int kBatchMaxSB = 128;     // s*b of a problem in a shared round
constexpr int kBatchMaxB = 16;       // b of a problem (chain with lookahead)
constexpr int kSegMaxRounds = 64;    // rounds per segment (graph size)
constexpr int kTrialSB[3] = {128, 64, 32};

struct BInst {
  DenseProblem pb;
  int method = 0, b = 0, s = 0, s_fixed = 0;
  long long H = 0, h = 0;  // block updates to do / done
  long long k = 0;         // outer steps done
  int recompute_every = 0;
  int* idx_all = nullptr;  // H x b sampled indices (from opts.h0)
  double* R = nullptr;
  float2* Rs = nullptr;
  double* pvec = nullptr;
  float2* Ginv = nullptr;
  double* delta[2] = {nullptr, nullptr};
  int par = 0;
  const int* prev_idx = nullptr;  // pending deferred update
  int prev_sb = 0;
  const double* prev_delta = nullptr;
  double* z = nullptr;  // primal: X^T w_H out (optional)
  bool done = false;
  ca_opts o{};
  CheckArgs ck{};       // stopping test (check_every > 0)
  ca_info info{};       // its outcome
};

int sb_class(int sb) { return sb <= 32 ? 32 : (sb <= 64 ? 64 : 128); }

// Rows of an outer step of problem q in the next round.
int step_rows(const BInst& q) { return (int)std::min<long long>(q.s, q.H - q.h) * q.b; }

// Reducing CTAs of a problem: its diagonal blocks, then 64 entries a pass.
int reduce_ctas(int sb, int scur) {
  const long long entries = (long long)sb * (sb + 1) / 2 + sb;
  return scur + (int)std::max<long long>(1, (entries + 63) / 64);
}

// Reduce-grid roles of a round: per problem its diagonal blocks and up to
// (128 * 129 / 2 + 128) / 64 passes of 64 entries.
size_t max_roles_of(int count) {
  return (size_t)count *
         (kBatchMaxSB + (kBatchMaxSB * (kBatchMaxSB + 1) / 2 + kBatchMaxSB + 63) / 64);
}

// Checks the requests and sizes the scratch of a batched solve (the arena
// bytes ca_batch_solve takes from ctx).
int batch_need(ca_ctx* ctx, int count, const ca_request* reqs, size_t* out, bool* any_tuned_out) {
  const int P = std::max(1, ctx->num_sms - 1);
  const int prec = reqs[0].opts.prec;
  if (!tc_prec(prec)) return CA_ERR_UNSUPPORTED;  // FP32 X with a tcgen05 Gram mode
  size_t need = 8 * 256;
  bool any_tuned = false;
  for (int i = 0; i < count; ++i) {
    const ca_request& r = reqs[i];
    const ca_opts& o = r.opts;
    if (r.method != 0 && r.method != 1) return CA_ERR_ARG;
    if (r.xfmt != CA_DENSE_F32 && r.xfmt != CA_DENSE_F32_PANELS) return CA_ERR_UNSUPPORTED;
    if (o.prec != prec) return CA_ERR_ARG;  // one Gram mode per batch
    const long long d = r.d, n = r.n;
    if (!r.X || !r.y || !r.x || d < 1 || n < 1) return CA_ERR_ARG;
    if (r.method == 1 && !r.aux) return CA_ERR_ARG;
    const long long N = r.method == 0 ? d : n, K = r.method == 0 ? n : d;
    ca_opts oc = o;
    if (oc.s == 0) {
      oc.s = 1;  // checked with the smallest depth; the tuner keeps s b <= 128
      any_tuned = true;
    }
    CA_TRY(check_opts(&oc, N));
    if (o.b > kBatchMaxB || (o.s > 0 && (long long)std::min<long long>(o.s, o.H) * o.b > kBatchMaxSB))
      return CA_ERR_UNSUPPORTED;
    if (o.solve != CA_SOLVE_DF) return CA_ERR_UNSUPPORTED;
    const bool pre = r.xfmt == CA_DENSE_F32_PANELS;
    if (!pre && (r.ld < K || (r.ld & 3) != 0 || (reinterpret_cast<uintptr_t>(r.X) & 15) != 0))
      return CA_ERR_ARG;
    for (const void* q : {r.X, (const void*)r.y, (const void*)r.x})
      if (!is_device_ptr(q)) return CA_ERR_ARG;
    if (r.aux && !is_device_ptr(r.aux)) return CA_ERR_ARG;
    const long long Kp = (K + 31) / 32 * 32;
    if (!pre) need += align256(panel_bytes(N, K)) + 256;
    need += align256((size_t)Kp * 8) + align256((size_t)N * 8) + align256((size_t)o.H * o.b * 4);
    if (r.method == 0) need += align256((size_t)K * 8);  // rho
    need += 2 * align256((size_t)kBatchMaxSB * kBatchMaxSB * 8) + 3 * align256((size_t)kBatchMaxSB * 8) +
            align256((size_t)kBatchMaxSB * kBatchMaxB * 8);
    if (prec == CA_GRAM_FP16_SCALED) need += align256((size_t)N * 4);
    if (o.check_every > 0) need += align256((size_t)check_rows(&o, N, K) * 8) + 512;
  }
  // shared: partial slot pools (at most P + count units), round arrays
  const size_t nslot_max = (size_t)P + (size_t)count;
  need += align256(nslot_max * kBatchMaxSB * kBatchMaxSB * 4) + align256(nslot_max * kBatchMaxSB * 8);
  need += align256((size_t)kSegMaxRounds * count * sizeof(GramInst)) +
          align256((size_t)kSegMaxRounds * count * sizeof(RedInst)) +
          align256(nslot_max * sizeof(GramUnit)) + align256((size_t)(P + 1) * sizeof(int));
  need += align256(max_roles_of(count) * sizeof(RedRole)) + 4096;
  *out = need;
  *any_tuned_out = any_tuned;
  return CA_OK;
}

}  // namespace

using namespace caint;

extern "C" int ca_batch_scratch_bytes(ca_ctx* ctx, int count, const ca_request* reqs,
                                      size_t* bytes) {
  t_cur_ctx = ctx;
  if (!ctx || count < 1 || !reqs || !bytes) return CA_ERR_ARG;
  bool tuned = false;
  return batch_need(ctx, count, reqs, bytes, &tuned);
}

extern "C" int ca_batch_solve(ca_ctx* ctx, int count, const ca_request* reqs, int flags,
                              ca_result* out) {
  t_cur_ctx = ctx;
  if (!ctx || count < 1 || !reqs || !out) return CA_ERR_ARG;
  if (flags & ~CA_BATCH_GRAPH) return CA_ERR_ARG;
  ctx->prof.cls.clear();
  CA_TRY_CUDA(cudaSetDevice(ctx->device));
  const int prec = reqs[0].opts.prec;
  if (!tc_prec(prec)) return CA_ERR_UNSUPPORTED;  // FP32 X with a tcgen05 Gram mode
  const int three = prec == CA_GRAM_FP32_EXACT ? 1 : prec == CA_GRAM_BF16X3 ? 2
                    : prec == CA_GRAM_FP16_SCALED ? 3 : 0;
  const int P = std::max(1, ctx->num_sms - 1);
  std::vector<BInst> in((size_t)count);
  size_t need = 0;
  bool any_tuned = false;
  CA_TRY(batch_need(ctx, count, reqs, &need, &any_tuned));
  const size_t nslot_max = (size_t)P + (size_t)count;
  const size_t max_roles = max_roles_of(count);
  CA_TRY(ensure_arena(ctx, need));
  Carve cv{static_cast<char*>(ctx->arena)};
  CA_TRY_CUDA(cudaMemsetAsync(ctx->d_err, 0, 33 * sizeof(unsigned), ctx->stream));

  // per-problem set-up: panels, v0 = its definition, the sampled indices
  for (int i = 0; i < count; ++i) {
    const ca_request& r = reqs[i];
    const ca_opts& o = r.opts;
    BInst& q = in[(size_t)i];
    const long long d = r.d, n = r.n;
    const long long N = r.method == 0 ? d : n, K = r.method == 0 ? n : d;
    const double ln = o.lam * (double)n;
    q.method = r.method;
    q.b = o.b;
    q.s_fixed = o.s;
    q.s = o.s > 0 ? o.s : kTrialSB[0] / o.b;
    q.H = o.H;
    q.recompute_every = o.recompute_every;
    q.o = o;
    q.info = ca_info{o.H, 0, 0.0, 0.0, 0.0, 0.0, -1.0};
    DenseProblem& pb = q.pb;
    pb.xfmt = CA_DENSE_F32;
    pb.panel = true;
    pb.method = r.method;
    pb.N = N;
    pb.K = K;
    pb.lda = r.ld;
    const float* Ap = static_cast<const float*>(r.X);
    if (r.xfmt != CA_DENSE_F32_PANELS) {
      float* pk = cv.take<float>(panel_bytes(N, K) / 4);
      launch_pack(ctx, Ap, N, K, r.ld, pk);
      Ap = pk;
    }
    pb.A = Ap;
    const long long Kp = (K + 31) / 32 * 32;
    pb.v2 = cv.take<float2>((size_t)Kp);
    pb.x2 = cv.take<float2>((size_t)N);
    q.idx_all = cv.take<int>((size_t)o.H * o.b);
    pb.x = r.x;
    if (r.method == 0) {
      pb.v = cv.take<double>((size_t)K);  // rho = y - X^T w
      pb.yv = nullptr;
      pb.cG = 1.0 / (double)n;
      pb.cI = o.lam;
      pb.cP = 1.0 / (double)n;
      pb.cY = 0.0;
      pb.cU = 1.0;
      pb.y0 = r.y;
      pb.c0 = 1.0;
      pb.c1 = -1.0;
      q.z = r.aux;
    } else {
      pb.v = r.aux;  // w = -X alpha/(lambda n)
      pb.yv = r.y;
      pb.cG = 1.0 / ln;
      pb.cI = 1.0;
      pb.cP = 1.0;
      pb.cY = 1.0;
      pb.cU = 1.0 / ln;
      pb.y0 = nullptr;
      pb.c0 = 0.0;
      pb.c1 = -1.0 / ln;
    }
    q.R = cv.take<double>((size_t)kBatchMaxSB * kBatchMaxSB);
    q.Rs = cv.take<float2>((size_t)kBatchMaxSB * kBatchMaxSB);
    q.pvec = cv.take<double>(kBatchMaxSB);
    q.delta[0] = cv.take<double>(kBatchMaxSB);
    q.delta[1] = cv.take<double>(kBatchMaxSB);
    q.Ginv = cv.take<float2>((size_t)kBatchMaxSB * kBatchMaxB);
    if (prec == CA_GRAM_FP16_SCALED) {
      float* rs = cv.take<float>((size_t)N);
      launch_row_scale_ctx(ctx, static_cast<const float*>(pb.A), N, K, rs);
      pb.rscale = rs;
    }
    CA_TRY(launch_recompute(ctx, pb, pb.v, pb.y0, pb.c0, pb.c1));  // v0 and its split
    k_sample<<<(unsigned)((o.H + 7) / 8), 256, 0, ctx->stream>>>(o.seed, o.h0, o.H, o.b, N,
                                                                  q.idx_all);
    ctx->prof.kernel_launches += 1;
    CA_TRY_CUDA(cudaGetLastError());
    if (o.check_every > 0) {  // stopping test: scratch, and the check at the start
      const long long rows = check_rows(&o, N, K);
      double* rq = cv.take<double>((size_t)rows);
      double* racc = cv.take<double>(kCheckAcc);
      CA_TRY_CUDA(cudaMemsetAsync(rq, 0, (size_t)rows * 8, ctx->stream));
      q.ck = CheckArgs{r.method, o.stop == CA_STOP_OBJECTIVE, o.lam, pb.A, false, true, pb.lda,
                       N, K, pb.v, pb.v2, nullptr, rq, racc, pb.x, pb.yv, pb.cP, pb.cI, pb.cY};
      CA_TRY(full_check(ctx, q.ck, 0, &q.info.res0, &q.info.gap, &q.info.fval));
      q.info.res = q.info.res0;
      q.info.bound = q.ck.objective ? certified_bound(q.info.fval, q.info.gap) : -1.0;
    }
  }
  float* part_pool = cv.take<float>(nslot_max * kBatchMaxSB * kBatchMaxSB);
  double* ppart_pool = cv.take<double>(nslot_max * kBatchMaxSB);
  GramInst* d_ginst = cv.take<GramInst>((size_t)kSegMaxRounds * count);
  RedInst* d_rinst = cv.take<RedInst>((size_t)kSegMaxRounds * count);
  GramUnit* d_units = cv.take<GramUnit>(nslot_max);
  int* d_ubeg = cv.take<int>((size_t)P + 1);
  RedRole* d_roles = cv.take<RedRole>(max_roles);

  std::vector<GramInst> h_ginst;
  std::vector<RedInst> h_rinst;
  std::vector<GramUnit> h_units;
  std::vector<int> h_ubeg;
  std::vector<RedRole> h_roles;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  CA_TRY_CUDA(cudaEventCreate(&ev0));
  CA_TRY_CUDA(cudaEventCreate(&ev1));
  int trial = any_tuned ? 0 : 3;  // next trial depth (3: trials over)
  double trial_cost[3] = {0, 0, 0};
  bool warm = !any_tuned;         // the first round runs untimed
  int status = CA_OK;
  const bool graph = (flags & CA_BATCH_GRAPH) && ctx->stream != nullptr;

  auto run_segment = [&](const std::vector<int>& act, int rounds, bool timed) -> int {
    const int na = (int)act.size();
    // the plan: every active problem's atoms over P CTAs, one slot pool
    std::vector<cabatch::Instance> pi;
    int sbp = 32, bmax = 8, sbmax = 1;
    for (int a : act) {
      const BInst& q = in[(size_t)a];
      const int sb = step_rows(q);
      pi.push_back(cabatch::Instance{q.pb.K, sb});
      // (the tile also holds the previous step's rows of the fused update)
      sbp = std::max(sbp, sb_class(std::max(sb, q.prev_sb)));
      bmax = std::max(bmax, q.b <= 8 ? 8 : 16);
      sbmax = std::max(sbmax, sb);
    }
    cabatch::Plan pl;
    if (!cabatch::plan(pi, P, &pl)) return CA_ERR_ARG;
    std::vector<int> slot_base((size_t)na, 0);
    for (int j = 1; j < na; ++j) slot_base[(size_t)j] = slot_base[(size_t)j - 1] + pl.nslots[(size_t)j - 1];
    h_units.clear();
    h_ubeg.assign((size_t)P + 1, 0);
    for (int c = 0; c < P; ++c) {
      h_ubeg[(size_t)c] = (int)h_units.size();
      for (const cabatch::Unit& u : pl.cta[(size_t)c]) h_units.push_back(GramUnit{u.inst, u.slot, u.a0, u.a1});
    }
    h_ubeg[(size_t)P] = (int)h_units.size();
    // reduce roles: each problem's CTAs (same in every round of the segment)
    h_roles.clear();
    for (int j = 0; j < na; ++j) {
      const BInst& q = in[(size_t)act[(size_t)j]];
      const int sb = step_rows(q), sc = sb / q.b;
      const int nc = reduce_ctas(sb, sc);
      for (int t = 0; t < nc; ++t) h_roles.push_back(RedRole{j, t, nc});
    }
    // per-round descriptors
    h_ginst.assign((size_t)rounds * na, GramInst{});
    h_rinst.assign((size_t)rounds * na, RedInst{});
    for (int rr = 0; rr < rounds; ++rr) {
      for (int j = 0; j < na; ++j) {
        BInst& q = in[(size_t)act[(size_t)j]];
        const int sb = step_rows(q), sc = sb / q.b;
        const int* idx = q.idx_all + (size_t)q.h * q.b;
        double* dl = q.delta[q.par];
        float* part = part_pool + (size_t)slot_base[(size_t)j] * sbp * sbp;
        double* ppart = ppart_pool + (size_t)slot_base[(size_t)j] * sbp;
        GramUpdate u{q.prev_idx, q.prev_sb, q.prev_delta, q.pb.cU, q.pb.v2, q.pb.rscale, false};
        h_ginst[(size_t)rr * na + j] = GramInst{static_cast<const float*>(q.pb.A), q.pb.lda, q.pb.N,
                                                q.pb.K, idx, sb, q.pb.v2, part, ppart, u};
        SolveArgs sa{idx, q.pb.N, q.b, sc, sb, sbp, q.pb.cG, q.pb.cI, q.pb.cP, q.pb.cY, q.pb.x,
                     q.pb.yv, dl};
        h_rinst[(size_t)rr * na + j] = RedInst{part, ppart, pl.nslots[(size_t)j], sbp, sc, q.R, q.Rs,
                                               q.pvec, q.Ginv, sa};
        // advance: this step's update is pending for the next round
        q.prev_idx = idx;
        q.prev_sb = sb;
        q.prev_delta = dl;
        q.par ^= 1;
        q.h += sc;
        q.k += 1;
      }
    }
    CA_TRY_CUDA(cudaMemcpyAsync(d_ginst, h_ginst.data(), h_ginst.size() * sizeof(GramInst),
                                cudaMemcpyHostToDevice, ctx->stream));
    CA_TRY_CUDA(cudaMemcpyAsync(d_rinst, h_rinst.data(), h_rinst.size() * sizeof(RedInst),
                                cudaMemcpyHostToDevice, ctx->stream));
    CA_TRY_CUDA(cudaMemcpyAsync(d_units, h_units.data(), h_units.size() * sizeof(GramUnit),
                                cudaMemcpyHostToDevice, ctx->stream));
    CA_TRY_CUDA(cudaMemcpyAsync(d_ubeg, h_ubeg.data(), h_ubeg.size() * sizeof(int),
                                cudaMemcpyHostToDevice, ctx->stream));
    CA_TRY_CUDA(cudaMemcpyAsync(d_roles, h_roles.data(), h_roles.size() * sizeof(RedRole),
                                cudaMemcpyHostToDevice, ctx->stream));
    const size_t csm = chain_smem(bmax, sbmax);
    auto launch_rounds = [&]() -> int {
      for (int rr = 0; rr < rounds; ++rr) {
        GramBatchArgs bt{d_ginst + (size_t)rr * na, d_units, d_ubeg, rr > 0};
        prof_mark(ctx, PC_GRAM);
        int e = launch_gram_tc_batch(bt, P, sbp, three, ctx->d_err, ctx->stream);
        prof_mark(ctx, PC_GRAM);
        if (e) return cuda_fail((cudaError_t)e, __LINE__);
        prof_mark(ctx, PC_SOLVE);
        e = launch_reduce_batch((int)h_roles.size(), ctx->stream, d_rinst + (size_t)rr * na, d_roles,
                                ctx->d_err);
        if (e) return cuda_fail((cudaError_t)e, __LINE__);
        e = launch_chain_batch(na, bmax, csm, ctx->stream, d_rinst + (size_t)rr * na, ctx->d_err);
        prof_mark(ctx, PC_SOLVE);
        if (e) return cuda_fail((cudaError_t)e, __LINE__);
        ctx->prof.kernel_launches += 3;
      }
      return CA_OK;
    };
    if (timed) CA_TRY_CUDA(cudaEventRecord(ev0, ctx->stream));
    if (graph && !ctx->prof.on) {
      cudaGraph_t gr = nullptr;
      cudaGraphExec_t ge = nullptr;
      CA_TRY_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      const int e = launch_rounds();
      const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &gr);
      if (e != CA_OK) {
        if (gr) cudaGraphDestroy(gr);
        return e;
      }
      CA_TRY_CUDA(ce);
      const cudaError_t ie = cudaGraphInstantiate(&ge, gr, 0);
      cudaGraphDestroy(gr);
      CA_TRY_CUDA(ie);
      const cudaError_t le = cudaGraphLaunch(ge, ctx->stream);
      if (le == cudaSuccess && timed) cudaEventRecord(ev1, ctx->stream);
      // the next segment rewrites the descriptor arrays: wait for this one
      const cudaError_t se = le == cudaSuccess ? cudaStreamSynchronize(ctx->stream) : le;
      cudaGraphExecDestroy(ge);
      CA_TRY_CUDA(se);
      return CA_OK;
    }
    CA_TRY(launch_rounds());
    if (timed) CA_TRY_CUDA(cudaEventRecord(ev1, ctx->stream));
    // the next segment rewrites the descriptor arrays: wait for this one
    CA_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    return CA_OK;
  };

  for (;;) {
    std::vector<int> act;
    for (int i = 0; i < count; ++i)
      if (!in[(size_t)i].done) act.push_back(i);
    if (act.empty()) break;
    // depth of the tuned problems for this segment (trial rounds, then the best)
    bool timed = false;
    if (any_tuned) {
      int t = 3;
      if (!warm) t = 0;
      else if (trial < 3) t = trial;
      int sbt = kTrialSB[t < 3 ? t : 0];
      if (t == 3) {
        const int best = (int)(std::min_element(trial_cost, trial_cost + 3) - trial_cost);
        sbt = kTrialSB[best];
      }
      for (int a : act) {
        BInst& q = in[(size_t)a];
        if (q.s_fixed == 0) q.s = std::max(1, sbt / q.b);
      }
      timed = warm && trial < 3;
    }
    // rounds of this segment: the active set and every step's rows stay the
    // same, no recomputation falls inside
    int rounds = (timed || (any_tuned && !warm)) ? 1 : kSegMaxRounds;
    for (int a : act) {
      const BInst& q = in[(size_t)a];
      const long long full_steps = (q.H - q.h) / q.s;  // steps with s blocks
      long long r = full_steps > 0 ? full_steps : 1;   // (else one short step)
      if (q.recompute_every > 0) {
        const long long to_due = q.recompute_every - (q.k % q.recompute_every);
        r = std::min(r, to_due);
      }
      if (q.o.check_every > 0) {
        const long long to_check = q.o.check_every - (q.k % q.o.check_every);
        r = std::min(r, to_check);
      }
      rounds = (int)std::min<long long>(rounds, r);
    }
    long long blocks = 0;
    for (int a : act) blocks += std::min<long long>(in[(size_t)a].s, in[(size_t)a].H - in[(size_t)a].h);
    status = run_segment(act, rounds, timed);
    if (status != CA_OK) break;
    if (timed) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev0, ev1);
      trial_cost[trial] = (double)ms / (double)std::max(1LL, blocks * rounds);
      ++trial;
    }
    if (any_tuned && !warm) warm = true;
    // after the segment: finished problems and due recomputations apply their
    // pending update now (as the solve alone does)
    for (int a : act) {
      BInst& q = in[(size_t)a];
      const bool fin = q.h >= q.H;
      const bool due = q.recompute_every > 0 && q.k % q.recompute_every == 0;
      const bool chk = q.o.check_every > 0 && (fin || q.k % q.o.check_every == 0);
      if (fin || due || chk) {
        status = launch_update_alone(ctx, q.pb, q.prev_idx, q.prev_sb, q.prev_delta);
        if (status != CA_OK) break;
        q.prev_sb = 0;
        q.prev_idx = nullptr;
        q.prev_delta = nullptr;
        // a check first rebuilds v from its definition (FP32 X: the updates
        // round their products to FP32), as the solve alone does
        if (due || chk) {
          status = launch_recompute(ctx, q.pb, q.pb.v, q.pb.y0, q.pb.c0, q.pb.c1);
          if (status != CA_OK) break;
        }
      }
      if (chk) {
        status = full_check(ctx, q.ck, q.h, &q.info.res, &q.info.gap, &q.info.fval);
        if (status != CA_OK) break;
        ++q.info.checks;
        q.info.bound = q.ck.objective ? certified_bound(q.info.fval, q.info.gap) : -1.0;
        if (!fin && check_says_stop(&q.o, q.info)) {
          q.info.h_done = q.h;
          q.done = true;
        }
      }
      if (fin) q.done = true;
      if (q.done && q.method == 0 && q.z) {
        status = launch_recompute(ctx, q.pb, q.z, nullptr, 0.0, 1.0);  // z = X^T w_H
        if (status != CA_OK) break;
      }
    }
    if (status != CA_OK) break;
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  const int fst = finish(ctx);
  if (status == CA_OK) status = fst;
  ctx->trace.clear();  // (the checks of several problems: no single trace)
  for (int i = 0; i < count; ++i) {
    const BInst& q = in[(size_t)i];
    ca_result& o = out[i];
    std::memset(&o, 0, sizeof(o));
    o.status = status;
    o.worker = -1;
    o.s = q.s;
    o.h_done = status == CA_OK ? q.h : 0;
    o.res0 = q.info.res0;
    o.res = q.info.res;
    o.gap = q.info.gap;
    o.fval = q.ck.objective ? q.info.fval : 0.0;
    o.bound = status == CA_OK ? q.info.bound : -1.0;
  }
  return status;
}
