// ca_api.cu -- the C ABI (include/ca_bcd.h): contexts, scratch, staging of
// host buffers and the outer-step loops of CA-BCD (Alg. 2) and CA-BDCD (Alg. 4).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ca_bcd.h"
#include "ca_check.h"
#include "ca_internal.h"
#include "ca_kernels.cuh"

namespace caint {

thread_local ca_ctx* t_cur_ctx = nullptr;  // context of the running entry point

int cuda_fail(cudaError_t e, int line) {
  if (t_cur_ctx)
    snprintf(t_cur_ctx->last_error, sizeof(t_cur_ctx->last_error), "ca_api.cu:%d: %s (%s)", line,
             cudaGetErrorName(e), cudaGetErrorString(e));
  return CA_ERR_CUDA;
}

int cuda_status_at(cudaError_t e, int line) { return e == cudaSuccess ? CA_OK : cuda_fail(e, line); }



bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device-accessible address of page-locked, mapped host memory (the same
// address under unified addressing), or nullptr for any other pointer.
const void* mapped_host_ptr(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int ensure_arena(ca_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->arena_bytes) return CA_OK;
  if (ctx->scratch_max && bytes > ctx->scratch_max) return CA_ERR_OOM;
  if (ctx->arena) {
    CA_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->arena);
    ctx->arena = nullptr;
    ctx->arena_bytes = 0;
  }
  if (cudaMalloc(&ctx->arena, bytes) != cudaSuccess) {
    cudaGetLastError();
    return CA_ERR_OOM;
  }
  ctx->arena_bytes = bytes;
  return CA_OK;
}

int status_from_err(unsigned e) {
  if (e & CA_DEV_ERR_TIMEOUT) return CA_ERR_TIMEOUT;
  if (e & CA_DEV_ERR_NONFINITE) return CA_ERR_NONFINITE;
  if (e & CA_DEV_ERR_NOT_SPD) return CA_ERR_NOT_SPD;
  if (e & CA_DEV_ERR_ARG) return CA_ERR_ARG;
  return CA_OK;
}

int finish(ca_ctx* ctx) {
  CA_TRY_CUDA(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost,
                              ctx->stream));
  CA_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->prof.on) {
    Profile& pr = ctx->prof;
    for (size_t i = 0; i + 1 < pr.cls.size(); i += 2) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, pr.pool[i], pr.pool[i + 1]);
      pr.ms[pr.cls[i]] += ms;
      pr.launches[pr.cls[i]] += 1;
    }
    pr.cls.clear();
  }
  return status_from_err(*ctx->h_err);
}

// Record an event of class cls on the context's stream (profiling only).
void prof_mark(ca_ctx* ctx, int cls) {
  Profile& pr = ctx->prof;
  if (!pr.on) return;
  if (pr.cls.size() == pr.pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    pr.pool.push_back(e);
  }
  cudaEventRecord(pr.pool[pr.cls.size()], ctx->stream);
  pr.cls.push_back(cls);
}

int check_opts(const ca_opts* o, long long N) {
  if (!o) return CA_ERR_ARG;
  if (o->b < 1 || (long long)o->b > N || o->s < 1 || o->H < 1 || o->h0 < 0) return CA_ERR_ARG;
  if (!(o->lam > 0.0) || !std::isfinite(o->lam)) return CA_ERR_ARG;
  if (o->recompute_every < 0) return CA_ERR_ARG;
  if (o->check_every < 0 || !(o->tol >= 0.0) || !std::isfinite(o->tol)) return CA_ERR_ARG;
  if (o->stop != CA_STOP_RESIDUAL && o->stop != CA_STOP_OBJECTIVE) return CA_ERR_ARG;
  if (o->solve != CA_SOLVE_DF && o->solve != CA_SOLVE_F64) return CA_ERR_ARG;
  if (o->prec < CA_GRAM_F64 || o->prec > CA_GRAM_FP16_SCALED) return CA_ERR_ARG;
  if (N > 2147483647LL) return CA_ERR_UNSUPPORTED;
  if (o->b > kMaxB) return CA_ERR_UNSUPPORTED;
  const long long sbm = (long long)std::min<long long>(o->s, o->H) * o->b;
  if (sbm > kMaxSB) return CA_ERR_UNSUPPORTED;
  return CA_OK;
}


// Stopping test (Sec. 5.1.5).  A check forms ||r||_2 of the current
// iterate, r = cP A v - cI x - cY y (one pass over A, then a wait for the
// GPU), and the duality gap of Sec. 2.2 that it gives in closed form:
// primal (method 0; x = w, v = rho = y - X^T w, n = K), at the dual point
// alpha = X^T w - y, gap = ||r||^2/(2 lambda); dual (method 1; x = alpha,
// v = w = -X alpha/(lambda n), n = N), gap = ||r||^2/(2n).  Under the
// objective rule it also forms f(w) of the model from the maintained vectors:
// primal lambda/2 ||w||^2 + ||rho||^2/(2n); dual ||y||^2/(2n) - D(alpha) +
// gap with D(alpha) = lambda/2 ||w||^2 + ||alpha + y||^2/(2n).
int full_check(ca_ctx* ctx, const CheckArgs& c, long long h_at, double* res, double* gap,
               double* fval) {
  const int nacc = c.objective ? kCheckAcc : 1;
  CA_TRY_CUDA(cudaMemsetAsync(c.racc, 0, nacc * sizeof(double), ctx->stream));
  prof_mark(ctx, PC_OTHER);
  launch_residual(ctx->stream, ctx->num_sms, c.A, c.f64, c.panel, c.lda, c.N, c.K, c.v, c.v2,
                  c.csr, c.rq, c.x, c.yv, c.cP, c.cI, c.cY, c.racc);
  ctx->prof.kernel_launches += 2;
  if (c.objective) {
    launch_sumsq(ctx->stream, ctx->num_sms, c.rq, c.v, nullptr, c.K, 1.0, 0.0, c.racc + 1);
    if (c.method == 0) {  // ||w||^2
      launch_sumsq(ctx->stream, ctx->num_sms, c.rq, c.x, nullptr, c.N, 1.0, 0.0, c.racc + 2);
      ctx->prof.kernel_launches += 2;
    } else {              // ||alpha + y||^2, ||y||^2
      launch_sumsq(ctx->stream, ctx->num_sms, c.rq, c.x, c.yv, c.N, 1.0, 1.0, c.racc + 2);
      launch_sumsq(ctx->stream, ctx->num_sms, c.rq, c.yv, nullptr, c.N, 1.0, 0.0, c.racc + 3);
      ctx->prof.kernel_launches += 3;
    }
  }
  prof_mark(ctx, PC_OTHER);
  CA_TRY_CUDA(cudaGetLastError());
  double* h = reinterpret_cast<double*>(reinterpret_cast<char*>(ctx->h_err) + 32);
  CA_TRY_CUDA(cudaMemcpyAsync(h, c.racc, nacc * sizeof(double), cudaMemcpyDeviceToHost,
                              ctx->stream));
  CA_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
  check_values(c.method, c.objective, c.lam, c.N, c.K, h, res, gap, fval);
  ctx->info.bound = c.objective ? certified_bound(*fval, *gap) : -1.0;
  ctx->trace.push_back(ca_check{h_at, *res, *gap, c.objective ? *fval : 0.0});
  return CA_OK;
}

// The decision of a check after the start (tol = 0: never stop).
bool check_says_stop(const ca_opts* o, const ca_info& in) {
  return check_stops(o->stop == CA_STOP_OBJECTIVE, o->tol, in.res0, in.res, in.gap, in.fval);
}

int launch_recompute(ca_ctx* ctx, const DenseProblem& pb, double* vout, const double* y0,
                     double c0, double c1) {
  const long long K = pb.K, N = pb.N;
  const long long gx = (K + 1023) / 1024;
  long long ysplit = (4LL * ctx->num_sms + gx - 1) / gx;  // about 4 CTAs per SM
  ysplit = std::max(1LL, std::min(ysplit, (N + 63) / 64));
  const long long rps = (N + ysplit - 1) / ysplit;
  ysplit = (N + rps - 1) / rps;
  dim3 grid((unsigned)gx, (unsigned)ysplit);
  prof_mark(ctx, PC_OTHER);
  // x = 0 (a solve started from zero) leaves v = c0 y0 without reading A:
  // the recomputation skips its pass when k_nonzero finds no nonzero x
  unsigned* nz = ctx->d_err + 56;
  k_axpby_init<<<(unsigned)((K + 255) / 256), 256, 0, ctx->stream>>>(y0, c0, K, vout, nz);
  k_nonzero<<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(
      pb.x, N, pb.xfmt == CA_DENSE_F32 ? pb.x2 : nullptr, nz);
  launch_recompute_dense(pb.xfmt == CA_DENSE_F64, grid, ctx->stream, pb.A, pb.lda, N, K, pb.x, pb.x2,
                         c1, rps, vout, pb.panel, nz);
  ctx->prof.kernel_launches += 3;
  if (vout == pb.v && pb.v2) {
    const long long Kp = (K + 31) / 32 * 32;
    k_split<<<(unsigned)((Kp + 255) / 256), 256, 0, ctx->stream>>>(pb.v, K, Kp, pb.v2);
    ctx->prof.kernel_launches += 1;
  }
  prof_mark(ctx, PC_OTHER);
  return cuda_status(cudaGetLastError());
}

// Gram precisions that run on the tcgen05 path (FP32 X only).
bool tc_prec(int prec) {
  return prec == CA_GRAM_TF32 || prec == CA_GRAM_FP32_EXACT || prec == CA_GRAM_BF16X3 ||
         prec == CA_GRAM_FP16_SCALED;
}

// Split-K plan of the a2+a3 pass for a given s*b bound.
struct GramPlan {
  bool tc;
  int three, sbp, P, ntiles;
  long long chunks_per_split;
};

GramPlan gram_plan(ca_ctx* ctx, int xfmt, int prec, int sbm, long long K) {
  GramPlan g{};
  g.tc = (xfmt == CA_DENSE_F32) && tc_prec(prec);
  g.three = prec == CA_GRAM_FP32_EXACT ? 1
            : prec == CA_GRAM_BF16X3    ? 2
            : prec == CA_GRAM_FP16_SCALED ? 3
                                          : 0;
  if (g.tc) {
    g.sbp = sbm <= 32 ? 32 : (sbm <= 64 ? 64 : (sbm <= 128 ? 128 : 256));
    g.P = (int)std::min<long long>(ctx->num_sms, (K + 31) / 32);
  } else {
    g.sbp = (sbm + 63) / 64 * 64;
    const int t = g.sbp / 64;
    g.ntiles = t * (t + 1) / 2;
    const long long nchunks = (K + 31) / 32;
    long long Pm = std::max(1LL, (long long)(2 * ctx->num_sms) / g.ntiles);
    Pm = std::min(Pm, nchunks);
    const long long cap = std::max(1LL, (long long)((256ull << 20) / ((size_t)g.sbp * g.sbp * 8)));
    Pm = std::min(Pm, cap);
    g.chunks_per_split = (nchunks + Pm - 1) / Pm;
    g.P = (int)((nchunks + g.chunks_per_split - 1) / g.chunks_per_split);
  }
  return g;
}

// a2+a3: split-K partials of Y Y^T and Y v for the sampled rows idx[0..sb).
// early: the preceding kernel in the stream is the reduce + chain launch,
// which writes nothing the Gram prologue reads (see GramUpdate::early).
int launch_gram(ca_ctx* ctx, const GramPlan& g, int xfmt, const void* A, long long lda, long long N,
                long long K, const int* idx, int sb, const double* v, const float2* v2, void* part,
                double* ppart, bool panel = false, const float* rscale = nullptr,
                bool early = false) {
  if (g.tc) {
    GramUpdate none{};
    none.rscale = rscale;
    none.early = early;
    const int e = launch_gram_tc(static_cast<const float*>(A), lda, N, K, idx, sb, v2, g.P, g.sbp,
                                 static_cast<float*>(part), ppart, ctx->d_err, g.three, ctx->stream,
                                 &none, panel);
    return e == 0 ? CA_OK : CA_ERR_CUDA;
  }
  launch_gram_simt(xfmt == CA_DENSE_F64, dim3(g.P, g.ntiles), ctx->stream, A, lda, N, K, idx, sb, v,
                   g.chunks_per_split, g.sbp, static_cast<double*>(part), ppart, ctx->d_err);
  return cuda_status(cudaGetLastError());
}

// The double-float fast form of a4 (inverted diagonal blocks + chain), unless
// the FP64 solve is asked for.
bool fast_solve(int b, int sb, bool f64solve = false) {
  return !f64solve && b <= CA_FAST_B && sb <= CA_FAST_SB;
}

size_t chain_smem(int b, int sb) {
  if (b <= 16) {  // lookahead chain: ring | Gamma^{-1} | rhs0 | Delta | hand-over | indices
    const size_t ring = b <= 8 ? (size_t)4 * 8 * 256 * 8 : (size_t)3 * 16 * 256 * 8;
    return ring + (size_t)sb * b * 8 + 256 * 8 + 256 * 8 + 64 * 8 + 256 * 4 + 64;
  }
  return (size_t)2 * 32 * 256 * 8 + (size_t)sb * b * 8 + 64 * 8 + (size_t)sb * 12 + 64;
}

// a4: the chain (fast form, from Rs, p and the inverted diagonal blocks
// Ginv) or the general block forward substitution (from R, p).
void launch_solve(ca_ctx* ctx, const double* R, const float2* Rs, const double* pvec,
                  const float2* Ginv, const SolveArgs& sa, bool f64solve) {
  if (fast_solve(sa.b, sa.sb, f64solve)) {
    launch_chain(sa.b, chain_smem(sa.b, sa.sb), ctx->stream, Rs, pvec, Ginv, sa, ctx->d_err);
  } else {
    k_solve<<<1, 256, (size_t)(sa.sb + sa.b * sa.b + sa.b) * sizeof(double), ctx->stream>>>(
        R, pvec, sa, ctx->d_err);
  }
}

// Whether launch_reduce_solve runs a4 as the single reduce + chain launch.
bool uses_reduce_chain(const GramPlan& g, const SolveArgs& sa, bool f64solve) {
  return g.tc && sa.s_cur > 0 && fast_solve(sa.b, sa.sb, f64solve) && sa.b <= 16;
}

// a4 entry: reduce the partials to R, p and invert the diagonal blocks (in
// the reduce launch for b <= 16, by k_factor otherwise), then (s_cur > 0) the
// inner solves.
int launch_reduce_solve(ca_ctx* ctx, const GramPlan& g, const void* part, const double* ppart,
                        double* R, float2* Rs, double* pvec, float2* Ginv, const SolveArgs& sa,
                        bool f64solve = false) {
  const bool fast = sa.s_cur > 0 && fast_solve(sa.b, sa.sb, f64solve);
  const long long entries = (long long)sa.sb * (sa.sb + 1) / 2 + sa.sb;
  const long long passes = (entries + 31) / 32;
  const int G = (int)std::max(1LL, std::min<long long>(passes, 8LL * ctx->num_sms));
  const int ndiag = (fast && sa.b <= 16) ? sa.s_cur : 0;
  if (g.tc && ndiag) {
    // one launch: reducing CTAs (64 entries per pass, + the diagonal
    // inverses) and one more CTA for the chain; at most one CTA per SM
    const int grid =
        (int)std::max<long long>(1, std::min<long long>((entries + 63) / 64 + ndiag,
                                                        ctx->num_sms - 1)) + 1;
    prof_mark(ctx, PC_SOLVE);
    const int e = launch_reduce_chain(grid, chain_smem(sa.b, sa.sb), ctx->stream,
                                      static_cast<const float*>(part), ppart, g.P, g.sbp, R, Rs,
                                      pvec, Ginv, ndiag, sa, ctx->d_err, ctx->d_ticket);
    prof_mark(ctx, PC_SOLVE);
    ctx->prof.kernel_launches += 1;
    return e != 0 ? cuda_fail((cudaError_t)e, __LINE__) : CA_OK;
  }
  prof_mark(ctx, PC_SOLVE);
  launch_reduce(g.tc, G + ndiag, 0, ctx->stream, part, ppart, g.P, g.sbp, R, fast ? Rs : nullptr,
                pvec, ndiag ? Ginv : nullptr, ndiag, sa, ctx->d_err);
  ctx->prof.kernel_launches += 1;
  if (fast && !ndiag) {
    launch_factor(ctx->stream, R, sa, Ginv, ctx->d_err);
    ctx->prof.kernel_launches += 1;
  }
  prof_mark(ctx, PC_SOLVE);
  if (sa.s_cur > 0) {
    prof_mark(ctx, PC_CHAIN);
    launch_solve(ctx, R, Rs, pvec, Ginv, sa, f64solve);
    prof_mark(ctx, PC_CHAIN);
    ctx->prof.kernel_launches += 1;
  }
  return cuda_status(cudaGetLastError());
}

int run_dense(ca_ctx* ctx, const DenseProblem& pb, const ca_opts* o, int* idx_all, char* work,
              size_t work_bytes) {
  const long long K = pb.K;
  const int b = o->b, s = o->s;
  const long long H = o->H;
  const int sbm = (int)(std::min<long long>(s, H) * b);
  Carve cv{work};
  (void)work_bytes;
  const bool f64solve = o->solve == CA_SOLVE_F64;
  GramPlan g = gram_plan(ctx, pb.xfmt, o->prec, sbm, K);
  if (g.tc && pb.panel && g.sbp <= 128 && b <= 16 && fast_solve(b, sbm, f64solve) &&
      ctx->num_sms > 1) {
    // the chain of step k runs on one SM (last CTA of the reduce launch) while
    // the Gram CTAs of step k+1 prepare: leave that SM to it, so that no Gram
    // CTA starts only after the chain
    g.P = (int)std::min<long long>(ctx->num_sms - 1, (K + 31) / 32);
  }
  const int sbp = g.sbp, P = g.P;
  void* part = g.tc ? (void*)cv.take<float>((size_t)P * sbp * sbp)
                    : (void*)cv.take<double>((size_t)P * sbp * sbp);
  double* ppart = cv.take<double>((size_t)P * sbp);
  double* R = cv.take<double>((size_t)sbp * sbp);
  double* pvec = cv.take<double>((size_t)sbp);
  double* delta2[2] = {cv.take<double>((size_t)sbp), cv.take<double>((size_t)sbp)};
  float2* Ginv = cv.take<float2>((size_t)sbp * CA_FAST_B);
  float2* Rs = cv.take<float2>((size_t)sbp * sbp);
  // The deferred update of outer step k (a5) runs inside the Gram launch of
  // step k+1 when the tensor-core path has s*b <= 128; otherwise, after the
  // last step, and before a due recomputation it runs on its own.
  const bool fuse = g.tc && g.sbp <= 128 && pb.panel;
  auto due = [&](long long k) { return o->recompute_every > 0 && (k + 1) % o->recompute_every == 0; };
  // stopping test (Sec. 5.1.5)
  const bool chk = o->check_every > 0;
  ctx->info = ca_info{H, 0, 0.0, 0.0, 0.0, 0.0, -1.0};
  ctx->trace.clear();
  const CheckArgs ck{pb.method, o->stop == CA_STOP_OBJECTIVE, o->lam, pb.A,
                     pb.xfmt == CA_DENSE_F64, pb.panel, pb.lda, pb.N, K, pb.v, pb.v2, nullptr,
                     pb.rq, pb.racc, pb.x, pb.yv, pb.cP, pb.cI, pb.cY};
  auto residual = [&](double* out, long long h_at) {
    return full_check(ctx, ck, h_at, out, &ctx->info.gap, &ctx->info.fval);
  };
  // FP32 X: the deferred updates round their products to FP32, so v drifts
  // from its definition by ~2^-24 of each step's increment; a check first
  // rebuilds v from the definition (a6 with exact products summed in
  // double-float) so that the residual, the gap and f(w) it reports are
  // those of the current iterate.  (FP64 X: the updates are FP64.)
  const bool rebuild_at_check = pb.xfmt == CA_DENSE_F32;
  if (chk) {  // (v was just formed from its definition)
    CA_TRY(residual(&ctx->info.res0, 0));
    ctx->info.res = ctx->info.res0;
  }
  bool pending = false;  // an update (prev_*) not yet applied
  bool after_rc = false;  // the last kernel in the stream is the reduce + chain launch
  const int* prev_idx = nullptr;
  int prev_sb = 0;
  const double* prev_delta = nullptr;
  auto update_alone = [&]() -> int {
    pending = false;
    after_rc = false;
    return launch_update_alone(ctx, pb, prev_idx, prev_sb, prev_delta);
  };

  const long long n_outer = (H + s - 1) / s;
  // Runs of full outer steps between two host decisions (a check, a due
  // recomputation, the short last step) go to one persistent launch
  // (ca_persist.cu) when the configuration fits it: BF16x3 or scaled-FP16
  // Gram on panels, s*b <= 128, b <= 8, the double-float solve, one Gram CTA
  // on every SM but one.
  const long long natoms = (K + 31) / 32;
  bool persist_ok = ctx->persist && g.tc && pb.panel && (g.three == 2 || g.three == 3) &&
                    sbp <= 128 && b <= 8 && fast_solve(b, sbm, f64solve) &&
                    P == ctx->num_sms - 1 && P > s && natoms >= P;
  int na = 0;  // region-A atoms per Gram CTA
  if (persist_ok) {
    // a stage's slice of v2 is read when the stage is issued, up to a
    // load-ring depth ahead: every pass must be longer than the ring so
    // that the previous pass has written the slice by then
    const int ring = persist_load_ring(sbp, g.three);
    const long long tmin = natoms / P;
    if (tmin <= ring) persist_ok = false;
    na = (int)std::min<long long>(tmin, std::llround(ctx->overlap * (double)tmin));
  }
  auto boundary_after = [&](long long j) {
    return due(j) || (chk && (j + 1) % o->check_every == 0 && j + 1 < n_outer);
  };
  for (long long k = 0; k < n_outer; ++k) {
    const int sk = (int)std::min<long long>(s, H - (long long)s * k);
    const int sb = sk * b;
    const int* idx = idx_all + (size_t)s * k * b;
    double* delta = delta2[k & 1];
    if (pending && (!fuse || due(k - 1))) {
      CA_TRY(update_alone());                                   // a5 of step k-1 (clears after_rc)
      if (due(k - 1)) CA_TRY(launch_recompute(ctx, pb, pb.v, pb.y0, pb.c0, pb.c1));  // a6
    }
    long long k1 = k + 1;  // end of the run that starts at k
    if (persist_ok && sk == s)
      while (k1 < n_outer && (long long)s * (k1 + 1) <= H && !boundary_after(k1 - 1)) ++k1;
    bool persisted = false;
    if (persist_ok && sk == s && k1 - k >= 2) {
      PersistArgs pa{};
      pa.A = static_cast<const float*>(pb.A);
      pa.N = pb.N;
      pa.K = K;
      pa.natoms = natoms;
      pa.idx_all = idx_all;
      pa.sb = sb;
      pa.k0 = k;
      pa.npass = (int)(k1 - k);
      pa.na = na;
      pa.prev_idx = pending ? prev_idx : nullptr;
      pa.prev_sb = pending ? prev_sb : 0;
      pa.delta2[0] = delta2[0];
      pa.delta2[1] = delta2[1];
      pa.v2 = pb.v2;
      pa.cU = pb.cU;
      pa.rscale = pb.rscale;
      pa.part = static_cast<float*>(part);
      pa.ppart = ppart;
      pa.R = R;
      pa.Rs = Rs;
      pa.pvec = pvec;
      pa.Ginv = Ginv;
      pa.sa = SolveArgs{nullptr, pb.N, b, s, sb, sbp, pb.cG, pb.cI, pb.cP, pb.cY, pb.x, pb.yv, nullptr};
      pa.cnt = ctx->d_cnt;
      pa.chain_smem = chain_smem(b, sb);
      CA_TRY_CUDA(cudaMemsetAsync(ctx->d_cnt, 0, 3 * sizeof(unsigned), ctx->stream));
      prof_mark(ctx, PC_GRAM);
      const int e = launch_persist(pa, P + 1, sbp, g.three, ctx->d_err, ctx->stream);
      prof_mark(ctx, PC_GRAM);
      if (e == (int)cudaErrorCooperativeLaunchTooLarge || e == (int)cudaErrorInvalidConfiguration) {
        (void)cudaGetLastError();  // not resident at once here: the launches per step instead
        persist_ok = false;
      } else if (e != 0) {
        return cuda_fail((cudaError_t)e, __LINE__);
      } else {
        ctx->prof.kernel_launches += 1;
        persisted = true;
        k = k1 - 1;  // the last step of the run; its update is pending
        after_rc = false;
        pending = true;
        prev_idx = idx_all + (size_t)s * k * b;
        prev_sb = sb;
        prev_delta = delta2[k & 1];
      }
    }
    if (!persisted) {
      // a2 + a3 (and a5 of step k-1 when fused)
      GramUpdate gu{prev_idx, pending ? prev_sb : 0, prev_delta, pb.cU, pb.v2, pb.rscale, after_rc};
      prof_mark(ctx, PC_GRAM);
      if (pending) {
        const int e = launch_gram_tc(static_cast<const float*>(pb.A), pb.lda, pb.N, K, idx, sb,
                                     pb.v2, P, sbp, static_cast<float*>(part), ppart, ctx->d_err,
                                     g.three, ctx->stream, &gu, true);
        if (e != 0) return cuda_fail((cudaError_t)e, __LINE__);
        pending = false;
      } else {
        CA_TRY(launch_gram(ctx, g, pb.xfmt, pb.A, pb.lda, pb.N, K, idx, sb, pb.v, pb.v2, part,
                           ppart, pb.panel, pb.rscale, after_rc));
      }
      prof_mark(ctx, PC_GRAM);
      ctx->prof.kernel_launches += 1;
      // a4 (reduce of the split-K partials, then the s unrolled solves)
      SolveArgs sa{idx, pb.N, b, sk, sb, sbp, pb.cG, pb.cI, pb.cP, pb.cY, pb.x, pb.yv, delta};
      CA_TRY(launch_reduce_solve(ctx, g, part, ppart, R, Rs, pvec, Ginv, sa, f64solve));
      CA_TRY_CUDA(cudaGetLastError());
      after_rc = uses_reduce_chain(g, sa, f64solve);
      pending = true;
      prev_idx = idx;
      prev_sb = sb;
      prev_delta = delta;
    }
    if (chk && (k + 1) % o->check_every == 0 && k + 1 < n_outer) {
      // the deferred update of this step first: the residual needs v current
      CA_TRY(update_alone());
      after_rc = false;  // (also after a recompute and the check's kernels)
      if (due(k) || rebuild_at_check) CA_TRY(launch_recompute(ctx, pb, pb.v, pb.y0, pb.c0, pb.c1));
      CA_TRY(residual(&ctx->info.res, (k + 1) * (long long)s));
      ++ctx->info.checks;
      if (check_says_stop(o, ctx->info)) {
        ctx->info.h_done = (k + 1) * (long long)s;
        return CA_OK;
      }
    }
  }
  bool fresh = false;  // v just rebuilt from its definition
  if (pending) {
    CA_TRY(update_alone());
    if (due(n_outer - 1)) {
      CA_TRY(launch_recompute(ctx, pb, pb.v, pb.y0, pb.c0, pb.c1));
      fresh = true;
    }
  }
  if (chk) {
    if (rebuild_at_check && !fresh) CA_TRY(launch_recompute(ctx, pb, pb.v, pb.y0, pb.c0, pb.c1));
    CA_TRY(residual(&ctx->info.res, H));
    ++ctx->info.checks;
  }
  return CA_OK;
}

size_t dense_work_bytes(ca_ctx* ctx, const ca_opts* o, long long K, int xfmt) {
  const int sbm = (int)(std::min<long long>(o->s, o->H) * o->b);
  const bool tc = (xfmt == CA_DENSE_F32) && tc_prec(o->prec);
  size_t sbp, P, el;
  if (tc) {
    sbp = sbm <= 128 ? 128 : 256;
    P = (size_t)std::min<long long>(ctx->num_sms, (K + 31) / 32);
    el = 4;
  } else {
    sbp = (size_t)(sbm + 63) / 64 * 64;
    P = (size_t)std::max<long long>(1, 2 * ctx->num_sms);  // upper bound of the split count
    const size_t cap = std::max<size_t>(1, (256ull << 20) / (sbp * sbp * 8));
    P = std::min(P, cap);
    el = 8;
  }
  return align256(P * sbp * sbp * el) + align256(P * sbp * 8) + 2 * align256(sbp * sbp * 8) +
         3 * align256(sbp * 8) + align256(sbp * CA_FAST_B * 8) + 4096;
}

size_t panel_bytes(long long N, long long K) { return (size_t)((K + 31) / 32) * (size_t)N * 128; }

// Arena bytes of a dense solve whose vectors are device-resident (host-resident
// inputs add their staging on top): the Gram / solve work area, the split
// copies of v and x, the sampled indices, rho (primal), the panel copy of X
// when the solve repacks it, the scaled-FP16 row multipliers and the
// stopping-test scratch.  method 0: primal (A = X, N = d, K = n); 1: dual
// (A = X^T, N = n, K = d).
size_t dense_base_need(ca_ctx* ctx, const ca_opts* o, int method, int xf, bool pre, long long d,
                       long long n) {
  const bool tc = (xf == CA_DENSE_F32) && tc_prec(o->prec);
  const long long N = method == 0 ? d : n, K = method == 0 ? n : d;
  size_t need = dense_work_bytes(ctx, o, K, xf) + align256((size_t)(K + 31) / 32 * 32 * 8) +
                align256((size_t)N * 8) + align256((size_t)o->H * o->b * 4) + 8 * 256;
  if (method == 0) need += align256((size_t)n * 8);  // rho
  if (tc && !pre) need += align256(panel_bytes(N, K)) + 256;
  if (tc && o->prec == CA_GRAM_FP16_SCALED) need += align256((size_t)N * 4) + 256;
  if (o->check_every > 0) need += align256((size_t)check_rows(o, N, K) * 8) + 512;
  return need;
}

void launch_pack(ca_ctx* ctx, const float* A, long long N, long long K, long long lda, float* out) {
  const long long units = N * ((K + 31) / 32);
  const long long blocks = std::min<long long>((units * 8 + 255) / 256, 16LL * ctx->num_sms);
  prof_mark(ctx, PC_OTHER);
  k_pack_panels<<<(unsigned)std::max(1LL, blocks), 256, 0, ctx->stream>>>(A, N, K, lda, out);
  prof_mark(ctx, PC_OTHER);
  ctx->prof.kernel_launches += 1;
}

// Stage a caller array on the device (copy in when `in`), return the device pointer.
template <typename T>
T* stage(ca_ctx* ctx, Carve& cv, const T* p, size_t count, bool in, bool* staged) {
  if (is_device_ptr(p)) {
    *staged = false;
    return const_cast<T*>(p);
  }
  *staged = true;
  T* d = cv.take<T>(count);
  if (in && count) cudaMemcpyAsync(d, p, count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream);
  return d;
}

int launch_update_alone(ca_ctx* ctx, const DenseProblem& pb, const int* prev_idx, int prev_sb,
                        const double* prev_delta) {
  const size_t usm = align256((size_t)prev_sb * 4) + (size_t)prev_sb * 8;  // sidx | delta
  const unsigned ug = (unsigned)((pb.K + 255) / 256);
  prof_mark(ctx, PC_UPDATE);
  launch_update_dense(pb.xfmt == CA_DENSE_F64, ug, usm, ctx->stream, pb.A, pb.lda, pb.N, pb.K,
                      prev_idx, prev_sb, prev_delta, pb.cU, pb.v, pb.v2, ctx->d_err, pb.panel);
  prof_mark(ctx, PC_UPDATE);
  ctx->prof.kernel_launches += 1;
  return cuda_status(cudaGetLastError());
}

void launch_row_scale_ctx(ca_ctx* ctx, const float* A, long long N, long long K, float* rscale) {
  launch_row_scale(ctx->stream, A, 0, N, K, true, rscale);
  ctx->prof.kernel_launches += 1;
}

}  // namespace caint

using namespace caint;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* ca_status_str(int status) {
  switch (status) {
    case CA_OK: return "CA_OK";
    case CA_ERR_ARG: return "CA_ERR_ARG: invalid argument";
    case CA_ERR_CUDA: return "CA_ERR_CUDA: CUDA runtime error";
    case CA_ERR_NOT_SPD: return "CA_ERR_NOT_SPD: a diagonal block is not positive definite";
    case CA_ERR_NONFINITE: return "CA_ERR_NONFINITE: non-finite value in a Gram block or solve";
    case CA_ERR_TIMEOUT: return "CA_ERR_TIMEOUT: a bounded device wait gave up";
    case CA_ERR_OOM: return "CA_ERR_OOM: scratch exceeds the context budget";
    case CA_ERR_UNSUPPORTED: return "CA_ERR_UNSUPPORTED: outside this build's limits";
    default: return "unknown ca_status";
  }
}

int ca_bcd_init(ca_ctx** out, int device, void* cuda_stream, size_t scratch_bytes_max) {
  if (!out) return CA_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return ndev == 0 ? CA_ERR_CUDA : CA_ERR_ARG;
  }
  CA_TRY_CUDA(cudaSetDevice(device));
  ca_ctx* ctx = new ca_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->scratch_max = scratch_bytes_max;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&ctx->d_err, 256) != cudaSuccess || cudaMallocHost(&ctx->h_err, 128) != cudaSuccess) {
    cudaGetLastError();
    ca_bcd_destroy(ctx);
    return CA_ERR_CUDA;
  }
  ctx->d_ticket = ctx->d_err + 32;
  ctx->d_cnt = ctx->d_err + 48;
  cudaMemset(ctx->d_err, 0, 256);
  if (set_solve_smem_limit(kSolveSmemMax) != 0) {
    cudaGetLastError();
    ca_bcd_destroy(ctx);
    return CA_ERR_CUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    ca_bcd_destroy(ctx);
    return CA_ERR_CUDA;
  }
  *out = ctx;
  return CA_OK;
}

void ca_bcd_destroy(ca_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
  }
  for (cudaEvent_t e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->h_err) cudaFreeHost(ctx->h_err);
  delete ctx;
}

int ca_sample_indices(ca_ctx* ctx, unsigned long long seed, long long h0, long long H, int b,
                      long long N, int* out) {
  t_cur_ctx = ctx;
  if (!ctx || !out || H < 0 || h0 < 0 || b < 1 || N < 1 || b > N || N > 2147483647LL)
    return CA_ERR_ARG;
  if (H == 0) return CA_OK;
  CA_TRY_CUDA(cudaSetDevice(ctx->device));
  const size_t bytes = (size_t)H * b * sizeof(int);
  int* d = out;
  const bool host = !is_device_ptr(out);
  if (host) {
    CA_TRY(ensure_arena(ctx, align256(bytes)));
    d = static_cast<int*>(ctx->arena);
  }
  k_sample<<<(unsigned)((H + 7) / 8), 256, 0, ctx->stream>>>(seed, h0, H, b, N, d);
  CA_TRY_CUDA(cudaGetLastError());
  if (host) CA_TRY_CUDA(cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CA_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
  return CA_OK;
}

int ca_bcd_solve(ca_ctx* ctx, int xfmt, const void* X, long long d, long long n, long long ld,
                 const double* y, const ca_opts* o, double* w, double* z) {
  t_cur_ctx = ctx;
  const bool pre = xfmt == CA_DENSE_F32_PANELS;
  if (!ctx || !X || !y || !w || d < 1 || n < 1 || (!pre && ld < n)) return CA_ERR_ARG;
  ctx->prof.cls.clear();  // marks of an earlier call that failed before finishing
  if (xfmt != CA_DENSE_F64 && xfmt != CA_DENSE_F32 && !pre) return CA_ERR_ARG;
  CA_TRY(check_opts(o, d));
  const int xf = pre ? (int)CA_DENSE_F32 : xfmt;  // element type of X
  const bool tc = (xf == CA_DENSE_F32) && tc_prec(o->prec);
  if (pre && !tc) return CA_ERR_ARG;
  if (tc) {
    if ((!pre && (ld & 3) != 0) || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return CA_ERR_ARG;
    if (std::min<long long>(o->s, o->H) * o->b > gram_tc_max_sb()) return CA_ERR_UNSUPPORTED;
  }
  CA_TRY_CUDA(cudaSetDevice(ctx->device));
  const size_t el = xf == CA_DENSE_F64 ? 8 : 4;
  const bool x_host = !is_device_ptr(X), y_host = !is_device_ptr(y), w_host = !is_device_ptr(w);
  const bool z_host = z && !is_device_ptr(z);
  const size_t xbytes = pre ? panel_bytes(d, n) : (size_t)(d - 1) * ld * el + (size_t)n * el;
  size_t need = dense_base_need(ctx, o, 0, xf, pre, d, n);
  // FP32 X in pinned host memory: the panel repack reads it in place (one
  // pass over the host link instead of a copy followed by a repack)
  const void* x_mapped = (x_host && tc && !pre) ? mapped_host_ptr(X) : nullptr;
  if (x_host && !x_mapped) need += align256(xbytes) + 256;
  const bool f16 = tc && o->prec == CA_GRAM_FP16_SCALED;
  if (y_host) need += align256((size_t)n * 8);
  if (w_host) need += align256((size_t)d * 8);
  if (z_host) need += align256((size_t)n * 8);
  CA_TRY(ensure_arena(ctx, need));
  Carve cv{static_cast<char*>(ctx->arena)};
  bool st;
  const void* Xd = X;
  if (x_mapped) {
    Xd = x_mapped;
  } else if (x_host) {
    void* p = cv.take<char>(xbytes);
    CA_TRY_CUDA(cudaMemcpyAsync(p, X, xbytes, cudaMemcpyHostToDevice, ctx->stream));
    Xd = p;
  }
  bool panel = pre;
  if (tc && !pre) {  // the gather reads 32-column panels (ca_pack_panels layout)
    float* pk = cv.take<float>(panel_bytes(d, n) / 4);
    launch_pack(ctx, static_cast<const float*>(Xd), d, n, ld, pk);
    Xd = pk;
    panel = true;
  }
  float* rsc = nullptr;  // scaled FP16 Gram: per-feature multipliers (one pass over X)
  if (f16) {
    rsc = cv.take<float>((size_t)d);
    launch_row_scale(ctx->stream, static_cast<const float*>(Xd), ld, d, n, panel, rsc);
    ctx->prof.kernel_launches += 1;
  }
  const double* yd = stage(ctx, cv, y, (size_t)n, true, &st);
  double* wd = stage(ctx, cv, w, (size_t)d, true, &st);
  double* zd = z ? stage(ctx, cv, z, (size_t)n, false, &st) : nullptr;
  double* rho = cv.take<double>((size_t)n);
  float2* rho2 = cv.take<float2>((size_t)(n + 31) / 32 * 32);
  float2* w2s = cv.take<float2>((size_t)d);
  int* idx = cv.take<int>((size_t)o->H * o->b);
  double* rq = nullptr;  // stopping test: zero scratch and the accumulators
  double* racc = nullptr;
  if (o->check_every > 0) {
    const long long rows = check_rows(o, d, n);
    rq = cv.take<double>((size_t)rows);
    racc = cv.take<double>(kCheckAcc);
    CA_TRY_CUDA(cudaMemsetAsync(rq, 0, (size_t)rows * 8, ctx->stream));
  }
  char* work = static_cast<char*>(ctx->arena) + align256(cv.off);  // after every carve above
  CA_TRY_CUDA(cudaMemsetAsync(ctx->d_err, 0, 33 * sizeof(unsigned), ctx->stream));

  DenseProblem pb;
  pb.xfmt = xf;
  pb.A = Xd;
  pb.panel = panel;
  pb.method = 0;
  pb.N = d;
  pb.K = n;
  pb.lda = ld;
  pb.v = rho;
  pb.v2 = rho2;
  pb.rscale = rsc;
  pb.rq = rq;
  pb.racc = racc;
  pb.x = wd;
  pb.x2 = w2s;
  pb.yv = nullptr;
  pb.cG = 1.0 / (double)n;
  pb.cI = o->lam;
  pb.cP = 1.0 / (double)n;
  pb.cY = 0.0;
  pb.cU = 1.0;
  pb.y0 = yd;
  pb.c0 = 1.0;
  pb.c1 = -1.0;
  // rho_0 = y - X^T w_0  (z_0 = X^T w_0, Alg. 1-2)
  CA_TRY(launch_recompute(ctx, pb, rho, yd, 1.0, -1.0));
  // a1 for all H blocks at once (counter-based, independent of the iterates)
  prof_mark(ctx, PC_OTHER);
  k_sample<<<(unsigned)((o->H + 7) / 8), 256, 0, ctx->stream>>>(o->seed, o->h0, o->H, o->b, d, idx);
  prof_mark(ctx, PC_OTHER);
  ctx->prof.kernel_launches += 1;
  CA_TRY_CUDA(cudaGetLastError());
  CA_TRY(run_dense(ctx, pb, o, idx, work, ctx->arena_bytes - (size_t)(work - (char*)ctx->arena)));
  if (zd) CA_TRY(launch_recompute(ctx, pb, zd, nullptr, 0.0, 1.0));  // z = X^T w_H
  if (w_host)
    CA_TRY_CUDA(cudaMemcpyAsync(w, wd, (size_t)d * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (z_host)
    CA_TRY_CUDA(cudaMemcpyAsync(z, zd, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  return finish(ctx);
}

int ca_bdcd_solve(ca_ctx* ctx, int xfmt, const void* XT, long long d, long long n, long long ld,
                  const double* y, const ca_opts* o, double* alpha, double* w) {
  t_cur_ctx = ctx;
  if (!ctx || !XT || !y || !alpha || !w || d < 1 || n < 1) return CA_ERR_ARG;
  ctx->prof.cls.clear();  // marks of an earlier call that failed before finishing
  if (xfmt != CA_DENSE_F64 && xfmt != CA_DENSE_F32 && xfmt != CA_CSR_F32 &&
      xfmt != CA_DENSE_F32_PANELS)
    return CA_ERR_ARG;
  CA_TRY(check_opts(o, n));
  CA_TRY_CUDA(cudaSetDevice(ctx->device));
  const double ln = o->lam * (double)n;
  const bool y_host = !is_device_ptr(y), a_host = !is_device_ptr(alpha), w_host = !is_device_ptr(w);
  size_t need_host = 0;  // staging of host-resident vectors
  if (y_host) need_host += align256((size_t)n * 8);
  if (a_host) need_host += align256((size_t)n * 8);
  if (w_host) need_host += align256((size_t)d * 8);
  size_t need = align256((size_t)o->H * o->b * 4) + 8 * 256 + need_host;

  if (xfmt == CA_CSR_F32) {
    const ca_csr* csr = static_cast<const ca_csr*>(XT);
    if (!csr->rowptr || !csr->col || !csr->val) return CA_ERR_ARG;
    const bool r_host = !is_device_ptr(csr->rowptr);
    long long nnz = 0;
    if (r_host) nnz = csr->rowptr[n];
    else CA_TRY_CUDA(cudaMemcpy(&nnz, csr->rowptr + n, sizeof(long long), cudaMemcpyDeviceToHost));
    if (nnz < 0) return CA_ERR_ARG;
    const bool c_host = !is_device_ptr(csr->col), v_host = !is_device_ptr(csr->val);
    if (r_host) need += align256((size_t)(n + 1) * 8);
    if (c_host) need += align256((size_t)nnz * 4);
    if (v_host) need += align256((size_t)nnz * 4);
    const int sbm = (int)(std::min<long long>(o->s, o->H) * o->b);
    // leading dimension of R / Rs: a multiple of 32 (the chain copies 16-byte
    // row pairs of the transposed Rs)
    const size_t sbp = (size_t)(sbm + 31) / 32 * 32;
    need += 5 * align256(sbp * sbp * 8) + 3 * align256(sbp * 8) + 2 * align256(sbp * CA_FAST_B * 8) +
            4096;
    if (o->check_every > 0) need += align256((size_t)check_rows(o, n, d) * 8) + 512;
    // the dense-sparse split of the Gram (s*b >= 32): column counts, the
    // dense map, and Xd (nrows x fd FP32, 64 MB at most)
    constexpr int kSplitMinSB = 32;  // below it the pair kernel is as fast
    const bool split = sbm >= kSplitMinSB && sbm <= 4096;
    // (a multiple of 8: Xd's rows are zero-padded to 16-byte multiples)
    const int fdmax = (int)std::min<long long>(
        CA_CSR_DENSE_MAX, ((64LL << 20) / (4 * std::max(1LL, n))) & ~7LL);
    if (split) need += 2 * align256((size_t)d * 4) + align256((size_t)n * std::max(fdmax, 8) * 4) + 512;
    need += align256((size_t)n * 8);  // row norms
    // where each feature range starts in every row (256 MB at most, else searched)
    const size_t roff_bytes = csr_rangeoff_bytes(n, d);
    const bool use_roff = split && roff_bytes <= ((size_t)256 << 20);
    if (use_roff) need += align256(roff_bytes);
    CA_TRY(ensure_arena(ctx, need));
    Carve cv{static_cast<char*>(ctx->arena)};
    bool st;
    const long long* rp = stage(ctx, cv, csr->rowptr, (size_t)(n + 1), true, &st);
    const int* col = stage(ctx, cv, csr->col, (size_t)nnz, true, &st);
    const float* val = stage(ctx, cv, csr->val, (size_t)nnz, true, &st);
    const double* yd = stage(ctx, cv, y, (size_t)n, true, &st);
    double* ad = stage(ctx, cv, alpha, (size_t)n, true, &st);
    double* wd = stage(ctx, cv, w, (size_t)d, false, &st);
    int* idx = cv.take<int>((size_t)o->H * o->b);
    double* R = cv.take<double>(sbp * sbp);
    double* pvec = cv.take<double>(sbp);
    double* delta = cv.take<double>(sbp);
    float2* Ginv = cv.take<float2>(sbp * CA_FAST_B);
    float2* Rs = cv.take<float2>(sbp * sbp);
    // the Gram (transposed lower triangle), Rs and the diagonal-block
    // inverses, two buffers each: what step k+1 needs of them is formed on
    // the side stream while step k's solves read the other
    double* Gbuf[2] = {cv.take<double>(sbp * sbp), cv.take<double>(sbp * sbp)};
    float2* RsB[2] = {Rs, cv.take<float2>(sbp * sbp)};
    float2* GinvB[2] = {Ginv, cv.take<float2>(sbp * CA_FAST_B)};
    double* rn = cv.take<double>((size_t)n);  // row norms (the Grams' diagonals)
    double* pp1 = cv.take<double>(sbp);       // its projections
    CA_TRY_CUDA(cudaMemsetAsync(ctx->d_err, 0, 33 * sizeof(unsigned), ctx->stream));
    double* rq = nullptr;
    double* racc = nullptr;
    if (o->check_every > 0) {  // stopping test scratch (zero between uses)
      const long long rows = check_rows(o, n, d);
      rq = cv.take<double>((size_t)rows);
      racc = cv.take<double>(kCheckAcc);
      CA_TRY_CUDA(cudaMemsetAsync(rq, 0, (size_t)rows * 8, ctx->stream));
    }
    const ca_csr_dev cdev{rp, col, val};
    const CheckArgs ck{1, o->stop == CA_STOP_OBJECTIVE, o->lam, nullptr, false, false, 0, n, d,
                       wd, nullptr, &cdev, rq, racc, ad, yd, 1.0, 1.0, 1.0};
    auto residual = [&](double* out, long long h_at) {  // X^T w - alpha - y (Sec. 5.1.5)
      return full_check(ctx, ck, h_at, out, &ctx->info.gap, &ctx->info.fval);
    };
    auto recompute = [&]() {  // w = -X alpha/(lambda n)  (eq. "3")
      k_axpby_init<<<(unsigned)((d + 255) / 256), 256, 0, ctx->stream>>>(nullptr, 0.0, d, wd, nullptr);
      k_scatter_csr<<<(unsigned)((n + 7) / 8), 256, 0, ctx->stream>>>(rp, col, val, nullptr, n, d,
                                                                       n, ad, -1.0 / ln, wd,
                                                                       ctx->d_err);
      ctx->prof.kernel_launches += 2;
    };
    recompute();
    k_sample<<<(unsigned)((o->H + 7) / 8), 256, 0, ctx->stream>>>(o->seed, o->h0, o->H, o->b, n, idx);
    CA_TRY_CUDA(cudaGetLastError());
    // heavy features (in at least a quarter of the rows; the heaviest fdmax
    // at most) become the columns of Xd, chosen on the host from the counts
    int fd = 0;
    int* dmap = nullptr;
    float* Xd = nullptr;
    if (split) {
      int* cnt = cv.take<int>((size_t)d);
      dmap = cv.take<int>((size_t)d);
      CA_TRY_CUDA(cudaMemsetAsync(cnt, 0, (size_t)d * 4, ctx->stream));
      launch_csr_prepare(ctx->stream, ctx->num_sms, cdev, n, d, nnz, cnt, nullptr, 0, nullptr, false);
      std::vector<int> hc((size_t)d);
      CA_TRY_CUDA(cudaMemcpyAsync(hc.data(), cnt, (size_t)d * 4, cudaMemcpyDeviceToHost, ctx->stream));
      CA_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
      const long long heavy = (n + 3) / 4;
      std::vector<int> cand;
      for (long long f = 0; f < d; ++f)
        if (hc[(size_t)f] >= heavy) cand.push_back((int)f);
      if ((int)cand.size() > fdmax) {
        std::stable_sort(cand.begin(), cand.end(), [&](int x, int y2) { return hc[x] > hc[y2]; });
        cand.resize((size_t)fdmax);
        std::sort(cand.begin(), cand.end());
      }
      std::vector<int> hm((size_t)d, -1);
      for (size_t j = 0; j < cand.size(); ++j) hm[(size_t)cand[j]] = (int)j;
      fd = ((int)cand.size() + 7) & ~7;  // row length of Xd; the padding stays zero
      CA_TRY_CUDA(cudaMemcpy(dmap, hm.data(), (size_t)d * 4, cudaMemcpyHostToDevice));
      Xd = cv.take<float>((size_t)n * std::max(fd, 8));
      if (fd > 0) {
        CA_TRY_CUDA(cudaMemsetAsync(Xd, 0, (size_t)n * fd * 4, ctx->stream));
        launch_csr_prepare(ctx->stream, ctx->num_sms, cdev, n, d, nnz, nullptr, dmap, fd, Xd, true);
      }
      ctx->prof.kernel_launches += fd > 0 ? 2 : 1;
    }
    int* roff = nullptr;
    if (use_roff) {
      roff = cv.take<int>(roff_bytes / sizeof(int));
      launch_csr_rangeoff(ctx->stream, cdev, n, d, roff);
      ctx->prof.kernel_launches += 1;
    }
    const int b = o->b, s = o->s;
    const long long n_outer = (o->H + s - 1) / s;
    ctx->info = ca_info{o->H, 0, 0.0, 0.0, 0.0, 0.0, -1.0};
    ctx->trace.clear();
    if (o->check_every > 0) {
      CA_TRY(residual(&ctx->info.res0, 0));
      ctx->info.res = ctx->info.res0;
    }
    // s*b <= 4096: the strict lower triangle of each step's Gram (the split,
    // or one warp per pair) has no input that the solves change, so it runs
    // on the side stream one step ahead; events: ev[0] the start and the
    // join, ev[1 + k%2] buffer k%2 formed, ev[3 + k%2] buffer k%2 read
    const bool two = sbm <= 4096;
    if (two && !ctx->side) {
      for (cudaEvent_t& e : ctx->ev)
        if (!e) CA_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      CA_TRY_CUDA(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
    }
    struct SideJoin {  // every exit: the main stream waits for the side stream's work
      ca_ctx* c;
      bool on;
      void operator()() {
        if (!on) return;
        on = false;
        cudaEventRecord(c->ev[0], c->side);
        cudaStreamWaitEvent(c->stream, c->ev[0], 0);
      }
      ~SideJoin() { (*this)(); }
    } join{ctx, false};
    // the fast a4 (b <= 16) with s*b >= 128: the diagonal blocks' inverses
    // and Rs come from the side stream too, and the library stream runs the
    // projections, the chain and the scatter (below 128 rows the extra
    // launch on the side stream costs more than the reduction it moves)
    constexpr int kPrepMinSB = 128;
    const bool f64solve = o->solve == CA_SOLVE_F64;
    auto fast_step = [&](int sbk) {
      return two && fast_solve(b, sbk, f64solve) && b <= 16 && sbk >= kPrepMinSB;
    };
    auto step_args = [&](long long kk) {
      const int skk = (int)std::min<long long>(s, o->H - (long long)s * kk);
      return SolveArgs{idx + (size_t)s * kk * b, n, b, skk, skk * b, (int)sbp, 1.0 / ln, 1.0, 1.0,
                       1.0, ad, yd, delta};
    };
    auto offdiag = [&](long long kk) {
      const SolveArgs sk_args = step_args(kk);
      const int sbk = sk_args.sb;
      const bool sp = split && sbk >= kSplitMinSB;
      launch_csr_offdiag(ctx->side, cdev, sk_args.idx, n, d, sbk, (int)sbp, Gbuf[kk & 1], dmap, Xd,
                         fd, sp, roff);
      ctx->prof.kernel_launches += sbk <= 1 ? 0 : (sp ? 2 : 1);
      if (fast_step(sbk)) {
        launch_csr_prep(ctx->side, ctx->num_sms, rn, n, Gbuf[kk & 1], sk_args, RsB[kk & 1],
                        GinvB[kk & 1], ctx->d_err);
        ctx->prof.kernel_launches += 1;
      }
    };
    if (fast_step(sbm)) {  // before the side stream starts
      launch_csr_rownorm(ctx->stream, cdev, n, rn);
      ctx->prof.kernel_launches += 1;
    }
    if (two && n_outer > 0) {
      CA_TRY_CUDA(cudaEventRecord(ctx->ev[0], ctx->stream));
      CA_TRY_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev[0], 0));
      join.on = true;
      offdiag(0);
      CA_TRY_CUDA(cudaEventRecord(ctx->ev[1], ctx->side));
    }
    for (long long k = 0; k < n_outer; ++k) {
      const int sk = (int)std::min<long long>(s, o->H - (long long)s * k);
      const int sb = sk * b;
      const int* ik = idx + (size_t)s * k * b;
      double* Gt = Gbuf[k & 1];
      // a2+a3: the projections here (with the diagonal when s*b < 128); the
      // rest of the Gram comes from the side stream (all of it, by the row
      // hash tables, when s*b > 4096)
      const bool fk = fast_step(sb);
      prof_mark(ctx, PC_GRAM);
      if (fk) {
        launch_csr_proj(ctx->stream, cdev, ik, n, d, sb, wd, pp1, ctx->d_err);
        ctx->prof.kernel_launches += 1;
      } else if (two) {
        launch_csr_rows(ctx->stream, cdev, ik, n, d, sb, (int)sbp, wd, Gt, pp1, ctx->d_err);
        ctx->prof.kernel_launches += 1;
      } else {
        launch_csr_gram(ctx->stream, ctx->num_sms, cdev, ik, n, d, sb, (int)sbp, wd, Gt, pp1,
                        ctx->d_err);
        ctx->prof.kernel_launches += sb > 1 ? 2 : 1;
      }
      prof_mark(ctx, PC_GRAM);
      if (two) {
        if (k + 1 < n_outer) {  // buffer (k+1)%2 was last read by the solves of step k-1
          if (k >= 1) CA_TRY_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev[3 + ((k + 1) & 1)], 0));
          offdiag(k + 1);
          CA_TRY_CUDA(cudaEventRecord(ctx->ev[1 + ((k + 1) & 1)], ctx->side));
        }
        CA_TRY_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev[1 + (k & 1)], 0));
      }
      // a4: with b <= 16 the chain alone (its other inputs are ready), or
      // the Gram through the dense path's reduction as its one FP64
      // partial: reduce + diagonal inverses + chain in one launch, else the
      // general form
      const SolveArgs sa = step_args(k);
      if (fk) {
        prof_mark(ctx, PC_SOLVE);
        launch_chain(b, chain_smem(b, sb), ctx->stream, RsB[k & 1], pp1, GinvB[k & 1], sa,
                     ctx->d_err);
        prof_mark(ctx, PC_SOLVE);
        ctx->prof.kernel_launches += 1;
      } else if (fast_solve(b, sb, f64solve) && b <= 16) {
        const long long entries = (long long)sb * (sb + 1) / 2 + sb;
        const int grid = (int)std::max<long long>(
                             1, std::min<long long>((entries + 63) / 64 + sk, ctx->num_sms - 1)) + 1;
        prof_mark(ctx, PC_SOLVE);
        const int e = launch_reduce_chain_f64(grid, chain_smem(b, sb), ctx->stream, Gt, pp1,
                                              (int)sbp, R, RsB[k & 1], pvec, GinvB[k & 1], sk, sa,
                                              ctx->d_err, ctx->d_ticket);
        prof_mark(ctx, PC_SOLVE);
        ctx->prof.kernel_launches += 1;
        if (e != 0) return cuda_fail((cudaError_t)e, __LINE__);
      } else {
        GramPlan g{};
        g.tc = false;
        g.sbp = (int)sbp;
        g.P = 1;
        // (Rs and Ginv of this step's parity: the side stream may be
        // writing the other pair for the next step)
        CA_TRY(launch_reduce_solve(ctx, g, Gt, pp1, R, RsB[k & 1], pvec, GinvB[k & 1], sa,
                                   f64solve));
      }
      if (two) CA_TRY_CUDA(cudaEventRecord(ctx->ev[3 + (k & 1)], ctx->stream));
      // a5: w -= Y Delta/(lambda n)
      launch_scatter_csr(ctx->stream, cdev, ik, n, d, sb, delta, -1.0 / ln, wd, ctx->d_err);
      ctx->prof.kernel_launches += 1;
      CA_TRY_CUDA(cudaGetLastError());
      if (o->recompute_every > 0 && (k + 1) % o->recompute_every == 0) recompute();
      if (o->check_every > 0 && ((k + 1) % o->check_every == 0 || k + 1 == n_outer)) {
        CA_TRY(residual(&ctx->info.res, std::min<long long>((k + 1) * (long long)s, o->H)));
        ++ctx->info.checks;
        if (k + 1 < n_outer && check_says_stop(o, ctx->info)) {
          ctx->info.h_done = (k + 1) * (long long)s;
          break;
        }
      }
    }
    join();
    if (a_host)
      CA_TRY_CUDA(cudaMemcpyAsync(alpha, ad, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (w_host) CA_TRY_CUDA(cudaMemcpyAsync(w, wd, (size_t)d * 8, cudaMemcpyDeviceToHost, ctx->stream));
    return finish(ctx);
  }

  // dense dual: XT is n x d row-major (row i = sample i), or its panels
  const bool pre = xfmt == CA_DENSE_F32_PANELS;
  if (!pre && ld < d) return CA_ERR_ARG;
  const int xf = pre ? (int)CA_DENSE_F32 : xfmt;
  const bool tc = (xf == CA_DENSE_F32) && tc_prec(o->prec);
  if (pre && !tc) return CA_ERR_ARG;
  if (tc) {
    if ((!pre && (ld & 3) != 0) || (reinterpret_cast<uintptr_t>(XT) & 15) != 0) return CA_ERR_ARG;
    if (std::min<long long>(o->s, o->H) * o->b > gram_tc_max_sb()) return CA_ERR_UNSUPPORTED;
  }
  const size_t el = xf == CA_DENSE_F64 ? 8 : 4;
  const bool x_host = !is_device_ptr(XT);
  const size_t xbytes = pre ? panel_bytes(n, d) : (size_t)(n - 1) * ld * el + (size_t)d * el;
  need = need_host + dense_base_need(ctx, o, 1, xf, pre, d, n);
  const void* x_mapped = (x_host && tc && !pre) ? mapped_host_ptr(XT) : nullptr;
  if (x_host && !x_mapped) need += align256(xbytes) + 256;
  const bool f16 = tc && o->prec == CA_GRAM_FP16_SCALED;
  CA_TRY(ensure_arena(ctx, need));
  Carve cv{static_cast<char*>(ctx->arena)};
  bool st;
  const void* Xd = XT;
  if (x_mapped) {
    Xd = x_mapped;
  } else if (x_host) {
    void* p = cv.take<char>(xbytes);
    CA_TRY_CUDA(cudaMemcpyAsync(p, XT, xbytes, cudaMemcpyHostToDevice, ctx->stream));
    Xd = p;
  }
  bool panel = pre;
  if (tc && !pre) {  // the gather reads 32-column panels (ca_pack_panels layout)
    float* pk = cv.take<float>(panel_bytes(n, d) / 4);
    launch_pack(ctx, static_cast<const float*>(Xd), n, d, ld, pk);
    Xd = pk;
    panel = true;
  }
  float* rsc = nullptr;  // scaled FP16 Gram: per-sample multipliers (one pass over X)
  if (f16) {
    rsc = cv.take<float>((size_t)n);
    launch_row_scale(ctx->stream, static_cast<const float*>(Xd), ld, n, d, panel, rsc);
    ctx->prof.kernel_launches += 1;
  }
  const double* yd = stage(ctx, cv, y, (size_t)n, true, &st);
  double* ad = stage(ctx, cv, alpha, (size_t)n, true, &st);
  double* wd = stage(ctx, cv, w, (size_t)d, false, &st);
  float2* w2 = cv.take<float2>((size_t)(d + 31) / 32 * 32);
  float2* a2s = cv.take<float2>((size_t)n);
  int* idx = cv.take<int>((size_t)o->H * o->b);
  double* rq = nullptr;  // stopping test: zero scratch and the accumulators
  double* racc = nullptr;
  if (o->check_every > 0) {
    const long long rows = check_rows(o, n, d);
    rq = cv.take<double>((size_t)rows);
    racc = cv.take<double>(kCheckAcc);
    CA_TRY_CUDA(cudaMemsetAsync(rq, 0, (size_t)rows * 8, ctx->stream));
  }
  char* work = static_cast<char*>(ctx->arena) + align256(cv.off);  // after every carve above
  CA_TRY_CUDA(cudaMemsetAsync(ctx->d_err, 0, 33 * sizeof(unsigned), ctx->stream));
  DenseProblem pb;
  pb.xfmt = xf;
  pb.A = Xd;
  pb.panel = panel;
  pb.method = 1;
  pb.N = n;
  pb.K = d;
  pb.lda = ld;
  pb.v = wd;
  pb.v2 = w2;
  pb.rscale = rsc;
  pb.rq = rq;
  pb.racc = racc;
  pb.x = ad;
  pb.x2 = a2s;
  pb.yv = yd;
  pb.cG = 1.0 / ln;
  pb.cI = 1.0;
  pb.cP = 1.0;
  pb.cY = 1.0;
  pb.cU = 1.0 / ln;
  pb.y0 = nullptr;
  pb.c0 = 0.0;
  pb.c1 = -1.0 / ln;
  CA_TRY(launch_recompute(ctx, pb, wd, nullptr, 0.0, -1.0 / ln));  // w_0 = -X alpha_0/(lambda n)
  k_sample<<<(unsigned)((o->H + 7) / 8), 256, 0, ctx->stream>>>(o->seed, o->h0, o->H, o->b, n, idx);
  CA_TRY_CUDA(cudaGetLastError());
  CA_TRY(run_dense(ctx, pb, o, idx, work, ctx->arena_bytes - (size_t)(work - (char*)ctx->arena)));
  if (a_host)
    CA_TRY_CUDA(cudaMemcpyAsync(alpha, ad, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (w_host) CA_TRY_CUDA(cudaMemcpyAsync(w, wd, (size_t)d * 8, cudaMemcpyDeviceToHost, ctx->stream));
  return finish(ctx);
}

// Profiling of the Gram launches (CUDA events on the context's stream around
// every a2+a3 launch of the following solves).
int ca_pack_panels(ca_ctx* ctx, const float* A, long long N, long long K, long long ld, float* out) {
  t_cur_ctx = ctx;
  if (!ctx || !A || !out || N < 1 || K < 1 || ld < K || (ld & 3) != 0 ||
      (reinterpret_cast<uintptr_t>(A) & 15) != 0 || (reinterpret_cast<uintptr_t>(out) & 15) != 0)
    return CA_ERR_ARG;
  if (!is_device_ptr(A) || !is_device_ptr(out)) return CA_ERR_ARG;
  CA_TRY_CUDA(cudaSetDevice(ctx->device));
  launch_pack(ctx, A, N, K, ld, out);
  return cuda_status(cudaGetLastError());
}

const char* ca_last_error(ca_ctx* ctx) { return ctx ? ctx->last_error : "no context"; }

int ca_set_tuning(ca_ctx* ctx, int key, double value) {
  if (!ctx) return CA_ERR_ARG;
  if (key == CA_TUNE_PERSISTENT) {
    if (value != 0.0 && value != 1.0) return CA_ERR_ARG;
    ctx->persist = value != 0.0;
    return CA_OK;
  }
  if (key == CA_TUNE_OVERLAP) {
    if (!(value >= 0.0 && value <= 1.0)) return CA_ERR_ARG;
    ctx->overlap = value;
    return CA_OK;
  }
  return CA_ERR_ARG;
}

int ca_profile_enable(ca_ctx* ctx, int on) {
  if (!ctx) return CA_ERR_ARG;
  std::vector<cudaEvent_t> pool;
  pool.swap(ctx->prof.pool);  // keep the events across resets
  ctx->prof = Profile();
  ctx->prof.pool.swap(pool);
  ctx->prof.on = on != 0;
  return CA_OK;
}

int ca_profile_read(ca_ctx* ctx, double* ms, long long* launches, long long* kernel_launches) {
  if (!ctx) return CA_ERR_ARG;
  for (int c = 0; c < PC_N; ++c) {
    if (ms) ms[c] = ctx->prof.ms[c];
    if (launches) launches[c] = ctx->prof.launches[c];
  }
  if (kernel_launches) *kernel_launches = ctx->prof.kernel_launches;
  return CA_OK;
}

int ca_gram_project(ca_ctx* ctx, int xfmt, int prec, const void* A, long long N, long long K,
                    long long ld, const int* idx, int sb, const double* v, double* G, double* p) {
  t_cur_ctx = ctx;
  if (!ctx || !A || !idx || !v || !G || !p || N < 1 || K < 1 || ld < K || sb < 1 ||
      sb > kMaxSB)
    return CA_ERR_ARG;
  if (xfmt != CA_DENSE_F64 && xfmt != CA_DENSE_F32) return CA_ERR_ARG;
  if (prec < CA_GRAM_F64 || prec > CA_GRAM_FP16_SCALED) return CA_ERR_ARG;
  const bool tc = (xfmt == CA_DENSE_F32) && tc_prec(prec);
  if (tc) {
    if ((ld & 3) != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return CA_ERR_ARG;
    if (sb > gram_tc_max_sb()) return CA_ERR_UNSUPPORTED;
  }
  for (const void* q : {(const void*)A, (const void*)idx, (const void*)v, (const void*)G,
                        (const void*)p})
    if (!is_device_ptr(q)) return CA_ERR_ARG;
  CA_TRY_CUDA(cudaSetDevice(ctx->device));
  const GramPlan g = gram_plan(ctx, xfmt, prec, sb, K);
  const size_t el = g.tc ? 4 : 8;
  const long long Kp = (K + 31) / 32 * 32;
  const size_t need = align256((size_t)g.P * g.sbp * g.sbp * el) + align256((size_t)g.P * g.sbp * 8) +
                      align256((size_t)g.sbp * g.sbp * 8) + align256((size_t)g.sbp * 8) +
                      align256((size_t)Kp * 8) + align256((size_t)N * 4) + 1024;
  CA_TRY(ensure_arena(ctx, need));
  Carve cv{static_cast<char*>(ctx->arena)};
  const bool f16 = g.tc && prec == CA_GRAM_FP16_SCALED;
  float* rsc = f16 ? cv.take<float>((size_t)N) : nullptr;  // per-row FP16 multipliers
  void* part = g.tc ? (void*)cv.take<float>((size_t)g.P * g.sbp * g.sbp)
                    : (void*)cv.take<double>((size_t)g.P * g.sbp * g.sbp);
  double* ppart = cv.take<double>((size_t)g.P * g.sbp);
  double* R = cv.take<double>((size_t)g.sbp * g.sbp);
  float2* v2 = cv.take<float2>((size_t)Kp);
  CA_TRY_CUDA(cudaMemsetAsync(ctx->d_err, 0, 33 * sizeof(unsigned), ctx->stream));
  k_split<<<(unsigned)((Kp + 255) / 256), 256, 0, ctx->stream>>>(v, K, Kp, v2);
  if (f16) launch_row_scale(ctx->stream, static_cast<const float*>(A), ld, N, K, false, rsc);
  CA_TRY(launch_gram(ctx, g, xfmt, A, ld, N, K, idx, sb, v, v2, part, ppart, false, rsc));
  SolveArgs sa{idx, N, 1, 0, sb, g.sbp, 0.0, 0.0, 0.0, 0.0, nullptr, nullptr, nullptr};
  CA_TRY(launch_reduce_solve(ctx, g, part, ppart, R, nullptr, p, nullptr, sa));
  k_symmetrize<<<(unsigned)(((long long)sb * sb + 255) / 256), 256, 0, ctx->stream>>>(R, g.sbp, sb, G);
  CA_TRY_CUDA(cudaGetLastError());
  return finish(ctx);
}

int ca_solve_scratch_bytes(ca_ctx* ctx, int method, int xfmt, long long d, long long n,
                           const ca_opts* o, size_t* bytes) {
  t_cur_ctx = ctx;
  if (!ctx || !bytes || (method != 0 && method != 1) || d < 1 || n < 1) return CA_ERR_ARG;
  if (xfmt != CA_DENSE_F64 && xfmt != CA_DENSE_F32 && xfmt != CA_DENSE_F32_PANELS) return CA_ERR_ARG;
  CA_TRY(check_opts(o, method == 0 ? d : n));
  const bool pre = xfmt == CA_DENSE_F32_PANELS;
  const int xf = pre ? (int)CA_DENSE_F32 : xfmt;
  *bytes = dense_base_need(ctx, o, method, xf, pre, d, n);
  return CA_OK;
}

int ca_bcd_release_scratch(ca_ctx* ctx) {
  t_cur_ctx = ctx;
  if (!ctx) return CA_ERR_ARG;
  CA_TRY_CUDA(cudaSetDevice(ctx->device));
  if (ctx->arena) {
    CA_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    CA_TRY_CUDA(cudaFree(ctx->arena));
    ctx->arena = nullptr;
    ctx->arena_bytes = 0;
  }
  return CA_OK;
}

int ca_solve_info(const ca_ctx* ctx, ca_info* out) {
  if (!ctx || !out) return CA_ERR_ARG;
  *out = ctx->info;
  return CA_OK;
}

int ca_solve_trace(const ca_ctx* ctx, ca_check* out, int max, int* count) {
  if (!ctx || !count || max < 0 || (max > 0 && !out)) return CA_ERR_ARG;
  const int n = (int)ctx->trace.size();
  for (int i = 0; i < std::min(n, max); ++i) out[i] = ctx->trace[(size_t)i];
  *count = n;
  return CA_OK;
}

int ca_selftest_wait_timeout(ca_ctx* ctx, long long limit_ns) {
  t_cur_ctx = ctx;
  if (!ctx || limit_ns < 1 || limit_ns > 1000000000LL) return CA_ERR_ARG;
  CA_TRY_CUDA(cudaSetDevice(ctx->device));
  CA_TRY_CUDA(cudaMemsetAsync(ctx->d_err, 0, 33 * sizeof(unsigned), ctx->stream));
  k_selftest_wait<<<1, 32, 0, ctx->stream>>>((unsigned long long)limit_ns, ctx->d_err);
  CA_TRY_CUDA(cudaGetLastError());
  return finish(ctx);
}

}  // extern "C"
