// ca_internal.h -- the library's internal context and the host helpers that
// the entry points of ca_api.cu and the batched solves of ca_batch.cu share
// (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "ca_bcd.h"

struct ca_csr_dev;

namespace caint {

constexpr int kMaxB = 128;          // b x b block held in shared memory by the solve
constexpr int kMaxSB = 1024;        // s*b right-hand sides held in shared memory
constexpr int kSolveSmemMax = 220 * 1024;

// Kernel classes timed by the profiling hooks.
enum { PC_GRAM = 0, PC_SOLVE = 1, PC_UPDATE = 2, PC_OTHER = 3, PC_CHAIN = 4, PC_N = 5 };

struct Profile {
  bool on = false;
  std::vector<cudaEvent_t> pool;  // events, created once and reused
  std::vector<int> cls;           // class of pool[i] for the marks of this call: start / stop pairs
  double ms[PC_N] = {0, 0, 0, 0, 0};
  long long launches[PC_N] = {0, 0, 0, 0, 0};
  long long kernel_launches = 0;
};

}  // namespace caint

struct ca_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  // the sparse dual's second stream (the next step's off-diagonal Gram, and
  // for s*b >= 128 its diagonal-block inverses and Rs, run on it while the
  // current step's solves run) and its events; made on first use
  cudaStream_t side = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t scratch_max = 0;
  int num_sms = 0;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  unsigned* d_err = nullptr;     // device error word
  unsigned* d_ticket = nullptr;  // count of the reducing CTAs of the reduce/solve kernel
                                 // (d_err + 32; both cleared where a call starts)
  unsigned* d_cnt = nullptr;     // 3 counts of the persistent solve (d_err + 48; cleared
                                 // before each persistent launch); d_err + 56: whether
                                 // the x of a recomputation has a nonzero entry
  unsigned* h_err = nullptr;     // pinned copy (128 bytes: error word; check sums at +32)
  // tuning (ca_set_tuning): persistent launches for runs of outer steps, and
  // the share of a Gram CTA's atoms streamed before the previous step's
  // solve is known
  bool persist = true;
  double overlap = 0.4;
  caint::Profile prof;
  ca_info info{};                // outcome of the last solve
  std::vector<ca_check> trace;   // its checks of the stopping test
  char last_error[256] = {0};    // text of the last failing CUDA call
};

namespace caint {

struct Carve {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int cuda_fail(cudaError_t e, int line);
int cuda_status_at(cudaError_t e, int line);
bool is_device_ptr(const void* p);
int ensure_arena(ca_ctx* ctx, size_t bytes);
int finish(ca_ctx* ctx);
void prof_mark(ca_ctx* ctx, int cls);
int check_opts(const ca_opts* o, long long N);
bool tc_prec(int prec);
size_t chain_smem(int b, int sb);
size_t panel_bytes(long long N, long long K);
void launch_pack(ca_ctx* ctx, const float* A, long long N, long long K, long long lda, float* out);
void launch_row_scale_ctx(ca_ctx* ctx, const float* A, long long N, long long K, float* rscale);

// The dense outer-step loop shared by both methods.
struct DenseProblem {
  int xfmt;                 // CA_DENSE_F64 / CA_DENSE_F32
  const void* A;            // N x K row-major, leading dim lda (device), or panels
  bool panel = false;       // FP32 A stored as 32-column panels [K/32][N][32]
  long long N, K, lda;
  double* v;                // K: projection vector (rho or w), device
  float2* v2;               // its (hi, lo) FP32 split, zero-padded to a multiple of 32
  const float* rscale = nullptr;  // scaled FP16 Gram: per-row multipliers of A (N)
  double* x;                // N: variable updated by the solves (w or alpha), device
  float2* x2;               // N: scratch for the (hi, lo) FP32 split of x (recompute)
  const double* yv;         // dual: y (device), primal: nullptr
  double cG, cI, cP, cY, cU;
  // recompute of v: v = c0 * y0 + c1 * sum_r A[r] x[r]
  const double* y0;
  double c0, c1;
  int method = 0;           // 0: primal (A = X), 1: dual (A = X^T)
  // stopping test: check_rows(o, N, K) doubles of scratch (zero between uses)
  // and kCheckAcc accumulators
  double* rq = nullptr;
  double* racc = nullptr;
};

int launch_recompute(ca_ctx* ctx, const DenseProblem& pb, double* vout, const double* y0,
                     double c0, double c1);

// Stopping test (Sec. 5.1.5): one check forms ||r|| of the current iterate,
// the duality gap it gives and (objective rule) f(w); it waits for the GPU.
constexpr int kCheckAcc = 4;  // ||r||^2, then the sums of squares behind f(w)

// Rows of the check's zero scratch: the residual's N row sums; the objective
// rule also runs the sums of squares over the K entries of v through it.
inline long long check_rows(const ca_opts* o, long long N, long long K) {
  return o->stop == CA_STOP_OBJECTIVE ? (N > K ? N : K) : N;
}

struct CheckArgs {
  int method;
  bool objective;
  double lam;
  const void* A;  // dense A (nullptr with csr)
  bool f64, panel;
  long long lda, N, K;
  const double* v;
  const float2* v2;
  const ca_csr_dev* csr;
  double* rq;     // check_rows zeros
  double* racc;   // kCheckAcc doubles
  const double* x;
  const double* yv;
  double cP, cI, cY;
};

int full_check(ca_ctx* ctx, const CheckArgs& c, long long h_at, double* res, double* gap,
               double* fval);
bool check_says_stop(const ca_opts* o, const ca_info& in);
// a5 alone for the sb rows prev_idx with their Delta (FP32 panels or FP64 X)
int launch_update_alone(ca_ctx* ctx, const DenseProblem& pb, const int* prev_idx, int prev_sb,
                        const double* prev_delta);

extern thread_local ca_ctx* t_cur_ctx;  // context of the running entry point

}  // namespace caint

#define cuda_status(expr) caint::cuda_status_at((expr), __LINE__)

#define CA_TRY_CUDA(call)                                         \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return caint::cuda_fail(e_, __LINE__); \
  } while (0)

#define CA_TRY(call)            \
  do {                          \
    int s_ = (call);            \
    if (s_ != CA_OK) return s_; \
  } while (0)
