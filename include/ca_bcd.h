/*
 * ca_bcd.h -- C ABI of the GB300 (sm_103a) CA-BCD / CA-BDCD library.
 *
 * The library solves the ridge-regression problem of Sec. 2.2 of
 * Devarakonda, Fountoulakis, Demmel and Mahoney, "Avoiding communication in
 * primal and dual block coordinate descent methods" (arXiv 1612.04003):
 *
 *     argmin_w  lambda/2 ||w||^2 + 1/(2n) ||X^T w - y||^2          (eq. "primal")
 *
 * with X in R^{d x n} (rows = features, columns = samples), either by the
 * primal s-step method CA-BCD (Algorithm 2; Algorithm 1 when s = 1) or by the
 * dual s-step method CA-BDCD (Algorithm 4; Algorithm 3 when s = 1) on
 *
 *     argmin_alpha  lambda/2 ||X alpha/(lambda n)||^2 + 1/(2n) ||alpha + y||^2  (eq. "6")
 *
 * with w = -X alpha/(lambda n) (eq. "3").
 *
 * One outer step of either method (s inner block updates) is:
 *   a1  draw the s blocks of b indices (Alg. 2/4, inner sampling loop);
 *   a2  gather the s*b sampled rows (primal) / columns (dual) of X into Y;
 *   a3  form the Gram matrix and the projection of Y on the residual (primal)
 *       or on w (dual) in one pass over Y (Alg. 2/4, "compute the Gram matrix");
 *   a4  run the s unrolled b x b solves (eq. "recur" / its dual analogue);
 *   a5  apply the deferred vector update (Sec. 3.1 / 3.2, the s-step updates);
 *   a6  every `recompute_every` outer steps, rebuild the auxiliary vector from
 *       its definition (z = X^T w, Sec. 3.1; w = -X alpha/(lambda n), eq. "3").
 *
 * Conventions for every entry point:
 *   - Status: CA_OK (0) or a negative ca_status; nothing is thrown across the
 *     ABI.  ca_status_str() names a status.
 *   - Pointers: all arrays are caller-owned.  Array arguments of the solve
 *     calls may be device memory (used in place) or host memory (pinned or
 *     pageable; staged through device buffers the context owns, with the
 *     copies on the context's stream).  The library never frees caller memory.
 *   - Streams: work is issued on the stream given to ca_bcd_init.  A solve
 *     returns after its last kernel and copies finished (it synchronises the
 *     stream to read the device error word).
 *   - Sampling: block h (0-based global inner-iteration index, h0 .. h0+H-1)
 *     draws b distinct indices of [0, N) (N = d primal, n dual) by Floyd's
 *     algorithm fed by Philox4x64-10 with key (seed, 0) and counter
 *     (h, m/4, 0, 0), word m%4 for draw m, mapped to [0, J] as
 *     floor(u*(J+1)/2^64).  The same (seed, h) draws the same block for every
 *     s, so CA-BCD reproduces the s = 1 iterates in exact arithmetic (Sec. 3).
 */
#ifndef CA_BCD_H
#define CA_BCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
  CA_OK = 0,
  CA_ERR_ARG = -1,        /* invalid argument (sizes, b > N, lambda <= 0, ...) */
  CA_ERR_CUDA = -2,       /* a CUDA runtime call failed                        */
  CA_ERR_NOT_SPD = -3,    /* a b x b diagonal block had a non-positive pivot   */
  CA_ERR_NONFINITE = -4,  /* a non-finite value appeared in a Gram or solve    */
  CA_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up                */
  CA_ERR_OOM = -6,        /* scratch would exceed the context's budget         */
  CA_ERR_UNSUPPORTED = -7 /* valid input outside what this build implements    */
} ca_status;

/* Storage of X. */
typedef enum {
  CA_DENSE_F64 = 0, /* dense, FP64                                              */
  CA_DENSE_F32 = 1, /* dense, FP32                                              */
  CA_CSR_F32 = 2,   /* dual only: CSR of X^T (row i = sample i), FP32 values    */
  CA_DENSE_F32_PANELS = 3 /* dense FP32 in 32-column panels (ca_pack_panels);
                           * tcgen05 Gram modes only                          */
} ca_xfmt;

/* Arithmetic of the Gram matrix (step a3).  The vectors at the boundary
 * (y, w, alpha, z) are FP64 in every mode; on FP64 X every vector pass is
 * FP64.  On FP32 X: the projection (a3) and the deferred update (a5) form
 * FP32 products of X with the FP32 (hi, lo) split of the FP64 vector, summed
 * in FP32 and compensated FP32 pairs, the update applied in double-float
 * (two FP32 values, ~2^-44 relative) to the maintained vector; the
 * recomputation (a6), the final z and the stopping test's residual form
 * exact products (FMA error terms) summed in double-float, and a check of
 * the stopping test first rebuilds the maintained vector that way.  The
 * b x b solves (a4) run in double-float by default or in FP64 (ca_solve). */
typedef enum {
  CA_GRAM_F64 = 0,        /* FP64 on CUDA cores (any dense X)                   */
  CA_GRAM_FP32_EXACT = 1, /* FP32 X: 3xTF32 split products on tcgen05, FP32 acc. */
  CA_GRAM_TF32 = 2,       /* FP32 X: TF32 tcgen05 products, FP32 accumulate     */
  CA_GRAM_BF16X3 = 3,     /* FP32 X: x = b0 + b1 in BF16, b0 b0^T + b0 b1^T +
                           * b1 b0^T on tcgen05 (kind::f16), FP32 accumulate;
                           * each product within 3 * 2^-16 |x| |y|           */
  CA_GRAM_FP16_SCALED = 4 /* FP32 X: each row of A times a power of two that
                           * brings its largest magnitude into [2^14, 2^15),
                           * rounded to FP16, one product on tcgen05
                           * (kind::f16), FP32 accumulate, scales removed
                           * exactly; per-entry rounding 2^-11 (like TF32).
                           * The solve computes the scales in one pass over
                           * X.  Not in ca_gram_project_noalloc
                           * (CA_ERR_UNSUPPORTED).                           */
} ca_prec;

/* Arithmetic of the s unrolled b x b solves (step a4). */
typedef enum {
  CA_SOLVE_DF = 0,  /* b <= 32 and s*b <= 256: the diagonal blocks Gamma_j
                     * inverted up front (Gauss-Jordan sweep) and the
                     * dependent chain, both in double-float (pairs of FP32,
                     * ~2^-44 relative: GB300's FP64 pipe is ~1/64 of its
                     * FP32 pipe); larger b or s*b: as CA_SOLVE_F64          */
  CA_SOLVE_F64 = 1  /* FP64 throughout: a Cholesky factorisation of each
                     * Gamma_j in turn and the block forward substitution of
                     * eq. "recur", as Algorithm 2 / 4 write it (one CTA)     */
} ca_solve;

/* Stopping rule of the check every check_every outer steps (Sec. 5.1.5). */
typedef enum {
  CA_STOP_RESIDUAL = 0, /* end once ||r||_2 <= tol ||r_0||_2                  */
  CA_STOP_OBJECTIVE = 1 /* end once gap <= tol (f(w) - gap): the relative
                         * objective error (f(w) - f(w*))/f(w*) of the model
                         * w is then certified <= tol (gap and f: ca_info)  */
} ca_stop;

/* Solve options. */
typedef struct {
  int b;                /* block size b (primal) or b' (dual); 1 <= b <= N     */
  int s;                /* unrolling depth s >= 1 (s = 1: Algorithm 1 / 3)      */
  long long H;          /* number of inner iterations (block updates), H >= 1  */
  double lam;           /* regularisation lambda > 0                           */
  unsigned long long seed; /* sampler seed                                      */
  int prec;             /* ca_prec for the Gram of dense FP32 X                */
  int recompute_every;  /* a6 period in outer steps; 0 = never                  */
  long long h0;         /* index of the first block (resume point), >= 0      */
  /* Stopping criterion (Sec. 5.1.5): every check_every outer steps (0 = no
   * check) the full residual r of the current iterate is formed in one pass
   * over X -- primal: (1/n) X (y - X^T w) - lambda w, the negative gradient;
   * dual: X^T w - alpha - y, the dual residual up to sign; its rows at the
   * sampled indices are each block subproblem's right-hand side -- and the
   * solve ends once ||r||_2 <= tol ||r_0||_2 (tol = 0: never; the norms are
   * still reported).  r_0 is taken at the starting iterate; a check waits
   * for the GPU.  ca_solve_info reports what happened.
   * The norm also gives the duality gap of Sec. 2.2's primal / dual pair in
   * closed form: for the primal iterate w, at alpha = X^T w - y,
   * gap = f(w) + D(alpha) - ||y||^2/(2n) = ||r||^2/(2 lambda); for the dual
   * iterate alpha, at w = -X alpha/(lambda n), gap = ||r||^2/(2n).  Weak
   * duality gives f(w) - f(w*) <= gap (and D(alpha) - D(alpha*) <= gap).
   * With stop = CA_STOP_OBJECTIVE a check also forms f(w) from the
   * maintained vectors (primal: lambda/2 ||w||^2 + ||y - X^T w||^2/(2n);
   * dual: ||y||^2/(2n) - D(alpha) + gap; O(n + d) extra reads) and the
   * solve ends once gap <= tol (f(w) - gap): since f(w*) >= f(w) - gap,
   * the relative objective error is then certified <= tol.  The
   * certificate is as exact as the computed gap and f(w): on FP64 X to
   * FP64 rounding; on FP32 X each check rebuilds the maintained vector from
   * its definition and forms the residual with exact products summed in
   * double-float, so gap and f(w) carry errors of order 2^-44 of the sums
   * of |terms| behind them, far below any tol >= 1e-9 (the bounds are
   * derived by emulation and tested in the test suite's precision checks).
   * On FP32 X a check costs two passes over X.                          */
  double tol;
  int check_every;
  int stop;             /* ca_stop; CA_STOP_RESIDUAL unless set             */
  int solve;            /* ca_solve; CA_SOLVE_DF unless set                  */
} ca_opts;

/* What the last solve on a context did. */
typedef struct {
  long long h_done;     /* block updates performed: H unless the stopping test
                         * ended the solve (then a multiple of s); resume at
                         * h0 + h_done                                          */
  int checks;           /* full residuals formed after the start (the last one
                         * at the end of the solve when it ran to H)          */
  double res0;          /* ||r_0||_2 (0 without checks)                        */
  double res;           /* ||r||_2 at the last check                           */
  double gap;           /* duality gap at the last check (0 without checks)    */
  double fval;          /* f(w) of the model at the last check
                         * (CA_STOP_OBJECTIVE only; else 0)                    */
  double bound;         /* certified relative objective error at the last
                         * check, gap / (fval - gap) (CA_STOP_OBJECTIVE with
                         * fval > gap; else -1)                                */
} ca_info;

/* Dual CSR input: CSR of X^T with n rows (samples) and d columns (features).
 * rowptr has n+1 entries (int64), col and val have rowptr[n] entries; column
 * indices inside a row must be strictly increasing. */
typedef struct {
  const long long* rowptr;
  const int* col;
  const float* val;
} ca_csr;

typedef struct ca_ctx ca_ctx;

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  scratch_bytes_max
 * bounds the device memory the context may allocate for its scratch
 * (sampled indices, Gram partials, staging of host inputs); 0 = no bound.
 * Writes the new context to *ctx.  Errors: CA_ERR_ARG, CA_ERR_CUDA. */
int ca_bcd_init(ca_ctx** ctx, int device, void* cuda_stream, size_t scratch_bytes_max);

/* Primal CA-BCD (Algorithm 2; Algorithm 1 when s = 1).
 *   xfmt  CA_DENSE_F64, CA_DENSE_F32 or CA_DENSE_F32_PANELS.
 *   X     d x n row-major (row f = feature f), leading dimension ld >= n
 *         elements.  For the tcgen05 Gram modes, X and ld*4 bytes must be
 *         16-byte aligned; the solve then first repacks X into 32-column
 *         panels in its scratch (one pass over X; ca_pack_panels layout) and
 *         reads only the panels.  Host X: pageable memory is copied to the
 *         device first; page-locked (pinned) memory is read in place by the
 *         repack.  CA_DENSE_F32_PANELS: X is already in that
 *         layout (ceil(n/32) * d * 32 floats; ld is ignored); any of the
 *         tcgen05 Gram modes (TF32, 3xTF32, BF16x3, scaled FP16), not
 *         CA_GRAM_F64.
 *   y     n labels (FP64).
 *   w     d (FP64): w0 on entry, w_H on return.
 *   z     NULL, or n (FP64): receives X^T w_H computed by a final full pass.
 * Errors: CA_ERR_ARG (b > d, s < 1, H < 1, lambda <= 0, ld < n, bad format),
 * CA_ERR_UNSUPPORTED (s*b or b beyond this build's limits), CA_ERR_NOT_SPD,
 * CA_ERR_NONFINITE, CA_ERR_TIMEOUT, CA_ERR_OOM, CA_ERR_CUDA.  On error w and
 * z hold unspecified intermediate values. */
int ca_bcd_solve(ca_ctx* ctx, int xfmt, const void* X, long long d, long long n, long long ld,
                 const double* y, const ca_opts* opts, double* w, double* z);

/* Dual CA-BDCD (Algorithm 4; Algorithm 3 when s = 1).
 *   xfmt  CA_DENSE_F64 / CA_DENSE_F32: XT is X^T, n x d row-major (row i =
 *         sample i = column x_i of X), leading dimension ld >= d.
 *         CA_DENSE_F32_PANELS: X^T in 32-column panels (ceil(d/32) * n * 32
 *         floats).  FP32 with a tcgen05 Gram mode is repacked as for the
 *         primal.
 *         CA_CSR_F32: XT points to a ca_csr (ld is ignored).
 *   y     n labels (FP64).
 *   alpha n (FP64): alpha0 on entry, alpha_H on return.
 *   w     d (FP64): receives w_H (w0 = -X alpha0/(lambda n) is formed first,
 *         as Algorithms 3-4 initialise it).
 * Errors as ca_bcd_solve, with b <= n. */
int ca_bdcd_solve(ca_ctx* ctx, int xfmt, const void* XT, long long d, long long n, long long ld,
                  const double* y, const ca_opts* opts, double* alpha, double* w);

/* The sampler alone: writes blocks h0 .. h0+H-1 (H x b int32, row-major) of
 * b distinct indices of [0, N) to out, computed on the context's device.
 * out may be host or device memory.  Errors: CA_ERR_ARG, CA_ERR_CUDA. */
int ca_sample_indices(ca_ctx* ctx, unsigned long long seed, long long h0, long long H, int b,
                      long long N, int* out);

/* Outcome of the last ca_bcd_solve / ca_bdcd_solve on ctx (after it
 * returned CA_OK).  Errors: CA_ERR_ARG. */
int ca_solve_info(const ca_ctx* ctx, ca_info* out);

/* One check of the stopping test, as recorded by ca_solve_trace. */
typedef struct {
  long long h;          /* block updates of this solve done at the check (0:
                         * the start)                                         */
  double res;           /* ||r||_2                                            */
  double gap;           /* duality gap                                        */
  double fval;          /* f(w) of the model (CA_STOP_OBJECTIVE only; else 0) */
} ca_check;

/* Every check of the last solve on ctx, the one at the start first (the
 * trajectory behind Sec. 5.1.5's stopping test): copies the first
 * min(max, *count) of them to out (out may be NULL when max = 0) and their
 * number to *count.  A solve with check_every = 0 records none.  Errors:
 * CA_ERR_ARG. */
int ca_solve_trace(const ca_ctx* ctx, ca_check* out, int max, int* count);

/* Device scratch (bytes) a dense solve takes from ctx's arena when X, y and
 * the iterates are device memory: method 0 = ca_bcd_solve (X d x n), 1 =
 * ca_bdcd_solve (X^T n x d); xfmt CA_DENSE_F64, CA_DENSE_F32 or
 * CA_DENSE_F32_PANELS; o as for the solve.  The solve grows the arena to at
 * least this (host-resident inputs add their staging).  Used to admit work
 * by HBM footprint.  Errors: CA_ERR_ARG, CA_ERR_UNSUPPORTED. */
int ca_solve_scratch_bytes(ca_ctx* ctx, int method, int xfmt, long long d, long long n,
                           const ca_opts* o, size_t* bytes);

/* Free ctx's scratch arena (after the work on its stream ends); the next
 * call allocates what it needs again.  Errors: CA_ERR_ARG, CA_ERR_CUDA. */
int ca_bcd_release_scratch(ca_ctx* ctx);

/* Steps a2+a3 alone for given sampled rows (Alg. 2 / 4, "compute the Gram
 * matrix"): for the sb rows idx[0..sb) of the N x K row-major matrix A
 * (leading dimension ld), writes G = Y Y^T (sb x sb, row-major, FP64, full
 * symmetric, no scaling and no lambda) and p = Y v (sb, FP64), where v has K
 * entries.  A, idx, v, G and p must be device memory.  xfmt and prec as for
 * the solves (TF32 / 3xTF32 / BF16x3 / scaled FP16 need FP32 A, 16-byte
 * aligned rows, sb <= 256).
 * Errors: CA_ERR_ARG, CA_ERR_UNSUPPORTED, CA_ERR_OOM, CA_ERR_CUDA. */
int ca_gram_project(ca_ctx* ctx, int xfmt, int prec, const void* A, long long N, long long K,
                    long long ld, const int* idx, int sb, const double* v, double* G, double* p);

/* Steps a2+a3 as ca_gram_project computes them (the same kernels; the split-K
 * partials are summed in a different order, so the results agree to
 * rounding: within 1e-12 relative on FP64 A, and within the Gram mode's
 * product bound on FP32 A), for callers that must not allocate device memory
 * (the paper has no counterpart: this is an interface convenience).  Such callers include code running while a host
 * framework owns every device allocation through its own pool, code on a
 * latency-critical path where an allocation's implicit synchronisation is not
 * acceptable, and code that may only enqueue work on a stream it was given.
 * No context is needed and nothing is allocated: the scratch is one fixed
 * device array inside the library (6.5 MiB, held on every GPU that loads the
 * library until the process exits).
 *   cuda_stream  the cudaStream_t to run on (NULL = legacy default stream),
 *                on the current device.
 *   Limits: sb <= 128 and K <= 262144 (beyond them: CA_ERR_UNSUPPORTED);
 *   prec CA_GRAM_FP16_SCALED needs per-row scales the fixed array has no
 *   room for (CA_ERR_UNSUPPORTED).
 *   A, idx, v, G, p: as ca_gram_project, all device memory.
 * The first call on a device looks up the array's device address (keep that
 * first call outside any stream capture).  All calls share the array and it
 * keeps the previous call's contents; calls that overlap on the GPU race on
 * it, so order them (one stream, or events).  The call returns after the
 * stream has finished its work.  Errors: CA_ERR_ARG, CA_ERR_UNSUPPORTED,
 * CA_ERR_TIMEOUT, CA_ERR_CUDA. */
int ca_gram_project_noalloc(void* cuda_stream, int xfmt, int prec, const void* A, long long N,
                            long long K, long long ld, const int* idx, int sb, const double* v,
                            double* G, double* p);

/* Storage conversion for the tcgen05 Gram modes (not a step of the paper's
 * method: a layout of X that the gather reads at a higher fraction of HBM
 * bandwidth).  Writes the N x K row-major FP32 matrix A (leading dimension
 * ld, A and ld*4 bytes 16-byte aligned) as ceil(K/32) panels of N rows x 32
 * columns: out[(a*N + r)*32 + c] = A[r][32a + c], zero where 32a + c >= K.
 * out holds ceil(K/32)*N*32 floats.  A and out are device memory owned by the
 * caller; the work runs on the context's stream and the call returns when it
 * is enqueued (pass the result to the solves as CA_DENSE_F32_PANELS).
 * Errors: CA_ERR_ARG, CA_ERR_CUDA. */
int ca_pack_panels(ca_ctx* ctx, const float* A, long long N, long long K, long long ld, float* out);

/* Text of the last failing CUDA call seen by an entry point on this context
 * (empty if none); owned by the context, valid until the next call. */
const char* ca_last_error(ca_ctx* ctx);

/* Name of a status code (static string). */
const char* ca_status_str(int status);

/* Tuning of the dense tensor-core solves on ctx (kept until changed).
 *   CA_TUNE_PERSISTENT  1 (default): a run of full outer steps between two
 *       host decisions (a check of the stopping test, a due recomputation,
 *       the short last step) runs as one persistent cooperative launch when
 *       the solve fits it (FP32 X in 32-column panels, BF16x3 or scaled-FP16
 *       Gram, s*b <= 128, b <= 8, CA_SOLVE_DF, at least s + 1 Gram CTAs):
 *       the s unrolled solves of step k (eq. "recur", Algorithms 2 and 4)
 *       then run while the Gram pass of step k+1 streams its rows, and that
 *       pass corrects its projection by the cross Gram of the two steps'
 *       rows (the same sums in exact arithmetic).  0: one Gram launch and
 *       one solve launch per outer step.
 *   CA_TUNE_OVERLAP  share in [0, 1] of each Gram CTA's columns streamed
 *       before the previous step's solve is known (default 0.4; 0: none).
 * Errors: CA_ERR_ARG (NULL context, unknown key, value out of range). */
#define CA_TUNE_PERSISTENT 1
#define CA_TUNE_OVERLAP 2
int ca_set_tuning(ca_ctx* ctx, int key, double value);

/* Measurement hooks.  With profiling on, every following solve records CUDA
 * event pairs on the context's stream around each launch of five kernel
 * classes: [0] the Gram pass (a2+a3), [1] the reduction of its partials (and
 * the factorisation of the diagonal blocks, a4), [2] the deferred update
 * (a5), [3] everything else (sampling a1, the recomputations a6), [4] the
 * dependent chain of inner solves (a4).  ca_profile_read fills ms[5] (summed
 * event time per class), launches[5] (timed intervals per class) and
 * *kernel_launches (all kernels the solves launched) since the last
 * ca_profile_enable; any pointer may be NULL.  Errors: CA_ERR_ARG for a NULL
 * context. */
int ca_profile_enable(ca_ctx* ctx, int on);
int ca_profile_read(ca_ctx* ctx, double* ms, long long* launches, long long* kernel_launches);

/* Diagnostic: runs one kernel whose thread waits on a device barrier that
 * nothing completes, through the same bounded wait the Gram kernel uses,
 * with a limit of limit_ns nanoseconds (1 .. 1e9).  Returns CA_ERR_TIMEOUT
 * when the wait gave up as designed (the context stays usable), CA_OK if it
 * did not, CA_ERR_ARG / CA_ERR_CUDA on bad input or a CUDA failure. */
int ca_selftest_wait_timeout(ca_ctx* ctx, long long limit_ns);

/* Release the context and its scratch (caller memory is untouched). */
void ca_bcd_destroy(ca_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CA_BCD_H */
