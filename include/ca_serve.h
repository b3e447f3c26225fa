/* Serving loop for ridge solves on one GPU (not a step of the paper's
 * method; a host runtime around ca_bcd_solve / ca_bdcd_solve).
 *
 * A server owns `workers` library contexts, each on its own CUDA stream and
 * host thread, so admitted requests run concurrently on the device.
 * Requests are admitted in submission order (strict FIFO) when a worker is
 * idle and the scratch arenas of all workers, with the chosen one grown to
 * the request's need (ca_solve_scratch_bytes), fit `budget_bytes`; when the
 * head request fits on no idle worker, idle workers' arenas are released
 * (largest first) before it waits for a running request to end.  A request
 * whose need exceeds the whole budget ends at once with CA_ERR_OOM.  The
 * request's own arrays (X, y, iterates) are device memory owned by the
 * caller and stay resident; they are not part of the budget.  Each request
 * computes exactly what the same call made alone computes.
 */
#ifndef CA_SERVE_H
#define CA_SERVE_H

#include <stddef.h>

#include "ca_bcd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ca_server ca_server;

typedef struct {
  int method;        /* 0: primal CA-BCD (ca_bcd_solve); 1: dual CA-BDCD (ca_bdcd_solve) */
  int xfmt;          /* CA_DENSE_F64, CA_DENSE_F32 or CA_DENSE_F32_PANELS */
  const void* X;     /* device: primal X (d x ld), dual X^T (n x ld), or panels */
  long long d, n, ld;
  const double* y;   /* device, n labels */
  double* x;         /* device: primal w (d; w0 in, w_H out); dual alpha (n; in/out) */
  double* aux;       /* device: primal z = X^T w_H (n) or NULL; dual w (d, out) */
  ca_opts opts;      /* as for the solve (stopping test included); opts.s = 0:
                      * the server picks s by measured cost: requests of one
                      * shape class (method, xfmt, prec, b, binades of N and
                      * K) try each s with s*b <= 256 once, then run the one
                      * with the least measured time per block update        */
} ca_request;

typedef struct {
  int status;             /* CA_OK or the solve's error code                */
  int worker;             /* context that ran it (-1: rejected)             */
  int s;                  /* unrolling depth it ran with                    */
  long long h_done;       /* block updates performed (ca_solve_info)        */
  double res0, res;       /* residual norms of the stopping test (or 0)     */
  double gap, fval;       /* duality gap and f(w) at the last check
                           * (ca_info; fval under CA_STOP_OBJECTIVE only)   */
  double bound;           /* certified relative objective error there
                           * (ca_info.bound; -1 when none)                  */
  double queue_ms;        /* submission -> start                            */
  double run_ms;          /* start -> end                                   */
  double latency_ms;      /* submission -> end                              */
  size_t scratch_bytes;   /* the request's footprint                        */
} ca_result;

typedef struct {
  long long submitted, completed, rejected;
  double p50_ms, p99_ms, mean_ms, max_ms; /* latency, submission -> end     */
  double wall_s;                          /* first submission -> last end   */
  double block_updates_per_s;             /* sum of h_done / wall_s         */
  size_t peak_footprint;                  /* largest admitted sum of arenas */
  int peak_concurrency;                   /* most requests running at once */
} ca_server_stats;

/* Create a server on CUDA device `device` with `workers` >= 1 contexts and a
 * scratch budget of budget_bytes >= 1.  Errors: CA_ERR_ARG, CA_ERR_CUDA. */
int ca_server_create(ca_server** out, int device, int workers, size_t budget_bytes);

/* Queue a copy of *r; returns at once with its id (0, 1, ...).  The arrays
 * it points to must be memory of the server's device (or managed memory)
 * and stay valid until the request ends.
 * Errors: CA_ERR_ARG (host pointers, or options the solve would refuse),
 * CA_ERR_UNSUPPORTED. */
int ca_server_submit(ca_server* s, const ca_request* r, long long* id);

/* Batching: from now on the scheduler may start the queue's head together
 * with up to max_group - 1 requests queued right behind it that a batched
 * solve accepts (ca_batch_solve: FP32 X, the head's tcgen05 Gram mode,
 * b <= 16, s*b <= 128 or s = 0), as one ca_batch_solve on one worker, when
 * the group's scratch (the sum of each member's ca_batch_scratch_bytes
 * alone) fits the budget.  The group's requests share the Gram, reduction
 * and chain launches of each round and end together.  max_group = 1: every
 * request runs alone (the default).  Errors: CA_ERR_ARG. */
int ca_server_set_batching(ca_server* s, int max_group);

/* Block until request id has ended; its outcome in *out.  Errors:
 * CA_ERR_ARG (unknown id). */
int ca_server_wait(ca_server* s, long long id, ca_result* out);

/* Block until every submitted request has ended.  Errors: CA_ERR_ARG. */
int ca_server_drain(ca_server* s);

/* Latency percentiles and throughput over the requests ended so far.
 * Errors: CA_ERR_ARG. */
int ca_server_get_stats(ca_server* s, ca_server_stats* out);

/* Drain, then free the contexts and streams.  NULL is a no-op. */
void ca_server_destroy(ca_server* s);

/* Batched solves: `count` dense problems of uneven sizes solved together on
 * ctx (its stream, its scratch arena).  Each round runs one outer step of
 * every unfinished problem in three shared launches: one Gram pass whose
 * CTAs split the concatenation of all problems' 32-column atoms into
 * stretches of equal HBM cost (steps a2+a3, with each problem's deferred
 * update a5 fused in), one reduction of every problem's split-K partials
 * with the inversion of its diagonal blocks, and one chain CTA per problem
 * (the s unrolled solves of eq. "recur" / its dual analogue, step a4).
 * Problems are independent: each computes what ca_bcd_solve / ca_bdcd_solve
 * computes alone, up to the order of the FP32 Gram sums (the split-K
 * partition of its atoms differs).
 *   reqs[i]  method 0 (primal: x = w, aux = z or NULL) or 1 (dual: x =
 *            alpha, aux = w, required); xfmt CA_DENSE_F32 (row-major, ld a
 *            multiple of 4, repacked into panels in ctx's scratch) or
 *            CA_DENSE_F32_PANELS; every array device memory.  opts: one
 *            tcgen05 Gram mode for all problems; b <= 16; s*b <= 128, or
 *            s = 0: the depth is chosen by measured cost (a warm-up round,
 *            then one timed round each at s*b = 128, 64, 32 rows per outer
 *            step, then the cheapest per block update; changing s between
 *            outer steps keeps the s = 1 iterates in exact arithmetic);
 *            recompute_every and the stopping test (check_every, tol, stop)
 *            as for the solves (a check rebuilds the problem's maintained
 *            vector, forms its residual and waits for the GPU; a problem
 *            that meets its rule leaves the rounds); solve CA_SOLVE_DF
 *            (else CA_ERR_UNSUPPORTED).
 *   flags    CA_BATCH_GRAPH: rounds that differ only in pointers (a segment,
 *            up to 64 rounds) are captured into one CUDA graph and launched
 *            as one (needs a non-NULL stream on ctx; ignored while
 *            profiling).
 *   out      count results: status, s (the depth of the last step), h_done,
 *            and the stopping test's res0, res, gap, fval and bound.
 * Returns after the work finished.  Errors: CA_ERR_ARG, CA_ERR_UNSUPPORTED,
 * CA_ERR_OOM, CA_ERR_CUDA, and the device errors of the solves (then no
 * result is valid). */
#define CA_BATCH_GRAPH 1
int ca_batch_solve(ca_ctx* ctx, int count, const ca_request* reqs, int flags, ca_result* out);

/* Device scratch (bytes) ca_batch_solve takes from ctx's arena for these
 * requests (with the same checks of the requests).  Errors: as
 * ca_batch_solve's argument checks. */
int ca_batch_scratch_bytes(ca_ctx* ctx, int count, const ca_request* reqs, size_t* bytes);

#ifdef __cplusplus
}
#endif

#endif /* CA_SERVE_H */
