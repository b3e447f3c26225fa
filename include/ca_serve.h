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

#ifdef __cplusplus
}
#endif

#endif /* CA_SERVE_H */
