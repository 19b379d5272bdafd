/*
 * nufft_serve.h -- a request loop over the transforms of nufft_gb300.h for
 * serving: type-1 / type-2 requests of any dimension, mode counts, point
 * count, precision and eps arrive at any time and are run with continuous
 * batching on one GPU.
 *
 *  - Requests are admitted in arrival order (FIFO) as soon as an execution
 *    slot is free and their device footprint fits the memory budget; each
 *    admitted request runs on its own slot stream, so requests that arrive
 *    while others are on the GPU start at once and their kernels overlap
 *    with the earlier ones'.
 *  - Plans stay resident between requests ("plan entries", keyed by kind,
 *    dimension, mode counts, sign, precision and eps, with a point capacity);
 *    an idle entry with the same key and enough capacity is reused, and its
 *    sorted points too when the request carries the same nonzero points_key
 *    and point count (the binning step, Sec. 3.1 / Sec. 5.1, is then skipped).
 *  - Admission counts each entry's device bytes: fine grid n_1...n_d complex
 *    values, correction factors, bins, point records and subproblem lists,
 *    cuFFT's work area, and the scratch of gradient requests.  The paper
 *    stresses this footprint (RAM column of its Table t:big).  Idle entries
 *    are destroyed, least recently used first, when a new one would not fit.
 *  - The host never blocks on the device: completions arrive through host
 *    callbacks on the slot streams.  A request that is not done within the
 *    time limit is reported early with NUFFT_ERR_TIMEOUT and pending = 1: its
 *    kernels may still be running and writing its outputs.  Its entry and
 *    slot stay out of use until the work ends, and then a second, final
 *    completion for the same ticket (pending = 0, status of the work) follows.
 *
 * Threading: one scheduler thread per server; submit / poll / drain /
 * stats may be called from any host thread.  All pointers in a request are
 * device memory on the server's device, owned by the caller, and must stay
 * valid (inputs unchanged) until the request's FINAL completion (pending = 0)
 * has been polled, or until nufft_server_drain has returned NUFFT_OK.  A
 * pending TIMEOUT completion does not release them.
 */
#ifndef NUFFT_SERVE_H
#define NUFFT_SERVE_H

#include "nufft_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

/* request kinds */
#define NUFFT_REQ_TYPE1 1    /* f = F1(x) c   (Eq. (1)) */
#define NUFFT_REQ_TYPE2 2    /* c = F2(x) f   (Eq. (2)) */
#define NUFFT_REQ_LSQ_GRAD 3 /* loss = sum_j |F2(f; x)_j - y_j|^2 and its gradients in f and x */

/* request flags */
#define NUFFT_FLAG_XGRAD_KERNEL 1 /* LSQ_GRAD: grad_x through the ES kernel's derivative (nufft_execute_grad,
                                     one FFT) instead of dim extra type-2 transforms of (i k_d) f */

typedef struct {
  int kind;            /* NUFFT_REQ_* */
  int flags;           /* NUFFT_FLAG_* or 0 */
  int dim;             /* 1, 2 or 3 */
  int64_t nmodes[3];   /* N_1 .. N_dim (entries above dim ignored) */
  int isign;           /* +1 or -1: the sign of the exponent (of F2 for LSQ_GRAD) */
  int prec;            /* NUFFT_C64 or NUFFT_C128 */
  double eps;          /* tolerance, as for nufft_makeplan */
  double upsampfac;    /* 2 or 1.25 (opts.upsampfac), or 0: the server picks per request by a cost model
                          (fine-grid cells against M w^d stencil cells; see nufft_request_upsampfac) */
  int64_t M;           /* number of points, 0 <= M < 2^31 */
  const void* x;       /* M coordinates each (float / double per prec); y NULL if dim < 2, z if dim < 3 */
  const void* y;
  const void* z;
  const void* in;      /* TYPE1: c (M complex); TYPE2 and LSQ_GRAD: f (modes, dimension 1 fastest, increasing k) */
  const void* in2;     /* LSQ_GRAD: y (M complex targets); otherwise unused */
  void* out;           /* TYPE1: f (modes); TYPE2: c (M); LSQ_GRAD: grad_f (modes) */
  void* out2;          /* LSQ_GRAD: grad_x, dim rows of M reals (row d at offset d*M); otherwise unused */
  void* out3;          /* LSQ_GRAD: the loss, ONE double; otherwise unused */
  uint64_t points_key; /* 0, or an id the caller gives to a point set it does not change */
  void* ready_event;   /* NULL or a cudaEvent_t recorded after the inputs were written */
  uint64_t tag;        /* returned unchanged in the completion */
} nufft_request;

typedef struct {
  int64_t ticket;  /* from nufft_server_submit */
  uint64_t tag;
  int status;      /* NUFFT_OK, NUFFT_ERR_TIMEOUT, NUFFT_ERR_REJECTED, NUFFT_ERR_SHUTDOWN, or a plan error */
  int reused;      /* 1: ran on a resident plan entry; 2: and skipped the binning step */
  double t_submit; /* seconds on nufft_server_clock() */
  double t_admit;  /* slot and memory granted, work enqueued */
  double t_done;   /* the device finished (or the time limit expired) */
  int pending;     /* 1: an early NUFFT_ERR_TIMEOUT report; the request's device work has not ended and a
                      final completion with the same ticket follows.  0: final; the request's buffers are free */
} nufft_completion;

/* completed counts final completions; timeouts counts early NUFFT_ERR_TIMEOUT reports */
typedef struct {
  int64_t submitted, completed, timeouts, rejected;
  int64_t entries_created, entries_evicted, entries_reused, binning_skipped;
  int64_t queued, inflight, peak_inflight;
  int64_t bytes_in_use, peak_bytes, budget_bytes;
} nufft_server_stats;

typedef struct nufft_server_s* nufft_server;

/* A server on the current CUDA device.  budget_bytes: device bytes the plan
 * entries may hold in total; max_inflight: execution slots (1..64);
 * timeout_s: per-request limit from admission (<= 0: none).  Returns
 * NUFFT_OK, NUFFT_ERR_BAD_ARG, NUFFT_ERR_CUDA, NUFFT_ERR_ALLOC. */
int nufft_server_create(size_t budget_bytes, int max_inflight, double timeout_s, nufft_server* out);

/* Queue a request (copied; returns at once).  NUFFT_ERR_BAD_ARG for an
 * invalid request (the server is unchanged); *ticket numbers requests from 1. */
int nufft_server_submit(nufft_server s, const nufft_request* r, int64_t* ticket);

/* Move up to max completions to out (in completion order), waiting up to
 * wait_s seconds for the first one; *n = number moved (0 on time-out). */
int nufft_server_poll(nufft_server s, nufft_completion* out, int max, int* n, double wait_s);

/* Wait until nothing is queued or running (at most timeout_s seconds, <= 0:
 * no limit).  NUFFT_OK, or NUFFT_ERR_TIMEOUT if work is left. */
int nufft_server_drain(nufft_server s, double timeout_s);

int nufft_server_stats_get(nufft_server s, nufft_server_stats* st);

/* Stop the scheduler, fail queued requests with NUFFT_ERR_SHUTDOWN, wait for
 * running work (up to 60 s), free every plan entry.  Entries whose work the
 * executor has not reported by then are left allocated (leaked), not freed
 * under running kernels.  NULL is accepted. */
int nufft_server_destroy(nufft_server s);

/* Seconds on the clock the completions use (a monotonic clock). */
double nufft_server_clock(void);

/* Host-only: the upsampling factor the server uses for r: r->upsampfac when
 * it is 2 or 1.25; for 0, 1.25 when eps needs no more than w = 16 at 1.25 and
 *   a prod(n_i(1.25)) + b M w(1.25)^dim  <  a prod(n_i(2)) + b M w(2)^dim,
 * with a = 13 ps per fine-grid cell (zeroing or pre-correcting, FFT and
 * correction of one transform) and b = 0.7 ps per stencil cell of a point, as
 * measured on the GB300 for 3D complex64; otherwise 2.  Returns 0 for an
 * invalid request. */
double nufft_request_upsampfac(const nufft_request* r);

/* Host-only: upper estimate of the device bytes a plan entry for r needs
 * with room for mcap points (the figure admission uses). */
int nufft_request_bytes(const nufft_request* r, int64_t mcap, size_t* bytes); /* pointers in r are not read */

/* ---- test seam: the scheduler over caller-supplied execution callbacks ----
 * The same admission, reuse, eviction, slot and time-limit policy, but plan
 * entries are created, run and destroyed by these callbacks instead of the
 * GPU; used to test the policy without a device.  launch must arrange for
 * nufft_server_complete(server, ticket, status) to be called once, from any
 * thread, when the request's work is done. */
typedef struct {
  void* ctx;
  int (*estimate)(void* ctx, const nufft_request* r, int64_t mcap, size_t* bytes);
  int (*create)(void* ctx, const nufft_request* r, int64_t mcap, void** entry, size_t* bytes);
  int (*launch)(void* ctx, void* entry, const nufft_request* r, int slot, int skip_binning, int64_t ticket);
  void (*destroy)(void* ctx, void* entry);
} nufft_executor;

int nufft_server_create_with_executor(const nufft_executor* ex, size_t budget_bytes, int max_inflight,
                                      double timeout_s, nufft_server* out);
void nufft_server_complete(nufft_server s, int64_t ticket, int status);
/* How long nufft_server_destroy waits for running work before it leaks the
 * entries of requests the executor has not reported (default 60 s; > 0). */
int nufft_server_set_shutdown_wait(nufft_server s, double seconds);

#ifdef __cplusplus
}
#endif

#endif /* NUFFT_SERVE_H */
