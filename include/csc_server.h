/*
 * csc_server.h - a serving engine for convolutional sparse coding requests
 * (Eq. sparse_code of Moreau, Oudre & Vayatis, "DICOD", ICML 2018) on one GPU.
 *
 * The paper solves one signal at a time; it has no serving counterpart.  This
 * interface is the deployment side of the same solver (include/csc.h): many
 * requests of uneven length against a few resident dictionaries, solved with
 * continuous batching.
 *
 *   - Dictionaries are set up once (DtD and norms stay on the GPU).
 *   - csc_server_submit queues a request: a signal X [P][T] for one
 *     dictionary, its lambda and its tolerance.  The server copies X.
 *   - Each csc_server_step (a scheduling round) admits queued requests, in
 *     submission order per dictionary, while their device state fits in the
 *     device-memory budget (one pool allocated at creation: the server never
 *     allocates beyond it; while other dictionaries have requests waiting, a
 *     dictionary holds at most its fair share, pool / dictionaries), runs a
 *     fixed number of CD sweeps over ALL active
 *     requests of each dictionary in the same phase launches (every request
 *     is cut into its own segments, Sec. 2.2; the dictionaries' launches run
 *     on separate streams and overlap on the device), re-synchronises and
 *     checks the requests whose CD round ended, and retires the converged
 *     ones.  A request admitted while others run joins the next round's
 *     launches; memory freed by a retired request admits the next ones.
 *   - csc_server_fetch copies a finished request's Z out and releases its
 *     memory.
 * A request's arithmetic does not depend on the other requests: its
 * segments, phases, sweeps per round, resyncs and reductions are its own, so
 * its result is bitwise the same alone and in any mix.
 *
 * Per request the solve is that of csc_solve: CD to tol/2, FP64-accurate
 * resync, accepted when the refreshed max |Delta Z| < tol (at most
 * max_resyncs resyncs), objective in FP64 from the explicit residual.
 *
 * Errors: int status as in csc.h (CSC_OK, CSC_EINVAL, CSC_ENOMEM, CSC_ECUDA,
 * CSC_ESTATE); text from csc_last_error_string().  A server is used by one
 * host thread at a time.
 */
#ifndef CSC_SERVER_H
#define CSC_SERVER_H

#include <stdint.h>

#include "csc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct csc_server_s *csc_server_t;

#define CSC_REQ_QUEUED 0
#define CSC_REQ_ACTIVE 1
#define CSC_REQ_DONE 2

typedef struct csc_server_opts {
    int64_t hbm_budget_bytes;  /* device memory for request state, allocated once at
                                  creation; 0 = 40 GiB */
    int32_t sweeps_per_step;   /* CD sweeps per dictionary per csc_server_step; 0 = 4 */
    int32_t max_resyncs;       /* per request, -1 = 3 */
    int32_t max_active;        /* active requests per dictionary, 0 = no limit */
    int32_t reserved[3];       /* must be zero */
} csc_server_opts;

typedef struct csc_request_info {
    int32_t state;           /* CSC_REQ_* */
    int32_t dict;
    int64_t T;               /* samples */
    double lambda;           /* lambda used */
    double lambda_max;       /* max |D~ * X| (set at admission) */
    double objective;        /* E(Z) in FP64 (DONE) */
    double max_delta_z;      /* max |Delta Z| on the last refreshed state */
    int32_t resyncs;
    int32_t converged;       /* 1: accepted at tol; 0: stopped after max_resyncs */
    int64_t rounds;          /* scheduling rounds the request was active in */
    int64_t device_bytes;    /* pool bytes it holds (0 once fetched) */
    double t_submit, t_admit, t_done;  /* seconds on the server's monotonic clock */
} csc_request_info;

/* Creates a server on the current device; allocates the request pool. */
int csc_server_create(csc_server_t *s, const csc_server_opts *opts);

/*
 * Adds a resident dictionary D [K][P][L] (host or device; copied) and
 * returns its index.  segment_width (>= 1, 0 = 2L-2) and updates_per_visit
 * (0 = 24) apply to all its requests; every request of the dictionary runs in
 * the same c = 1 + ceil((2L-2) / segment_width) phases (2 at the default
 * width; narrower segments take less shared memory each, so more of them run
 * at once).  CSC_EINVAL if sweeps_per_step x c exceeds 4096 launches.
 */
int csc_server_add_dictionary(csc_server_t s, const float *D, int K, int P, int L,
                              int32_t segment_width, int32_t updates_per_visit, int *dict);

/*
 * Queues a request: X [P][T] float32 (host or device; copied now), T >= L.
 * lambda > 0: absolute; lambda < 0: |lambda| * lambda_max of this X (e.g.
 * -0.1 for 0.1 lambda_max, computed on the device at admission).  tol > 0.
 * A request whose state cannot fit in the whole pool is rejected (CSC_ENOMEM).
 */
int csc_server_submit(csc_server_t s, int dict, const float *X, int64_t T, double lambda,
                      double tol, int64_t *request);

/* One scheduling round (see above).  Receives the counts after the round. */
int csc_server_step(csc_server_t s, int *n_active, int *n_queued, int *n_done);

/* Completion queue: up to cap ids of requests that finished (DONE) since the
 * previous call, in finishing order, into requests[]; *n receives the count
 * (ids beyond cap stay queued for the next call).  Every finished request is
 * reported exactly once, also when it was fetched before it was reported;
 * the queue keeps 8 bytes per finished request until it is read.
 * cap = 0 with requests = NULL only reads nothing (returns *n = 0). */
int csc_server_completed(csc_server_t s, int64_t *requests, int cap, int *n);

/* State and statistics of a request (any state). */
int csc_server_info(csc_server_t s, int64_t request, csc_request_info *info);

/* For a DONE request: copies Z [K][T-L+1] (host or device, NULL to skip),
 * fills info, and releases the request. */
int csc_server_fetch(csc_server_t s, int64_t request, float *Z_out, csc_request_info *info);

/* Pool size, bytes held by requests now, and the most ever held. */
int csc_server_memory(csc_server_t s, int64_t *pool_bytes, int64_t *in_use, int64_t *peak);

/* Kernels launched by the server since creation. */
int csc_server_kernel_launches(csc_server_t s, int64_t *out);

/* Releases everything (queued and unfetched requests included). */
int csc_server_destroy(csc_server_t s);

#ifdef __cplusplus
}
#endif

#endif /* CSC_SERVER_H */
