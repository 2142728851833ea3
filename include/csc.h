/*
 * csc.h - C ABI of the GB300 convolutional sparse coding solver.
 *
 * Problem (Eq. sparse_code, Sec. 2.1 of Moreau, Oudre & Vayatis, "DICOD",
 * ICML 2018): given atoms D[K][P][L] and a signal X[P][T], find
 *     Z* = argmin_Z  1/2 || X - sum_k Z_k * D_k ||_2^2 + lambda sum_k ||Z_k||_1,
 * with Z[K][Tz], Tz = T - L + 1 ("valid" placement: atom k at offset t covers
 * samples t..t+L-1 of X; X is zero outside [0,T), Sec. 2 "Notations").
 * The paper writes W for the atom length and L for Tz.
 *
 * Method: locally greedy coordinate descent on M contiguous time segments
 * (Sec. 2.2 DICOD, Alg. 2; Sec. 2.3 Alg. 3).  Each GPU thread block owns one
 * segment, picks argmax |Delta Z| inside it, applies Eq. pb_coord and updates
 * beta by Eq. beta_up on the window [t0-L+1, t0+L-1], writing directly into
 * idle neighbouring segments (the paper's neighbour messages).  Segments run
 * in c phases (segments m == p mod c together); c is chosen so that no two
 * co-active segments touch the same beta entries, which makes every phase
 * equivalent to a sequential run of its segments (hypothesis H2 of Theorem
 * conv_dcp holds with A = c phases; H3 is not needed).
 *
 * Layouts (all row-major, float32 unless stated):
 *   D      [K][P][L]        atom k, channel p, lag tau
 *   X      [P][T]
 *   Z      [K][Tz]
 *   beta   [K][Tz]
 *   DtD    [K][K][2L-1]     DtD[k0][k][s] = sum_p sum_tau D[k][p][tau] D[k0][p][tau+s-(L-1)]
 *                           (= S_{k,k0}[s-(L-1)] of Eq. beta_up; the slice for one
 *                           updated atom k0 is contiguous)
 *
 * Pointers: every array argument may be a device pointer (cudaMalloc, torch)
 * or a host pointer (pageable or pinned); the library detects which with
 * cudaPointerGetAttributes and copies host data itself.  The caller keeps
 * ownership of every array it passes; the library copies what it keeps.
 *
 * Errors: every entry point returns an int status.  CSC_OK (0) is success;
 * CSC_NOT_CONVERGED (1) means max_updates or the sweep limit was reached, or
 * the exact check after the last resync allowed still found a coordinate
 * with |Delta Z| >= tol (Z and the objective are still valid).  Negative values are errors; the
 * text of the last error of the calling thread is csc_last_error_string().
 * No C++ exception crosses this boundary.
 *
 * Threads and streams: a handle is used by one host thread at a time; all of
 * its GPU work is ordered on the stream given to csc_setup.  A handle lives
 * on the device that was current at its first csc_setup; every call on it
 * switches to that device and restores the caller's current device before
 * returning.  Calls that read
 * results back (csc_solve, the getters) synchronise that stream.
 */
#ifndef CSC_H
#define CSC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CSC_OK 0
#define CSC_NOT_CONVERGED 1
#define CSC_EINVAL (-1)   /* bad argument: sizes, lambda, tol, null pointer */
#define CSC_ENOMEM (-2)   /* device or host allocation failed */
#define CSC_ECUDA (-3)    /* a CUDA call or kernel failed */
#define CSC_ETIMEOUT (-4) /* a bounded device wait gave up */
#define CSC_ESTATE (-5)   /* call out of order (e.g. csc_solve before csc_init) */

typedef struct csc_handle_s *csc_handle_t;

typedef struct csc_opts {
    int32_t segments;          /* M >= 1 for a single signal; 0 = automatic (see
                                  segment_width).  Batches always use segment_width */
    int32_t updates_per_visit; /* u: updates a segment may apply per phase; 0 = until local
                                  convergence (bounded internally by 2^20) */
    int32_t max_resyncs;       /* exact re-synchronisations of beta (double-float
                                  accumulation from D~*X) after the float32 loop settles;
                                  CD resumes after one that finds |Delta Z| >= tol.  When
                                  the loop settles again after the last one allowed, one
                                  more exact refresh decides the status: CSC_OK if it finds
                                  every |Delta Z| below tol, else CSC_NOT_CONVERGED.
                                  -1 = default (3); 0 = none (the status is then the float32
                                  loop's own test; stats.max_delta_z reports the exact one) */
    int32_t sweeps_per_poll;   /* sweeps between two convergence tests (a batch); 0 =
                                  default (4) */
    int32_t max_sweeps;        /* 0 = default (1,000,000) */
    int32_t time_kernels;      /* 1 = time every phase launch with a CUDA event pair
                                  (csc_stats.phase_ms); 0 = off */
    int32_t segment_width;     /* target segment width in columns when segments is 0 or
                                  the problem is a batch: each signal gets
                                  max(1, floor(Tz_i / width)) segments.  0 = 2L-2, the
                                  narrowest width that needs only 2 phases */
    int32_t init_mode;         /* beta0 = D~ * X in csc_init: 1 = tensor cores, X and D
                                  split into three BF16 terms, six products accumulated
                                  in FP32 (FP32-grade); 2 = tensor cores, one BF16 product
                                  (only to measure its error); 3 = FP32 CUDA cores with
                                  compensated sums; 0 = automatic: mode 1 where one of its
                                  CTAs fits on an SM (shared memory grows with P * L), else
                                  mode 3.  Modes 1-2 need K <= 64; other sizes use mode 3 */
    int32_t launch_mode;       /* 0 = each CD round runs as one CUDA graph, a while loop over
                                  batches whose convergence test runs on the device (captured
                                  the second time a plan is solved; a plan solved once runs
                                  direct launches with a host wait per batch); 1 = direct
                                  kernel launches.  Same results */
    int32_t threads_per_segment; /* threads that run one segment's visit: 0 = automatic
                                  (a block), 128 = a block of at least 2L-1 threads per
                                  segment, 32 = one warp per segment where eligible (K =
                                  25, 2L-1 <= 128, the segment's tile fits shared memory;
                                  else a block).  Both meet the same bars */
} csc_opts;

typedef struct csc_stats {
    int64_t updates;          /* applied coordinate updates (each with |Delta Z| >= tol) */
    int64_t sweeps;           /* full sweeps (c phases) launched */
    int32_t segments;         /* M used */
    int32_t phases;           /* c used */
    int32_t resyncs;          /* exact re-synchronisations performed after the loop settled
                                 (including the final refresh that decides the status) */
    int32_t converged;        /* 1 if a sweep applied no update and the exact check on the
                                 refreshed state found every |Delta Z| below tol */
    double objective;         /* E(Z) in FP64 from the explicit residual */
    double max_drift;         /* max |beta_float32 - beta_exact| seen at a resync */
    /* The optimality report of the returned Z: beta recomputed from Z with
     * double-float accumulation (about 48 bits) from D~*X and rounded once to
     * float32; the gaps below are then evaluated in float32. */
    double kkt_zero_excess;   /* max over Z == 0 of |beta| - lambda (floored at 0) */
    double kkt_nonzero_gap;   /* max over Z != 0 of |Z - Sh(beta,lambda)/n| */
    double max_delta_z;       /* max over all coordinates of |Z - Sh(beta,lambda)/n| */
    double solve_ms;          /* device time from the first phase to the last resync */
    double phase_ms;          /* summed duration of the phase launches (time_kernels = 1) */
    int64_t phase_launches;   /* phase-kernel launches issued */
    int64_t visits;           /* segment visits that applied at least one update */
    int64_t kernel_launches;  /* all kernels this call launched */
    int64_t drift_resyncs;    /* resyncs that interrupted a CD round still running after
                                 32 sweeps (float32 drift on strongly coupled atoms);
                                 they do not count towards max_resyncs */
    double resync_ms;         /* summed device time of the resyncs (nonzero lists + resync
                                 kernel; time_kernels = 1, else 0) */
    double objective_ms;      /* device time of the final objective (time_kernels = 1) */
} csc_stats;

/* Fill *o with the defaults (all zero / -1 as documented above). */
void csc_default_opts(csc_opts *o);

/*
 * Step a1 (constants of Sec. 4 "computations for constants"; S of Eq. beta_up).
 * Creates a handle (if *h == NULL) or re-uses *h, copies D, and computes
 * DtD[K][K][2L-1] and the atom norms ||D_k||^2 (Eq. pb_coord) on the GPU.
 *   D       [K][P][L] float32, host or device, caller-owned, read only
 *   K,P,L   K >= 1, P >= 1, 1 <= L <= 512
 *   opts    NULL for defaults
 *   stream  cudaStream_t (NULL = legacy default stream)
 * Re-using a handle invalidates any previous csc_init.
 */
int csc_setup(csc_handle_t *h, const float *D, int K, int P, int L, const csc_opts *opts,
              void *stream);

/*
 * Step a2 (Alg. 1 initialisation; Alg. 2/3 "initialize beta and Z").
 * Copies X, sets Z = Z0 (or 0) and computes beta = D~ * X (FP32 with
 * compensated summation) and, for a warm start, subtracts the contribution of
 * Z0 in FP64.  Also records lambda_max = max |D~ * X|.
 *   X       [P][T] float32, host or device, caller-owned; T >= L and
 *           K*(T-L+1) < 2^32 - 1 (flat coordinate indices are 32-bit)
 *   lambda  > 0, absolute (not scaled)
 *   Z0      NULL (cold start) or [K][T-L+1] float32 warm start
 * The call does not wait for its kernels (X and Z0 may be reused once it
 * returns): lambda_max, the beta0 kernel's time and its status are read back
 * by the first call that needs them (csc_lambda_max, csc_lambda_max_batch,
 * csc_init_time, csc_solve, csc_objective, csc_kkt, csc_get_beta,
 * csc_autotune), which returns CSC_ETIMEOUT if the tensor-core kernel's
 * bounded wait gave up (the handle then needs a new csc_init).
 */
int csc_init(csc_handle_t h, const float *X, int64_t T, double lambda, const float *Z0);

/*
 * Steps a3-a7: phase-scheduled locally greedy CD until a full sweep applies
 * no update with |Delta Z| >= tol, then an exact resync of beta (double-float
 * accumulation, see max_resyncs) and a final FP64 objective and optimality
 * report.  The solver keeps r = beta - ||D_k||^2 Z in float32; a coordinate
 * counts as converged when its change computed in float32 is below
 * max(tol, 2^-21 |r| / ||D_k||^2 + 2^-22 |Z|): smaller changes are under the
 * resolution of the float32 state (a few ulps of r/n and of Z) and chasing
 * them only accumulates rounding drift.
 *   tol          > 0 (the paper's epsilon)
 *   max_updates  > 0, cap on applied updates (checked between phases)
 *   Z_out        NULL or [K][T-L+1] float32, host or device, caller-owned
 *   objective    NULL or receives E(Z) (FP64)
 *   stats        NULL or receives csc_stats
 * Returns CSC_OK, CSC_NOT_CONVERGED, or an error.  May be called again to
 * continue from the current Z.
 */
int csc_solve(csc_handle_t h, double tol, int64_t max_updates, float *Z_out, double *objective,
              csc_stats *stats);

/*
 * A batch of n independent problems sharing the atoms of csc_setup: signal i
 * is X_i [P][T[i]] with its own lambda[i].  The signals are concatenated in
 * time, X [P][sum T] (row p holds X_0[p], X_1[p], ... back to back), and so
 * is Z: [K][sum T - L + 1], where the columns of signal i are
 * [a_i, a_i + T[i] - L + 1) with a_i = T[0] + ... + T[i-1].  The L-1 columns
 * after each signal's last valid one straddle two signals; they are kept at 0
 * and belong to no problem (a warm start must hold 0 there).  Each signal is
 * cut into its own segments (Sec. 2.2), so one solve runs the segments of all
 * signals in the same phases and stops when every signal has converged; the
 * result of each signal is that of solving it alone (Eq. sparse_code).
 *   X       host or device, caller-owned; T[i] >= L; sum T - L + 1 < 2^31 - 1
 *   T       [n] host array;  n >= 1
 *   lambda  [n] host array, each > 0 and finite
 *   Z0      NULL or the concatenated warm start
 * csc_init(h, X, T, lambda, Z0) is csc_init_batch with n = 1.
 */
int csc_init_batch(csc_handle_t h, const float *X, const int64_t *T, int n, const double *lambda,
                   const float *Z0);

/* Replaces the lambdas of the current batch ([n] host array, each > 0) and
 * keeps Z and beta: the next csc_solve continues from the current Z (a warm
 * start along a regularisation path). */
int csc_set_lambda(csc_handle_t h, const double *lambda);

/* lambda_max of every signal of the current batch into out[n] (host). */
int csc_lambda_max_batch(csc_handle_t h, double *out);

/* E_i(Z) of every signal (host out[n]) from the last csc_solve or
 * csc_objective; csc_solve's objective is their sum. */
int csc_get_objectives(csc_handle_t h, double *out);

typedef struct csc_tune_result {
    int32_t segment_width;     /* chosen width (columns) */
    int32_t updates_per_visit; /* chosen u (0 = until local convergence) */
    int32_t phases;            /* c of the chosen plan */
    int32_t candidates;        /* solves timed */
    double best_ms;            /* csc_stats.solve_ms of the choice */
    double default_ms;         /* the same for width 2L-2 at the starting u (-1 if not run) */
    int32_t threads_per_segment; /* chosen threads per segment (32 or 128) */
} csc_tune_result;

/*
 * Autotuner (a deployment tool; the paper has no counterpart, its Thm. speedup
 * only predicts that narrower segments help until the phase count grows).
 * Solves the current problem (csc_init / csc_init_batch) to tol once per
 * candidate and keeps the fastest by device solve time: first the segment
 * width among L-1, 2L-2, 3L-3, 4L-4, 6L-6 (which sets the number of phases c)
 * at the handle's updates_per_visit (24 if 0), then updates_per_visit among
 * 8, 24, 64 and 0 at that width, then (where both forms apply) one warp or a
 * block of threads per segment (csc_opts.threads_per_segment).  Every
 * candidate starts from the state the problem had when csc_autotune was
 * called, and that state is restored afterwards; the choice is stored in the
 * handle's options (segments = 0, segment_width, updates_per_visit,
 * threads_per_segment) for the following solves and, when out is not NULL,
 * reported.  Tune on a representative problem of the (K, L, P) at
 * hand and re-use the result through csc_opts for others.
 */
int csc_autotune(csc_handle_t h, double tol, int64_t max_updates, csc_tune_result *out);

/* Releases every device and host resource of the handle.  NULL is accepted. */
int csc_destroy(csc_handle_t h);

/* max_{k,t} |(D~_k * X)[t]| of the last csc_init: Z* = 0 iff lambda >= this
 * (for a batch, the largest over its signals). */
int csc_lambda_max(csc_handle_t h, double *out);

/* Copies the current beta [K][Tz] (float32) to host or device memory. */
int csc_get_beta(csc_handle_t h, float *beta_out);

/* Copies DtD [K][K][2L-1] (layout above) and the norms [K] (either may be NULL). */
int csc_get_dtd(csc_handle_t h, float *dtd_out, float *norms_out);

/* FP64 objective E(Z) of Eq. sparse_code for the handle's X and lambda and an
 * arbitrary Z [K][Tz] (host or device); for a batch, the sum over its signals
 * (each one then available from csc_get_objectives). */
int csc_objective(csc_handle_t h, const float *Z, double *out);

/*
 * Optimality report of an arbitrary Z [K][Tz] (host or device, the layout of
 * csc_solve's Z_out) for the handle's X and lambda, by coordinate-wise
 * optimality (Theorem A.1): with beta = D~ * (X - sum_l Z_l * D_l) + ||D_k||^2 Z_k
 * recomputed from Z (double-float accumulation from the stored D~ * X,
 * rounded once to float32),
 *   out[0] = max over Z_k[t] == 0 of |beta_k[t]| - lambda   (floored at 0)
 *   out[1] = max over Z_k[t] != 0 of |Z_k[t] - Sh(beta_k[t], lambda)/||D_k||^2|
 *   out[2] = max over all coordinates of the same gap (max |Delta Z|)
 * out: three doubles, host memory; for a batch, the maxima over its signals.
 * The handle's state (beta, Z, flags) is not changed.
 */
int csc_kkt(csc_handle_t h, const float *Z, double *out);

/*
 * Per-phase trace of the last csc_solve: for phase launch g (0-based, in
 * launch order) the updates it applied, the objective decrease it achieved
 * (sum of Prop. A.1 cost variations, FP64) and the device time in ns of the
 * end of its last thread block, relative to the start of the solve.  The
 * objective before the solve is *E_start.  Arrays hold cap entries; *n
 * receives the number of phases recorded (may exceed cap).
 */
int csc_get_trace(csc_handle_t h, int64_t cap, int64_t *updates, double *decrease,
                  int64_t *t_ns, int64_t *n, double *E_start);

/*
 * Host-only planning (no GPU): the segment schedule for Tz samples, atoms of
 * length L and M segments (Sec. 2.2, 0-based): segment m is
 * [floor(m*Tz/M), floor((m+1)*Tz/M)); *phases receives c, the number of
 * phases such that co-active segments' update windows never overlap.
 * starts may be NULL or hold M+1 entries.  M == 0 picks the automatic M.
 * Returns CSC_EINVAL if M > Tz or sizes are not positive.
 */
int csc_plan(int64_t Tz, int L, int M, int *M_out, int *phases, int64_t *starts);

/*
 * E(Z) of Eq. sparse_code in FP64, like csc_objective, for callers that must
 * not allocate device memory: code running under a fixed device-memory budget
 * (e.g. a serving loop that admits requests by HBM budget and cannot grow it
 * mid-request) or latency-critical code that cannot take the implicit device
 * synchronisation of cudaMalloc/cudaFree.  The paper has no counterpart; this
 * is a deployment interface.  It needs no handle and calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *   D [K][P][L], X [P][T], Z [K][T-L+1]  float32 DEVICE arrays, caller-owned
 *   lambda >= 0;  E_out: one double, host or device memory
 *   stream  cudaStream_t (NULL = legacy default stream)
 * D, X and Z must be memory of the current device (or managed memory); a
 * device E_out likewise.  The binding checks that X is [P][T] and Z is
 * [K][T-L+1]; this entry point cannot, so wrong sizes read out of bounds.
 * Scratch: a static device array of 1 MiB that every GPU loading this library
 * keeps until process exit; it limits T to 16,777,216 samples (larger T gives
 * CSC_EINVAL).  Each call looks up that array's address on the current device
 * (cudaGetSymbolAddress); the first call on a device also loads the module
 * there, so make that first call before any stream capture.  All calls share
 * the array: calls whose GPU work may overlap (other streams, other threads)
 * race and must be ordered by the caller.  With a host E_out the call
 * synchronises the stream.
 */
int csc_objective_noalloc(const float *D, int K, int P, int L, const float *X, int64_t T,
                          const float *Z, double lambda, double *E_out, void *stream);

/*
 * Failure detection check.  Every device-side wait of this library (the
 * tensor-core beta0 kernel's mbarrier waits) is a bounded poll: when it gives
 * up, the kernel sets an error flag, stops issuing work, waits (bounded) for
 * the work already issued, releases tensor memory and returns, and the call
 * returns CSC_ETIMEOUT with the device still usable.  This entry runs that
 * wait in a one-warp kernel on an mbarrier that nothing arrives at, limited to
 * `polls` polls (1 .. 2^22), on the current device and the legacy default
 * stream (synchronous).  Expected result: CSC_ETIMEOUT (the wait gave up and
 * the kernel returned).  CSC_OK would mean the barrier completed; CSC_EINVAL
 * for polls out of range; CSC_ECUDA / CSC_ENOMEM on a CUDA error.
 */
int csc_check_wait_timeout(int64_t polls);

/* Device time in ms of the beta0 kernel (D~ * X) of the last csc_init,
 * measured with a CUDA event pair on the handle's stream when the handle's
 * opts.time_kernels is 1; -1 otherwise. */
int csc_init_time(csc_handle_t h, double *beta0_ms);

/* Number of kernels launched through this handle since it was created. */
int csc_kernel_launches(csc_handle_t h, int64_t *out);

/* Text of the last error on the calling thread ("" if none). */
const char *csc_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* CSC_H */
