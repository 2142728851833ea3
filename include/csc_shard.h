/*
 * csc_shard.h - one signal solved by several processes (one GPU each).
 *
 * DICOD (Sec. 2.2, Alg. 2 of Moreau, Oudre & Vayatis, ICML 2018) cuts the
 * activation axis into M segments and gives each of W workers a contiguous
 * run of them; a worker that updates a coordinate within L-1 of its border
 * sends the update to the neighbour, which applies Eq. beta_up to its own
 * columns.  Here a worker is a process with its own handle (its own GPU):
 * rank q of W owns the segments [q M / W, (q+1) M / W) of the single-process
 * cut (csc_plan), and the segments of the whole signal still run in the c
 * phases of the single-process schedule (segment m in phase m mod c,
 * whichever rank owns it).  A rank holds its own columns plus up to L-1
 * columns on each side (its halo); during a phase the updates of its
 * segments change r on the halo too, and those changes are exactly what the
 * neighbour must add to its own columns.  The caller moves them between
 * phases:
 *
 *   for each phase p:  csc_shard_phase(p)            (stream-ordered)
 *                      csc_shard_halo_out(to_left, to_right)
 *                      send to_left to rank q-1 and to_right to rank q+1,
 *                      receive from_left from q-1 and from_right from q+1
 *                      csc_shard_halo_in(from_left, from_right)
 *   after each sweep (c phases): sum csc_shard_updates over ranks; a sweep in
 *                      which no rank applied an update ends the CD round
 *   end of a round:    exchange csc_shard_z_out / csc_shard_z_in the same way,
 *                      csc_shard_resync on every rank, max of its result over
 *                      ranks: below tol = converged, else the next round
 *   objective:         sum of csc_shard_objective over ranks (Eq. sparse_code)
 *
 * Because co-active segments' update windows never overlap, the changes a
 * rank receives after a phase fall in its segments that were idle in it: the
 * result is the single-process solve's, up to the order of float additions
 * at the borders.  The exchanged blocks are [K][L-1] float32 (the halo widths
 * of neighbouring ranks are equal), row-major; buffers may be host or device
 * memory of the handle's device.  Ranks at the ends of the signal have no
 * halo on their outer side (width 0, buffer may be NULL).
 *
 * Errors as in csc.h.  csc_solve refuses a handle that holds a shard.
 */
#ifndef CSC_SHARD_H
#define CSC_SHARD_H

#include <stdint.h>

#include "csc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct csc_shard_plan {
    int64_t T, Tz;                  /* the whole signal: samples, columns T - L + 1 */
    int32_t L, M, phases;           /* atom length, segments of the whole signal, c */
    int32_t world, rank;
    int32_t seg_first, seg_count;   /* this rank's segments */
    int64_t col_first, col_count;   /* the columns they cover (owned) */
    int64_t halo_left, halo_right;  /* columns held beyond them, min(L-1, to the signal's end) */
    int64_t x_first, x_count;       /* samples of X the rank holds:
                                       [col_first - halo_left,
                                        col_first + col_count + halo_right + L - 1) */
} csc_shard_plan;

/* Host only.  The plan of rank `rank` of `world` for a signal of T samples,
 * atoms of length L and M segments (0 = automatic: width 2L-2, as csc_plan).
 * CSC_EINVAL unless world <= M <= Tz and every rank owns at least L-1
 * columns (so that each halo lies in one neighbour). */
int csc_shard_plan_make(int64_t T, int L, int M, int world, int rank, csc_shard_plan *plan);

/* csc_init on the rank's samples X [P][plan->x_count] (host or device,
 * caller-owned) with Z = 0, then the shard's segments and phase lists; the
 * halo columns of r start at 0.  plan must be csc_shard_plan_make's, with the
 * handle's L.  lambda > 0 is absolute (the same on every rank). */
int csc_shard_init(csc_handle_t h, const csc_shard_plan *plan, const float *X, double lambda);

/* Phase p (0 <= p < plan->phases) of the global schedule on this rank's
 * segments: each segment that needs a visit applies up to u updates
 * (opts.updates_per_visit) with |Delta Z| >= tol (the float32 resolution
 * floor of csc_solve applies).  Enqueued on the handle's stream. */
int csc_shard_phase(csc_handle_t h, int p, double tol);

/* The changes of r accumulated in the halo since the last call, to_left
 * [K][halo_left] and to_right [K][halo_right]; the halo is reset to 0. */
int csc_shard_halo_out(csc_handle_t h, float *to_left, float *to_right);

/* Adds the neighbours' changes to this rank's own border columns:
 * from_left [K][halo_left] to columns [col_first, col_first + halo_left),
 * from_right [K][halo_right] to the last halo_right owned columns; the
 * segments that receive a nonzero change need a visit again. */
int csc_shard_halo_in(csc_handle_t h, const float *from_left, const float *from_right);

/* Z of the owned columns within halo_left of the left border (to_left) and
 * within halo_right of the right border (to_right), [K][width] each. */
int csc_shard_z_out(csc_handle_t h, float *to_left, float *to_right);

/* Sets the halo's Z from the neighbours' csc_shard_z_out blocks. */
int csc_shard_z_in(csc_handle_t h, const float *from_left, const float *from_right);

/* Updates applied by this rank since csc_shard_init (synchronises). */
int csc_shard_updates(csc_handle_t h, int64_t *total);

/* Exact resync of r on the owned columns (double-float accumulation from
 * D~ * X; needs the halo's Z current) and *max_dz = the largest change a
 * coordinate step would make on the refreshed state (with the float32
 * floor).  Every owned segment needs a visit again afterwards. */
int csc_shard_resync(csc_handle_t h, double tol, double *max_dz);

/* This rank's part of E(Z) in FP64: 1/2 the squared residual over the
 * samples [col_first, col_first + col_count) (the last rank also
 * [Tz, T)) plus lambda times the l1 norm of its own columns; needs the halo's
 * Z current.  E(Z) is the sum over ranks. */
int csc_shard_objective(csc_handle_t h, double *out);

/* Z of the owned columns, [K][col_count] (host or device). */
int csc_shard_get_z(csc_handle_t h, float *Z_out);

#ifdef __cplusplus
}
#endif

#endif /* CSC_SHARD_H */
