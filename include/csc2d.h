/*
 * csc2d.h - the 2-D variant: convolutional sparse coding of images, with the
 * image cut into row bands and, on the GPU, each band into column blocks.
 *
 * The paper's conclusion names cutting images along one direction as the way
 * to carry DICOD over to images while each worker keeps two neighbours.
 * Every definition is that of Sec. 2.1 with 2-D lags: image X[P][H][W],
 * atoms D[K][P][h][w], activations Z[K][Hz][Wz] with Hz = H-h+1, Wz = W-w+1
 * ("valid" placement: activation (i, j) covers rows i..i+h-1 and columns
 * j..j+w-1), and the problem
 *     Z* = argmin_Z 1/2 || X - sum_k Z_k * D_k ||^2 + lambda sum_k ||Z_k||_1
 * (Eq. sparse_code).  Row band m of M covers the activation rows
 * [floor(m Hz / M), floor((m+1) Hz / M)); column block n of N covers the
 * columns [floor(n Wz / N), floor((n+1) Wz / N)).  With cr phases over rows
 * and cc over columns (csc2d_plan on each axis), tile (m, n) runs in phase
 * (m mod cr) cc + (n mod cc): co-active tiles' update windows ((2h-1) x
 * (2w-1) positions around an update) never meet.  N = 1 is the paper's cut
 * along one axis (bands only).  Ties of the argmax go to the lowest flat
 * index (k Hz + i) Wz + j.
 *
 * Errors as in csc.h.  Layouts row-major, float32.
 */
#ifndef CSC2D_H
#define CSC2D_H

#include <stdint.h>

#include "csc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct csc2d_stats {
    int64_t updates;         /* applied coordinate updates */
    int64_t sweeps;          /* sweeps of the c phases */
    int32_t bands;           /* M used (row bands) */
    int32_t col_blocks;      /* N used (column blocks) */
    int32_t phases;          /* cr x cc used */
    int32_t resyncs;         /* exact re-synchronisations of beta after a settled round */
    int32_t converged;       /* 1 if a sweep applied no update and the exact check found
                                every |Delta Z| below tol */
    int32_t reserved;
    double objective;        /* E(Z), FP64 from the explicit residual */
    double max_delta_z;      /* max over all coordinates of |Z - Sh(beta, lambda)/n| after
                                the last exact refresh */
    double solve_ms;         /* device time from the setup kernels to the last refresh */
    int64_t kernel_launches; /* kernels this call launched (sweeps go in batches of four per
                                read-back; those after the settling sweep launch blocks that
                                return at once) */
} csc2d_stats;

/* Host only: the cut of one axis, Hz activation rows (or columns), atoms of
 * height h (or width w) and M bands (0 = automatic: bands of 2h-2 rows);
 * *phases receives the phase count of that axis, 1 + ceil((2h-2) / narrowest
 * band) (at most M); starts (may be NULL) receives M+1 starts.  CSC_EINVAL
 * if M > Hz. */
int csc2d_plan(int64_t Hz, int h, int M, int *M_out, int *phases, int64_t *starts);

/*
 * Tile-scheduled locally greedy CD (Alg. 3 on the tiles, the phases above)
 * from Z = 0 to |Delta Z| < tol, with up to 3 exact re-synchronisations of
 * beta (FP64 sums from beta0 = D~ * X) that decide convergence, then the FP64
 * objective.  The state is float32 (the same numerics as csc_solve: the
 * float32 resolution floor applies).  The call allocates its device memory
 * on the current device and frees it before returning.
 *   D [K][P][h][w], X [P][H][W]: host or device, caller-owned
 *   1 <= K <= 64, P <= 64, K (2h-1) <= 2048, (2h-1)(2w-1) <= 4096; a tile's
 *   positions times 20 bytes must fit shared memory (about 226 KB; its r and
 *   Z are staged there too when 8 (K|1) bytes more per position fit): use
 *   more bands or column blocks for large tiles
 *   lambda > 0 (absolute), tol > 0, max_updates >= 1
 *   M: row bands, 0 = automatic (2h-2 rows each)
 *   N: column blocks, 0 = automatic (2w-2 columns each), 1 = bands only
 *   updates_per_visit: cap on updates per tile visit; 0 = automatic (8)
 *   Z_out: NULL or [K][Hz][Wz], host or device
 *   stream: cudaStream_t (NULL = legacy default stream); synchronised
 * Returns CSC_OK, CSC_NOT_CONVERGED (max_updates, or the exact check still
 * failed after the last resync) or an error.
 */
int csc2d_solve(const float *D, int K, int P, int h, int w, const float *X, int64_t H,
                int64_t W, double lambda, double tol, int64_t max_updates, int M, int N,
                int updates_per_visit, float *Z_out, double *objective, csc2d_stats *stats,
                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CSC2D_H */
