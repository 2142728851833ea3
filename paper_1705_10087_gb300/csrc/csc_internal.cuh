// Internal declarations of the GB300 CSC solver (not part of the C ABI).
//
// Array layouts follow include/csc.h.  Notation: K atoms of P channels and
// length L, Tz = T - L + 1 activations per atom, W2 = 2L - 1 lags.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "csc.h"

namespace csc {

constexpr int kMaxL = 512;
constexpr int kPhaseRing = 1 << 16;      // per-phase trace slots (ring)
constexpr int kDefaultMaxVisit = 1 << 20;  // cap on updates per segment visit
// A CD round that has not settled after this many sweeps is interrupted by a
// resync: on strongly coupled atoms float32 rounding in the incremental
// updates of r can otherwise keep driving updates that the exact r would not
// make (a cycle that never lowers E).
constexpr int kDriftSweeps = 32;
constexpr int kMaxSmem = 226 * 1024;     // dynamic shared memory per block (227 KB on sm_103a, less static)

// Segment m of M over [0,Tz) (Sec. 2.2, 0-based): [floor(m*Tz/M), floor((m+1)*Tz/M)).
__host__ __device__ __forceinline__ int64_t seg_start(int64_t Tz, int M, int64_t m)
{
    return m * Tz / M;
}

// The segment holding column t under that cut: the m with
// seg_start(m) <= t < seg_start(m+1), m = floor(((t+1) M - 1) / Tz).
__host__ __device__ __forceinline__ int segment_of(int64_t Tz, int M, int64_t t)
{
    return (int)(((t + 1) * (int64_t)M - 1) / Tz);
}

// Soft thresholding Sh(u, lam) = sign(u) max(|u| - lam, 0) (Sec. 2.1).
__device__ __forceinline__ float soft_f(float u, float lam)
{
    float a = fabsf(u) - lam;
    return a > 0.f ? copysignf(a, u) : 0.f;
}
__device__ __forceinline__ double soft_d(double u, double lam)
{
    double a = fabs(u) - lam;
    return a > 0.0 ? copysign(a, u) : 0.0;
}

// The solver keeps, instead of beta, r = beta - ||D_k||^2 Z: the correlation
// of each atom with the full residual X - sum Z*D (the beta of Sec. 2.1 with
// the coordinate's own term kept).  At the optimum |r| <= lambda everywhere,
// so r is small exactly where beta is large (active atoms) and its float32
// rounding is up to |beta|/lambda times finer.  Eq. beta_up becomes
// r_k[t] -= S_{k,k0}[t-t0] dZ for every (k,t), own coordinate included.
//
// coord_step: the coordinate optimum of Eq. pb_coord for one coordinate held
// as (r, z): Z' = Sh(r + n z, lambda) / n.  While Z' keeps the sign of z the
// change is Z' - z = (r - lambda sign z) / n, evaluated without forming
// r + n z (no cancellation).  Returns the change actually representable,
// fl(z + d) - z, in *delta and the new value in *znew; the change is reported
// as 0 when it is below the float32 resolution of the pair (about four ulps
// of r/n plus two ulps of z), where updates are rounding noise.
__device__ __forceinline__ void coord_step(float r, float z, float n, float rn, float lam,
                                           float *znew, float *delta)
{
    float d;
    if (z == 0.f) {
        d = soft_f(r, lam) * rn;
    } else {
        const float s = z > 0.f ? 1.f : -1.f;
        const float b = fmaf(n, z, r);
        d = b * s > lam ? (r - lam * s) * rn : soft_f(b, lam) * rn - z;
    }
    const float zn = z + d;
    const float dd = zn - z;
    const float floor_ = fabsf(r) * 4.76837158203125e-07f * rn + fabsf(z) * 2.384185791015625e-07f;
    if (fabsf(dd) < floor_) {
        *znew = z;
        *delta = 0.f;
    } else {
        *znew = zn;
        *delta = dd;
    }
}

// Double-float accumulation (hi + lo, about 48 significant bits) of products
// of floats, with error-free transformations: the rounding error of a*b is
// fma(a, b, -p) (exact), that of hi + p is Knuth's TwoSum.  The _rn
// intrinsics keep the compiler from contracting or reassociating them.  This
// runs on the FP32 pipes, which GB300 has about 64 times more of than FP64.
__device__ __forceinline__ void df_add_prod(float &hi, float &lo, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bv = __fsub_rn(s, hi);
    const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(se, pe));
}

// (hi, lo) += a, a float (TwoSum; the rounding error is carried in lo)
__device__ __forceinline__ void df_add(float &hi, float &lo, float a)
{
    const float s = __fadd_rn(hi, a);
    const float bv = __fsub_rn(s, hi);
    const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(a, bv));
    hi = s;
    lo = __fadd_rn(lo, se);
}

// (hi, lo) += (bh, bl), both double-float
__device__ __forceinline__ void df_add_df(float &hi, float &lo, float bh, float bl)
{
    df_add(hi, lo, bh);
    lo = __fadd_rn(lo, bl);
}

// (sh, sl) += (x - (ah + al))^2 in double-float: the residual with TwoSum,
// its square as rh^2 (exact error by fma) + 2 rh rl (rl^2 is below the
// pair's precision)
__device__ __forceinline__ void df_add_sq_residual(float &sh, float &sl, float x, float ah,
                                                   float al)
{
    float rh = x, rl = 0.f;
    df_add(rh, rl, -ah);
    df_add(rh, rl, -al);
    const float p = __fmul_rn(rh, rh);
    const float q = __fmaf_rn(__fmul_rn(2.f, rh), rl, __fmaf_rn(rh, rh, -p));
    df_add(sh, sl, p);
    sl = __fadd_rn(sl, q);
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Compensated FP32 accumulator (Kahan 1965): short FMA partial sums are
// added with their rounding error carried in c.  Explicit _rn intrinsics keep
// the compiler from contracting or reassociating the compensation.
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        float y = __fsub_rn(x, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ float value() const { return __fsub_rn(s, c); }
};

// One problem of a batch: its own activation arrays, row-major [K][ld] (atom
// k's row at r + k * ld), valid columns [0, Tz), samples X [P][ldx] with
// T = Tz + L - 1 of them, and its segments [seg0, seg0 + nseg) of the plan.
// The arrays of different problems never overlap, so every kernel is a set of
// independent per-problem computations.  A batch handle points the entries
// into one concatenation (ld = the concatenation's width); a server points
// them into separate allocations (ld = Tz).
struct SigDesc {
    float *r;            // r = beta - ||D_k||^2 Z
    float *Z;
    const float *beta0;  // D~ * X
    const float *X;
    int64_t ld, ldx, Tz;
    int seg0, nseg;
    float lam;
    float tol;  // CD stopping threshold of the problem (|Delta Z| below it: converged)
    double lam_d;
};

// Parameters of one phase launch (see kernel_phase.cu).
struct PhaseParams {
    const SigDesc *sig;        // problems of the batch
    const int *seg_sig;        // [M] problem of each segment
    const float *C;            // DtD [K][K][W2]
    const float *Ct;           // DtD by lag, float4 groups of atoms:
                               // Ct[((k0 * Kp/4 + k/4) * W2 + s) * 4 + k%4] = DtD[k0][k][s], 0 for k >= K
    const float *norms;        // [K]
    unsigned char *dirty;      // [M] segment needs a visit
    unsigned char *touched;    // [M] r changed in the segment since the last resync
    const int64_t *seg_s;      // [M] first column of each segment (in its problem)
    const int64_t *seg_e;      // [M] one past its last column
    const int *phase_list;     // segments of this phase (grid = their count)
    long long *upd;            // [kPhaseRing] updates per phase launch
    double *dec;               // [kPhaseRing] objective decrease per phase launch
    unsigned long long *tend;  // [kPhaseRing] globaltimer at the end of the launch
    long long *total;          // updates applied in this solve
    long long *visits;         // segment visits that applied updates
    int *done;                 // set once a full sweep applied nothing
    long long max_updates;
    int M, c, p, K, Kp, L;  // Kp = K rounded up to a multiple of 4
    int g;        // launch index (monotone within a solve); with g_dev, offset from *g_dev
    int g_round;  // first launch index of the current CD round (or *g_round_dev)
    const int *g_dev;        // NULL, or the launch index of the first launch of a graph replay
    const int *g_round_dev;  // NULL, or the first launch index of the round
    int u;        // cap on updates per visit
    int w_max;  // widest segment (shared-memory layout)
    // queue of the phase's segments that need a visit (drain launches):
    // qhead[0] = next entry to take, qhead[1] = queue length
    int *qhead;
    const int *qlen;
    int *queue;
};

struct PhaseConfig {
    int block;
    size_t smem;
    bool tile_in_smem;
};

// w_max: widest segment of the plan; threads_per_segment: 32 = one warp per
// segment where eligible (K = 25, 2L-1 <= 128, the tile fits shared memory),
// otherwise (and for 0) a block of 128, 512 or 1024 threads.
PhaseConfig phase_config(int K, int L, int w_max, int threads_per_segment);
bool phase_warp_eligible(int K, int L, int w_max);
// active = number of segments in pp.phase_list (the grid size).
cudaError_t launch_phase(const PhaseParams &pp, const PhaseConfig &cfg, int active,
                         cudaStream_t s);
// The last node of a poll batch in the graph of a CD round (a while loop over
// batches): gctr[0] += batch (the launch index of the next launch), then the
// loop's condition is set to go on unless the round's sweep found nothing to
// do (*done), the update budget is spent (*total >= lim[0]), the round reached
// lim[1] > 0 launches (a drift resync is due), the solve reached lim[2]
// launches (max_sweeps) or the next batch would pass lim[3] (the trace ring).
cudaError_t launch_round_step(cudaGraphConditionalHandle cond, int *gctr, int batch,
                              const int *done, const long long *total, const long long *lim,
                              cudaStream_t s);
// Start of a CD round: *done = 0, gctr[1] = g_round and the stopping rules
// lim = {max_updates, drift_launches, max_g, ring} tested by launch_round_step.
cudaError_t launch_round_begin(int *done, int *gctr, int g_round, long long *lim,
                               long long max_updates, long long drift_launches, long long max_g,
                               long long ring, cudaStream_t s);
// Start of a solve: zero[0 .. nwords) = 0, dirty[0 .. M) = touched[0 .. M) = 1
// and *tstart = the global timer, in one launch.
cudaError_t launch_solve_begin(unsigned long long *zero, int64_t nwords, unsigned char *dirty,
                               unsigned char *touched, int64_t M, unsigned long long *tstart,
                               cudaStream_t s);
// Blocks of the phase kernel that are resident at once on the whole GPU.
int phase_resident_blocks(const PhaseConfig &cfg, int K);
// The same phase as launch_phase, for phase lists much longer than the
// resident blocks: the segments of pp.phase_list[0..active) that need a visit
// are compacted into pp.queue and min(resident, active) persistent blocks
// drain it (three stream operations: reset, compaction, drain).
cudaError_t launch_phase_drain(const PhaseParams &pp, const PhaseConfig &cfg, int active,
                               int resident, cudaStream_t s);

cudaError_t launch_dtd(const float *D, int K, int P, int L, float *C, float *norms,
                       cudaStream_t s);
// Ct[((k0 * Kp/4 + q) * W2 + s) * 4 + e] = C[(k0 * K + 4 q + e) * W2 + s] (zero for
// 4 q + e >= K): the K coefficients an update of atom k0 applies at lag s are
// Kp/4 float4 words, one per group q, and consecutive lags' words are adjacent.
__host__ __device__ __forceinline__ int coef_pad(int K) { return (K + 3) & ~3; }
cudaError_t launch_coef_by_lag(const float *C, int K, int L, float *Ct, cudaStream_t s);

// beta0 = D~ * X, max |beta0| into *absmax_bits, and sum X^2 added to *x2sum
// (so E(0) = x2sum / 2).  r_out != NULL receives a second copy of beta0 (the
// state r of a cold start, Z = 0).
// Tile table of a batch: tile i of the problems belongs to signal sig[i] =
// the last j with off[j] <= i (off[n] = count, every signal has a tile) and
// starts at column (i - off[sig[i]]) * width of that signal.
cudaError_t launch_expand_tiles(const int64_t *off, int n, int width, int64_t count,
                                int64_t *start, int *sig, cudaStream_t s);

cudaError_t launch_dtx(const float *D, const float *X, int K, int P, int L, int64_t T,
                       float *beta0, float *r_out, unsigned int *absmax_bits, double *x2sum,
                       cudaStream_t s);

// Reduction / output tiles of a batch: tile b covers columns (or samples)
// [start[b], start[b] + width) of problem sig[b], clipped to the problem and,
// when end != NULL, to end[b] (a shard computes only the columns it owns; the
// columns beyond end[b] are still read as neighbours).
struct Tiles {
    const int *sig;
    const int64_t *start;
    int64_t n;
    const int64_t *end = nullptr;
};
constexpr int kResyncCols = 32;  // columns per resync tile
constexpr int kTile = 256;       // samples per objective tile, columns per absmax tile

// beta0 = D~ * X on the tensor cores (kernel_dtx_tc.cu): mode 1 = three-term
// BF16 split of X and D with six FP32-accumulated products (FP32-grade),
// mode 2 = one BF16 product.  Needs K <= 64 and dtx_tc_smem(K,P,L) <= kMaxSmem
// (cudaErrorNotSupported otherwise).  *err is set when a bounded wait gave up.
size_t dtx_tc_smem(int K, int P, int L);
// The beta0 kernel used by default: the tensor cores (mode 1) wherever one
// CTA fits on an SM, else the FP32 kernel.
inline bool dtx_tc_preferred(int K, int P, int L)
{
    return K <= 64 && dtx_tc_smem(K, P, L) <= (size_t)kMaxSmem;
}
// What the tensor-core beta0 kernel can do besides beta0 and r, in the same
// pass: z_out != NULL zeroes Z [K][Tz] (a cold start); lmax != NULL gathers the
// maximum |beta0| of each of the nsig problems of a batch (float bits, zeroed
// by the caller), problem i owning the columns [a[i], a[i+1] - L + 1).  done
// is set when the kernel that ran did both (the FP32 kernel does neither).
struct Dtx0Extras {
    float *z_out = nullptr;
    const int64_t *a = nullptr;  // [nsig + 1] first sample of each problem (device)
    int nsig = 0;
    unsigned int *lmax = nullptr;  // [nsig]
    bool done = false;
};
// beta0 with init_mode 0 (automatic), 1 or 2 (tensor cores), 3 (FP32 kernel).
cudaError_t launch_dtx_any(const float *D, const float *X, int K, int P, int L, int64_t T,
                           int init_mode, float *beta0, float *r_out, unsigned int *absmax_bits,
                           double *x2sum, int *err, cudaStream_t s, Dtx0Extras *ex = nullptr);
// One warp waits, bounded by `limit` polls, on an mbarrier nothing arrives
// at, and sets *gave_up when the wait gives up.
cudaError_t launch_wait_selftest(unsigned limit, int *gave_up, cudaStream_t s);
cudaError_t launch_dtx_tc(const float *D, const float *X, int K, int P, int L, int64_t T,
                          int mode, float *beta0, float *r_out, unsigned int *absmax_bits,
                          double *x2sum, int *err, cudaStream_t s, Dtx0Extras *ex = nullptr);

// Nonzeros of Z per resync tile ("bucket": the tile's kResyncCols columns),
// rebuilt at each resync where Z may have changed.  Bucket b holds
// min(count[b], kNzCap) entries ent[b * kNzCap + i] = (k * kResyncCols + j,
// bits of Z_k[start + j]) in (k, j) order; count[b] > kNzCap means the bucket
// overflowed and a tile that needs it scans Z itself.
constexpr int kNzCap = 64;
struct NzLists {
    int *count;  // [tiles]
    uint2 *ent;  // [tiles * kNzCap]
};

// Re-synchronisation of r with its definition, r = D~*X - sum_{l,t'} S Z
// (beta0 = D~*X), accumulated in double-float and rounded once to float, and
// the optimality report over the valid columns of every problem (tiles of
// kResyncCols columns).  red[0..4] receive (as non-negative double bit
// patterns for atomicMax): the drift max |r_old - r_new|, zero_excess,
// nonzero_gap, max_delta_z, and the largest coord_step change on the float
// state; with red_stride > 0, problem i reduces into red[i * red_stride + q]
// instead.  With dirty != NULL, also marks dirty[m] = 1 for every segment m
// (the problem's segments are the equal cut of seg_start, found with
// segment_of) that holds a coordinate whose coord_step change on the new state
// is >= tol_mark (tol_mark < 0: the problem's own tol).
// With touched != NULL (per segment: r changed there since r was last exact)
// a tile whose columns meet no touched segment is not recomputed: its r is
// already exact, and its report values are the ones stored in rep[5 b..5 b+4]
// when it was last computed (every computed tile stores them when rep != NULL).
// With lists.count != NULL the nonzeros of Z are first listed per tile (a
// tile's bucket is rebuilt unless touched says its Z did not change since the
// previous resync over the same tiles) and each tile reads the lists of the
// tiles within L-1 columns instead of scanning Z; the tiles of a problem must
// be consecutive in the table and in column order (both tables are).
// Ct: the by-lag table of PhaseParams::Ct (float4 groups of atoms).
cudaError_t launch_resync(const SigDesc *sig, Tiles tiles, const float *Ct, const float *norms,
                          int K, int L, int write_r, unsigned long long *red, int red_stride,
                          unsigned char *dirty, float tol_mark, const unsigned char *touched,
                          float *rep, NzLists lists, cudaStream_t s);

// out = r + n Z (beta of Sec. 2.1) in float, over one [K][ld] array.
cudaError_t launch_beta_from_r(const float *r, const float *Z, const float *norms, int K,
                               int64_t Tz, float *out, cudaStream_t s);

// FP64 objective E_i(Z) (Eq. sparse_code) of every problem into out[i] (tiles
// of kTile samples, partials[2b..2b+1] for tile b; tile_off[i] = first tile of
// problem i, n+1 entries).  Zalt != NULL replaces each problem's Z by
// Zalt + (its Z - Zbase) (same layout, another array).  lists: the nonzero
// buckets of the last resync, valid only if Z has not changed since (its
// tiles start at rtile_off[i] for problem i); {NULL, NULL} lists Z here.
cudaError_t launch_objective(const float *D, const SigDesc *sig, int n, Tiles tiles,
                             const int64_t *tile_off, int K, int P, int L, const float *Zbase,
                             const float *Zalt, double *partials, double *out, cudaStream_t s,
                             NzLists lists = NzLists{nullptr, nullptr},
                             const int64_t *rtile_off = nullptr);

// The same for one problem described on the host, with no tables: consecutive
// tiles, partials holds 2 * ceil(T / kTile) doubles; out[0] = E.
cudaError_t launch_objective_single(const float *D, const SigDesc &one, int K, int P, int L,
                                    double *partials, double *out, cudaStream_t s);

// max |beta0| over the valid columns of each problem (tiles of kTile columns;
// out: float bits, zeroed by the caller).
cudaError_t launch_signal_absmax(const SigDesc *sig, Tiles tiles, int K, unsigned int *out,
                                 cudaStream_t s);


}  // namespace csc
