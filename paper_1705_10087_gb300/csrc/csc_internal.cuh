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
constexpr int kMaxSmem = 226 * 1024;     // dynamic shared memory per block (227 KB on sm_103a, less static)

// Segment m of M over [0,Tz) (Sec. 2.2, 0-based): [floor(m*Tz/M), floor((m+1)*Tz/M)).
__host__ __device__ __forceinline__ int64_t seg_start(int64_t Tz, int M, int64_t m)
{
    return m * Tz / M;
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

// Smallest |Z' - Z| that the FP32 state resolves at a coordinate: Z' is
// Sh(beta)/n computed from a float beta, so changes under about four ulps of
// beta (2^-21 |beta| / n) are rounding noise.  Coordinates below it count as
// converged (max(tol, floor) is the effective stopping threshold).
__device__ __forceinline__ float resolution_floor(float beta, float n)
{
    return fabsf(beta) * 4.76837158203125e-07f / n;
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

// Parameters of one phase launch (see kernel_phase.cu).
struct PhaseParams {
    float *beta;               // [K][Tz]
    float *Z;                  // [K][Tz]
    const float *C;            // DtD [K][K][W2]
    const float *norms;        // [K]
    unsigned char *dirty;      // [M] segment needs a visit
    long long *upd;            // [kPhaseRing] updates per phase launch
    double *dec;               // [kPhaseRing] objective decrease per phase launch
    unsigned long long *tend;  // [kPhaseRing] globaltimer at the end of the launch
    long long *total;          // updates applied in this solve
    long long *visits;         // segment visits that applied updates
    int *done;                 // set once a full sweep applied nothing
    int64_t Tz;
    long long max_updates;
    int M, c, p, K, L;
    int g;        // launch index (monotone within a solve)
    int g_round;  // first launch index of the current CD round
    int u;        // cap on updates per visit
    float lam, tol;
    int wt_max, w_max;  // tile extents used for the shared-memory layout
};

struct PhaseConfig {
    int block;
    size_t smem;
    bool tile_in_smem;
};

PhaseConfig phase_config(int K, int L, int64_t Tz, int M);
cudaError_t launch_phase(const PhaseParams &pp, const PhaseConfig &cfg, cudaStream_t s);

cudaError_t launch_dtd(const float *D, int K, int P, int L, float *C, float *norms,
                       cudaStream_t s);
cudaError_t launch_dtx(const float *D, const float *X, int K, int P, int L, int64_t T,
                       float *beta0, unsigned int *absmax_bits, cudaStream_t s);

// FP64 re-synchronisation: beta = fp32(beta0 - sum_{(l,t')!=(k,t)} S Z) and the
// optimality report.  red[0..4] receive (as non-negative double bit patterns
// for atomicMax): drift, zero_excess, nonzero_gap, max_delta_z (FP64), and
// max |Delta Z| computed in FP32 from the rounded beta.
cudaError_t launch_resync(const float *beta0, float *beta, const float *Z, const float *C,
                          const float *norms, int K, int L, int64_t Tz, double lam,
                          float lam_f, int write_beta, unsigned long long *red, cudaStream_t s);

// FP64 objective E(Z) (Eq. sparse_code) into *out, via per-block partials.
int objective_blocks(int64_t T);
cudaError_t launch_objective(const float *D, const float *X, const float *Z, int K, int P, int L,
                             int64_t T, double lam, double *partials, double *out,
                             cudaStream_t s);

cudaError_t launch_stamp(unsigned long long *out, cudaStream_t s);

}  // namespace csc
