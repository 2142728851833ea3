// Setup kernels: the atom cross-correlation table DtD with the norms (step a1)
// and the initial beta = D~ * X with lambda_max (step a2).
//
// Both are dense contractions accumulated in FP32 with compensated summation:
// FMA partial sums over 8 consecutive lags, added into a Kahan accumulator, so
// that the rounding error stays at the level of the final rounding (well below
// the 1e-6 support threshold the solver is checked at).
#include "csc_internal.cuh"

namespace csc {

namespace {

// DtD[k0][k][s] = sum_p sum_tau D[k][p][tau] * D[k0][p][tau + s - (L-1)]
// = S_{k,k0}[s-(L-1)] of Eq. beta_up (Sec. 2.1).  One block per pair (k0, k),
// one thread per lag; with STAGE the two atoms are first copied to shared
// memory (every thread of the block reads all of both).
template <bool STAGE>
__global__ void dtd_kernel(const float *__restrict__ D, int K, int P, int L,
                           float *__restrict__ C, float *__restrict__ norms)
{
    extern __shared__ float dsm[];  // STAGE: [2][P][L], atom k then atom k0
    const int W2 = 2 * L - 1;
    const int k0 = blockIdx.x / K, k = blockIdx.x % K;
    const int PL = P * L;
    const float *da = D + (long long)k * PL, *db = D + (long long)k0 * PL;
    if (STAGE) {
        for (int i = threadIdx.x; i < PL; i += blockDim.x) {
            dsm[i] = __ldg(da + i);
            dsm[PL + i] = __ldg(db + i);
        }
        __syncthreads();
        da = dsm;
        db = dsm + PL;
    }
    for (int s = threadIdx.x; s < W2; s += blockDim.x) {
        const int lag = s - (L - 1);
        const int tlo = lag < 0 ? -lag : 0;
        const int thi = lag > 0 ? L - lag : L;
        KahanF acc;
        for (int p = 0; p < P; p++) {
            const float *a = da + p * L;
            const float *b = db + p * L + lag;
            for (int t8 = tlo; t8 < thi; t8 += 8) {
                // (unrolled with predicates: the loads of a chunk issue together)
                float part = 0.f;
#pragma unroll
                for (int u = 0; u < 8; u++)
                    if (t8 + u < thi)
                        part = fmaf(a[t8 + u], b[t8 + u], part);
                acc.add(part);
            }
        }
        const float v = acc.value();
        C[((long long)k0 * K + k) * W2 + s] = v;
        if (k == k0 && lag == 0)
            norms[k] = v;
    }
}

constexpr int kDtxThreads = 256;
constexpr int kDtxT = 4;                            // consecutive outputs per thread
constexpr int kDtxTile = kDtxThreads * kDtxT;       // output samples per block
constexpr int kDtxAtoms = 8;                        // atoms per block

// beta0[k][t] = sum_p sum_tau D[k][p][tau] X[p][t+tau] (Alg. 1 initialisation),
// plus max |beta0| (lambda_max) and sum X^2 (2 E(0)).  Block: 1024 consecutive
// t and 8 atoms; a thread owns 4 consecutive t, so each 8-lag step reads 12
// samples of X (3 vector loads) and the 8 atoms' 8 lags (broadcast vector
// loads) for 256 FMAs.  Lags are padded to a multiple of 8 with zeros.
__global__ void __launch_bounds__(kDtxThreads) dtx_kernel(const float *__restrict__ D,
                                                         const float *__restrict__ X, int K,
                                                         int P, int L, long long T,
                                                         float *__restrict__ beta0,
                                                         float *__restrict__ r_out,
                                                         unsigned int *__restrict__ absmax_bits,
                                                         double *__restrict__ x2sum)
{
    extern __shared__ __align__(16) float sm[];
    const int L8 = (L + 7) & ~7;
    const int xw = kDtxTile + L8 + 4;  // X tile width, multiple of 4
    float *xs = sm;                     // [P][xw]
    float *ds = sm + (size_t)P * xw;    // [kDtxAtoms][P][L8]
    const long long Tz = T - L + 1;
    const long long t0 = (long long)blockIdx.x * kDtxTile;
    const int k0 = blockIdx.y * kDtxAtoms;
    const int nk = min(kDtxAtoms, K - k0);

    double x2 = 0.0;
    const bool last = t0 + kDtxTile >= Tz;  // the last block also owns samples [Tz, T)
    for (int i = threadIdx.x; i < P * xw; i += blockDim.x) {
        const int p = i / xw, j = i % xw;
        const long long t = t0 + j;
        const float v = t < T ? X[(long long)p * T + t] : 0.f;
        xs[i] = v;
        if (blockIdx.y == 0 && (j < kDtxTile || last))
            x2 += (double)v * (double)v;
    }
    for (int i = threadIdx.x; i < kDtxAtoms * P * L8; i += blockDim.x) {
        const int kk = i / (P * L8), r = i % (P * L8), p = r / L8, tau = r % L8;
        ds[i] = (kk < nk && tau < L) ? D[((long long)(k0 + kk) * P + p) * L + tau] : 0.f;
    }
    __syncthreads();

    const int j4 = threadIdx.x * kDtxT;
    KahanF acc[kDtxAtoms][kDtxT];
    for (int p = 0; p < P; p++) {
        const float *xr = xs + (size_t)p * xw + j4;
        for (int tb = 0; tb < L8; tb += 8) {
            float x[12];
            const float4 a0 = *reinterpret_cast<const float4 *>(xr + tb);
            const float4 a1 = *reinterpret_cast<const float4 *>(xr + tb + 4);
            const float4 a2 = *reinterpret_cast<const float4 *>(xr + tb + 8);
            x[0] = a0.x; x[1] = a0.y; x[2] = a0.z; x[3] = a0.w;
            x[4] = a1.x; x[5] = a1.y; x[6] = a1.z; x[7] = a1.w;
            x[8] = a2.x; x[9] = a2.y; x[10] = a2.z; x[11] = a2.w;
#pragma unroll
            for (int kk = 0; kk < kDtxAtoms; kk++) {
                const float4 *dv = reinterpret_cast<const float4 *>(ds + ((size_t)kk * P + p) * L8 + tb);
                const float4 d0 = dv[0], d1 = dv[1];
#pragma unroll
                for (int q = 0; q < kDtxT; q++) {
                    float part = d0.x * x[q];
                    part = fmaf(d0.y, x[q + 1], part);
                    part = fmaf(d0.z, x[q + 2], part);
                    part = fmaf(d0.w, x[q + 3], part);
                    part = fmaf(d1.x, x[q + 4], part);
                    part = fmaf(d1.y, x[q + 5], part);
                    part = fmaf(d1.z, x[q + 6], part);
                    part = fmaf(d1.w, x[q + 7], part);
                    acc[kk][q].add(part);
                }
            }
        }
    }
    float amax = 0.f;
#pragma unroll
    for (int q = 0; q < kDtxT; q++) {
        const long long t = t0 + j4 + q;
        if (t < Tz) {
#pragma unroll
            for (int kk = 0; kk < kDtxAtoms; kk++) {
                if (kk < nk) {
                    const float v = acc[kk][q].value();
                    beta0[(long long)(k0 + kk) * Tz + t] = v;
                    if (r_out)
                        r_out[(long long)(k0 + kk) * Tz + t] = v;
                    amax = fmaxf(amax, fabsf(v));
                }
            }
        }
    }
    // block max of |beta0| -> one atomic per warp (non-negative floats order as uints)
    for (int off = 16; off > 0; off >>= 1) {
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
        x2 += __shfl_xor_sync(0xffffffffu, x2, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(absmax_bits, __float_as_uint(amax));
        if (blockIdx.y == 0)
            atomicAdd(x2sum, x2);
    }
}

// Ct[((k0 * Kp/4 + q) * W2 + s) * 4 + e] = C[k0][k = 4 q + e][s] (0 for k >= K):
// for one updated atom k0 and lag s the K coefficients are Kp/4 float4 words,
// and the words of consecutive lags are adjacent (coalesced across threads).
__global__ void coef_by_lag_kernel(const float *__restrict__ C, int K, int L, int Kp,
                                   float *__restrict__ Ct)
{
    const int W2 = 2 * L - 1, KQ = Kp / 4;
    const long long n = (long long)K * W2 * Kp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(i & 3);
        const long long rest = i >> 2;  // (k0 * KQ + q) * W2 + s
        const int s = (int)(rest % W2);
        const long long kq = rest / W2;
        const int q = (int)(kq % KQ), k0 = (int)(kq / KQ);
        const int k = 4 * q + e;
        Ct[i] = k < K ? C[((long long)k0 * K + k) * W2 + s] : 0.f;
    }
}

}  // namespace

cudaError_t launch_dtd(const float *D, int K, int P, int L, float *C, float *norms,
                       cudaStream_t s)
{
    const int W2 = 2 * L - 1;
    const int block = W2 <= 128 ? 128 : (W2 <= 256 ? 256 : 512);
    const size_t smem = 2 * sizeof(float) * (size_t)P * L;
    if (smem <= 48 * 1024)
        dtd_kernel<true><<<(unsigned)(K * K), block, smem, s>>>(D, K, P, L, C, norms);
    else
        dtd_kernel<false><<<(unsigned)(K * K), block, 0, s>>>(D, K, P, L, C, norms);
    return cudaGetLastError();
}

namespace {

// one thread per tile: binary search of its signal in off[0..n]
__global__ void expand_tiles_kernel(const int64_t *__restrict__ off, int n, int width,
                                    int64_t count, int64_t *__restrict__ start,
                                    int *__restrict__ sig)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n;  // off[lo] <= i < off[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= i)
                lo = mid;
            else
                hi = mid;
        }
        start[i] = (i - off[lo]) * width;
        sig[i] = lo;
    }
}

}  // namespace

cudaError_t launch_expand_tiles(const int64_t *off, int n, int width, int64_t count,
                                int64_t *start, int *sig, cudaStream_t s)
{
    if (count <= 0)
        return cudaSuccess;
    const int64_t blocks = (count + 255) / 256;
    expand_tiles_kernel<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(off, n, width,
                                                                                 count, start, sig);
    return cudaGetLastError();
}

cudaError_t launch_dtx(const float *D, const float *X, int K, int P, int L, int64_t T,
                       float *beta0, float *r_out, unsigned int *absmax_bits, double *x2sum,
                       cudaStream_t s)
{
    const int L8 = (L + 7) & ~7;
    const size_t smem =
        sizeof(float) * ((size_t)P * (kDtxTile + L8 + 4) + (size_t)kDtxAtoms * P * L8);
    if (smem > (size_t)kMaxSmem)
        return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(dtx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    const int64_t Tz = T - L + 1;
    dim3 grid((unsigned)((Tz + kDtxTile - 1) / kDtxTile), (unsigned)((K + kDtxAtoms - 1) / kDtxAtoms));
    dtx_kernel<<<grid, kDtxThreads, smem, s>>>(D, X, K, P, L, T, beta0, r_out, absmax_bits,
                                               x2sum);
    return cudaGetLastError();
}

cudaError_t launch_coef_by_lag(const float *C, int K, int L, float *Ct, cudaStream_t s)
{
    const long long n = (long long)K * (2 * L - 1) * coef_pad(K);
    const long long grid = (n + 255) / 256;
    coef_by_lag_kernel<<<(unsigned)(grid < 65535 ? grid : 65535), 256, 0, s>>>(C, K, L,
                                                                            coef_pad(K), Ct);
    return cudaGetLastError();
}

}  // namespace csc
