// The hot path: one phase of segmented, locally greedy coordinate descent.
//
// DICOD (Alg. 2) runs M workers, each greedy on its own segment C_m and
// sending (k0, t0, Delta Z) to its neighbours when an update lands within L
// of the border (Sec. 2.2, Fig. DCP).  Here a thread block is a worker: in
// phase p the blocks own the segments m == p (mod c) and every other segment
// is idle.  c is such that the beta windows [s_m-L+1, e_m+L-1) of co-active
// segments never meet, so a block may write Eq. beta_up straight into the
// idle neighbours' beta (the paper's message) and every phase equals a
// sequential run of its segments (Alg. 3 restricted to one phase).
//
// Per visit a block
//   1. loads beta on its window and Z on its segment into shared memory
//      (or works on global memory when the tile does not fit),
//   2. keeps, per owned column t, the best coordinate over k of
//      |Delta Z_k[t]| = |Z_k[t] - Sh(beta_k[t], lambda)/||D_k||^2| (Eq. pb_coord)
//      as a 64-bit key (|Delta Z| bits << 32 | ~(k*Tz + t)): the max key is
//      the largest |Delta Z| with ties to the lowest flat index,
//   3. repeats: block argmax (warp shuffle max, one barrier), stop if the
//      best |Delta Z| < tol (Alg. 1 stopping rule) or after u updates,
//      else Z_k0[t0] <- Z' and beta_k[t] -= S_{k,k0}[t-t0] (Z' - Z_old) on
//      the window (Eq. beta_up with the sign fixed by the beta definition),
//      re-evaluating only the columns of the window,
//   4. writes the tile back, marks the neighbours it spilled into as dirty
//      and adds its count and its objective decrease (Prop. A.1) to the
//      per-launch trace.
// A segment that ended its last visit converged and was not spilled into
// since is clean and is skipped: beta and Z on it have not changed.
#include "csc_internal.cuh"

namespace csc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
    unsigned hi = (unsigned)(v >> 32);
    const unsigned hmax = __reduce_max_sync(kFull, hi);
    unsigned lo = hi == hmax ? (unsigned)v : 0u;
    const unsigned lmax = __reduce_max_sync(kFull, lo);
    return ((unsigned long long)hmax << 32) | lmax;
}

template <bool SMEM>
__global__ void __launch_bounds__(1024) phase_kernel(PhaseParams pp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];

    // ---- early exits, decided by one thread so the block stays uniform ----
    // (total is being incremented by other blocks of this launch)
    __shared__ int s_go;
    const int m = pp.p + pp.c * (int)blockIdx.x;  // < M by the grid size
    if (threadIdx.x == 0) {
        int go = 1;
        if (*(volatile int *)pp.done) {
            go = 0;
        } else if (*(volatile long long *)pp.total >= pp.max_updates) {
            go = 0;  // out of budget: not a converged sweep, so done stays unset
        } else if (pp.g - pp.g_round >= pp.c) {
            // a full sweep (the previous c launches of this round) applied nothing
            long long s = 0;
            for (int j = pp.g - pp.c; j < pp.g; j++)
                s += *(volatile long long *)&pp.upd[j & (kPhaseRing - 1)];
            if (s == 0) {
                if (blockIdx.x == 0)
                    *(volatile int *)pp.done = pp.g + 1;
                go = 0;
            }
        }
        if (go && !*(volatile unsigned char *)&pp.dirty[m])
            go = 0;
        s_go = go;
    }
    __syncthreads();
    if (!s_go)
        return;

    const int K = pp.K, L = pp.L, W2 = 2 * L - 1;
    const int64_t Tz = pp.Tz;
    const int64_t s = seg_start(Tz, pp.M, m), e = seg_start(Tz, pp.M, m + 1);
    const int w = (int)(e - s);
    const int64_t ts = s - (L - 1) > 0 ? s - (L - 1) : 0;
    const int64_t te = e + (L - 1) < Tz ? e + (L - 1) : Tz;
    const int Wt = (int)(te - ts);
    const int j0 = (int)(s - ts);  // tile column of the segment's first sample
    const int tid = threadIdx.x, B = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = B >> 5;

    // ---- shared-memory layout ------------------------------------------
    unsigned char *ptr = smem_raw;
    unsigned long long *ckey = reinterpret_cast<unsigned long long *>(ptr);
    ptr += sizeof(unsigned long long) * pp.wt_max;
    unsigned long long *wkey = reinterpret_cast<unsigned long long *>(ptr);  // [2][32]
    ptr += sizeof(unsigned long long) * 64;
    float *cz = reinterpret_cast<float *>(ptr);
    ptr += sizeof(float) * pp.wt_max;
    float *cd = reinterpret_cast<float *>(ptr);
    ptr += sizeof(float) * pp.wt_max;
    float *wz = reinterpret_cast<float *>(ptr);  // [2][32]
    ptr += sizeof(float) * 64;
    float *wd = reinterpret_cast<float *>(ptr);  // [2][32]
    ptr += sizeof(float) * 64;
    float *nrm = reinterpret_cast<float *>(ptr);  // [K]
    ptr += sizeof(float) * ((K + 3) & ~3);

    float *bb;  // beta on the window: bb[k * bstride + j], j tile column
    float *zb;  // Z on the segment:   zb[k * zstride + j - j0]
    int64_t bstride, zstride;
    if (SMEM) {
        bb = reinterpret_cast<float *>(ptr);
        zb = bb + (size_t)K * pp.wt_max;
        bstride = pp.wt_max;
        zstride = pp.w_max;
        for (int k = 0; k < K; k++) {
            const float *src = pp.beta + (int64_t)k * Tz + ts;
            for (int j = tid; j < Wt; j += B)
                bb[(int64_t)k * bstride + j] = src[j];
            const float *zsrc = pp.Z + (int64_t)k * Tz + s;
            for (int j = tid; j < w; j += B)
                zb[(int64_t)k * zstride + j] = zsrc[j];
        }
    } else {
        bb = pp.beta + ts;
        zb = pp.Z + s;
        bstride = Tz;
        zstride = Tz;
    }
    for (int k = tid; k < K; k += B)
        nrm[k] = pp.norms[k];
    __syncthreads();

    const float lam = pp.lam, tol = pp.tol;

    // best coordinate of tile column j (owned segment column) over k
    auto col_eval = [&](int j) {
        const int jj = j - j0;
        float best = -1.f, bz = 0.f, bdz = 0.f;
        int bk = 0;
        for (int k = 0; k < K; k++) {
            const float b = bb[(int64_t)k * bstride + j];
            const float z = zb[(int64_t)k * zstride + jj];
            const float zp = __fdiv_rn(soft_f(b, lam), nrm[k]);
            const float d = zp - z;
            // below the FP32 resolution of Z' (a few ulps of beta) the change is
            // rounding noise, not descent: count the coordinate as converged
            const float ad = fabsf(d) >= resolution_floor(b, nrm[k]) ? fabsf(d) : 0.f;
            if (ad > best) {
                best = ad;
                bk = k;
                bz = zp;
                bdz = d;
            }
        }
        const unsigned flat = (unsigned)((int64_t)bk * Tz + (ts + j));
        ckey[j] = ((unsigned long long)__float_as_uint(best) << 32) | (unsigned)(~flat);
        cz[j] = bz;
        cd[j] = bdz;
    };

    for (int j = tid; j < Wt; j += B) {
        if (j >= j0 && j < j0 + w)
            col_eval(j);
        else
            ckey[j] = 0ull;
    }
    // (no barrier needed: each thread reads back only its own columns)

    int buf = 0, nupd = 0;
    double decrease = 0.0;
    int64_t tmin = Tz, tmax = -1;
    bool capped = false;
    for (int it = 0;; it++) {
        // ---- block argmax of the cached column keys ----------------------
        unsigned long long my = 0ull;
        float mz = 0.f, md = 0.f;
        for (int j = tid; j < Wt; j += B) {
            const unsigned long long kk = ckey[j];
            if (kk > my) {
                my = kk;
                mz = cz[j];
                md = cd[j];
            }
        }
        const unsigned long long wm = warp_max_u64(my);
        const int src = __ffs(__ballot_sync(kFull, my == wm)) - 1;
        const float wzv = __shfl_sync(kFull, mz, src), wdv = __shfl_sync(kFull, md, src);
        if (lane == 0) {
            wkey[buf * 32 + warp] = wm;
            wz[buf * 32 + warp] = wzv;
            wd[buf * 32 + warp] = wdv;
        }
        __syncthreads();
        unsigned long long bk = 0ull;
        float znew = 0.f, delta = 0.f;
        for (int i = 0; i < nwarps; i++) {
            const unsigned long long kk = wkey[buf * 32 + i];
            if (kk > bk) {
                bk = kk;
                znew = wz[buf * 32 + i];
                delta = wd[buf * 32 + i];
            }
        }
        const float adz = __uint_as_float((unsigned)(bk >> 32));
        if (!(adz >= tol))
            break;
        if (it >= pp.u) {
            capped = true;
            break;
        }
        const unsigned flat = ~(unsigned)(bk & 0xffffffffu);
        const int k0 = (int)(flat / (uint64_t)Tz);
        const int64_t t0 = (int64_t)flat - (int64_t)k0 * Tz;

        if (tid == 0) {
            // Prop. A.1: E(Z) - E(Z') = n/2 (z^2 - u^2) - beta (z - u) + lam (|z| - |u|)
            const double n = nrm[k0], u = znew, z = (double)znew - (double)delta;
            const double b = bb[(int64_t)k0 * bstride + (t0 - ts)];
            decrease += 0.5 * n * (z * z - u * u) - b * (z - u) + (double)lam * (fabs(z) - fabs(u));
        }

        // ---- Eq. beta_up on the window, re-evaluate its columns ---------
        const float *Ck0 = pp.C + (int64_t)k0 * K * W2;
        const int64_t wlo = t0 - (L - 1) > ts ? t0 - (L - 1) : ts;
        const int64_t whi = t0 + (L - 1) < te - 1 ? t0 + (L - 1) : te - 1;
        for (int j = tid; j < Wt; j += B) {
            const int64_t t = ts + j;
            if (t < wlo || t > whi)
                continue;
            const int sidx = (int)(t - t0) + (L - 1);
            for (int k = 0; k < K; k++) {
                if (k == k0 && t == t0)
                    continue;
                float *bp = bb + (int64_t)k * bstride + j;
                *bp = *bp - __ldg(Ck0 + (int64_t)k * W2 + sidx) * delta;
            }
            if (t == t0)
                zb[(int64_t)k0 * zstride + (j - j0)] = znew;
            if (j >= j0 && j < j0 + w)
                col_eval(j);
        }
        nupd++;
        tmin = t0 < tmin ? t0 : tmin;
        tmax = t0 > tmax ? t0 : tmax;
        buf ^= 1;
    }

    // ---- write back, spill bookkeeping, trace ---------------------------
    if (SMEM && nupd > 0) {
        for (int k = 0; k < K; k++) {
            float *dst = pp.beta + (int64_t)k * Tz + ts;
            for (int j = tid; j < Wt; j += B)
                dst[j] = bb[(int64_t)k * bstride + j];
            float *zdst = pp.Z + (int64_t)k * Tz + s;
            for (int j = tid; j < w; j += B)
                zdst[j] = zb[(int64_t)k * zstride + j];
        }
    }
    if (tid == 0) {
        pp.dirty[m] = capped ? 1 : 0;
        if (nupd > 0) {
            // neighbours whose beta changed: segments meeting [tmin-L+1, tmax+L-1]
            const int64_t lo = tmin - (L - 1), hi = tmax + (L - 1);
            for (int mm = m - 1; mm >= 0 && seg_start(Tz, pp.M, mm + 1) > lo; mm--)
                pp.dirty[mm] = 1;
            for (int mm = m + 1; mm < pp.M && seg_start(Tz, pp.M, mm) <= hi; mm++)
                pp.dirty[mm] = 1;
            const int slot = pp.g & (kPhaseRing - 1);
            atomicAdd(reinterpret_cast<unsigned long long *>(&pp.upd[slot]), (unsigned long long)nupd);
            atomicAdd(reinterpret_cast<unsigned long long *>(pp.total), (unsigned long long)nupd);
            atomicAdd(reinterpret_cast<unsigned long long *>(pp.visits), 1ull);
            atomicAdd(&pp.dec[slot], decrease);
            atomicMax(&pp.tend[slot], globaltimer_ns());
        }
    }
}

size_t smem_bytes(int K, int wt_max, int w_max, bool tile)
{
    size_t b = sizeof(unsigned long long) * ((size_t)wt_max + 64) +
               sizeof(float) * (2 * (size_t)wt_max + 128 + (((size_t)K + 3) & ~(size_t)3));
    if (tile)
        b += sizeof(float) * (size_t)K * ((size_t)wt_max + w_max);
    return b;
}

}  // namespace

PhaseConfig phase_config(int K, int L, int64_t Tz, int M)
{
    const int64_t wmax = (Tz + M - 1) / M;  // widest segment
    int64_t wtmax = wmax + 2 * (int64_t)(L - 1);
    if (wtmax > Tz)
        wtmax = Tz;
    PhaseConfig cfg;
    cfg.tile_in_smem = smem_bytes(K, (int)wtmax, (int)wmax, true) <= (size_t)kMaxSmem;
    cfg.smem = smem_bytes(K, (int)wtmax, (int)wmax, cfg.tile_in_smem);
    int b = (int)((wtmax + 31) / 32 * 32);
    cfg.block = b < 1024 ? (b < 64 ? 64 : b) : 1024;
    return cfg;
}

cudaError_t launch_phase(const PhaseParams &pp, const PhaseConfig &cfg, cudaStream_t s)
{
    const int active = pp.p < pp.M ? (pp.M - 1 - pp.p) / pp.c + 1 : 0;
    if (active == 0)
        return cudaSuccess;
    if (cfg.smem > (size_t)kMaxSmem)
        return cudaErrorInvalidConfiguration;
    if (cfg.tile_in_smem) {
        cudaError_t e = cudaFuncSetAttribute(phase_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)cfg.smem);
        if (e != cudaSuccess)
            return e;
        phase_kernel<true><<<active, cfg.block, cfg.smem, s>>>(pp);
    } else {
        cudaError_t e = cudaFuncSetAttribute(phase_kernel<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)cfg.smem);
        if (e != cudaSuccess)
            return e;
        phase_kernel<false><<<active, cfg.block, cfg.smem, s>>>(pp);
    }
    return cudaGetLastError();
}

}  // namespace csc
