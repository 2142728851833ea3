// The hot path: one phase of segmented, locally greedy coordinate descent.
//
// DICOD (Alg. 2) runs M workers, each greedy on its own segment C_m and
// sending (k0, t0, Delta Z) to its neighbours when an update lands within L
// of the border (Sec. 2.2, Fig. DCP).  Here a thread block is a worker: in
// phase p the blocks own the segments m == p (mod c) and every other segment
// is idle.  c is such that the windows [s_m-L+1, e_m+L-1) of co-active
// segments never meet, so a block may apply Eq. beta_up straight to the idle
// neighbours' state (the paper's message, here a fire-and-forget reduction
// into their r in global memory) and every phase equals a sequential run of
// its segments (Alg. 3 restricted to one phase).
//
// State: r = beta - ||D_k||^2 Z and Z (see coord_step in csc_internal.cuh).
// Per visit a block
//   1. loads r and Z of its own segment into shared memory (or works on
//      global memory when the segment does not fit),
//   2. keeps, per owned column t, the best coordinate over k of
//      |Delta Z_k[t]| = |Sh(beta_k[t], lambda)/||D_k||^2 - Z_k[t]| (Eq. pb_coord,
//      evaluated from r by coord_step) as a 64-bit key
//      (|Delta Z| bits << 32 | ~(k << 17 | (t - s) << 1 | sign of Delta Z)):
//      the max key is the largest |Delta Z| with ties to the lowest (k, t),
//      i.e. the lowest k*Tz + t,
//   3. repeats: block argmax (warp max, a shared atomicMax per warp, one
//      barrier; the key names the winner and its Delta Z), stop if the best
//      |Delta Z| < tol (Alg. 1 stopping rule) or after u updates, else
//      Z_k0[t0] <- Z' and r_k[t] -= S_{k,k0}[t-t0] (Z' - Z_old) for every k
//      and t in [t0-L+1, t0+L-1] (Eq. beta_up, sign fixed by the beta
//      definition, written for r); own columns are updated in shared memory
//      and re-evaluated, the others (idle neighbours) by atomicAdd,
//   4. writes its segment's r back (each new Z value went to global memory
//      when it was applied), marks the neighbours it spilled into as
//      dirty and adds its count and objective decrease (Prop. A.1) to the
//      per-launch trace.
// Thread i owns the segment columns jj == i (mod blockDim) and handles, in an
// update, the window column t with (t - s) == i (mod blockDim); blockDim >=
// 2L-1, so the 2L-1 window columns go to distinct threads and each own
// column is only ever touched by its owner.
// A segment that ended its last visit converged and was not spilled into
// since is clean and is skipped: r and Z on it have not changed.
#include <algorithm>
#include <type_traits>

#include "csc_internal.cuh"

namespace csc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kCoefBatch = 16;         // DtD coefficients loaded per round trip (multiple of 4)

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
    unsigned hi = (unsigned)(v >> 32);
    const unsigned hmax = __reduce_max_sync(kFull, hi);
    unsigned lo = hi == hmax ? (unsigned)v : 0u;
    const unsigned lmax = __reduce_max_sync(kFull, lo);
    return ((unsigned long long)hmax << 32) | lmax;
}

// Column stride of the staged tiles for the compile-time-K kernels: a
// multiple of 4 floats (16-byte aligned columns, 128-bit accesses) whose
// quarter is odd, so that the 8 lanes of a 128-bit shared-memory phase, on
// consecutive columns, cover all 32 banks.
__host__ __device__ constexpr int vec_stride(int K)
{
    return (((K + 3) / 4) | 1) * 4;
}
// Whether phase_config picks a compile-time-K kernel (vector tile layout).
__host__ __device__ inline bool vec_layout(int K, int block)
{
    return (K == 25 || K == 64) && block <= 512;
}

// Shared-memory layout of a block, in bytes from the start (16-byte aligned
// pieces).  w = widest segment; with smem the segment's r and Z are staged.
struct Layout {
    size_t key, cz, cd, ck, zm, nrm, rnrm, r, z, total;
    __host__ __device__ Layout(int K, int w, bool smem, bool vec)
    {
        size_t o = 0;
        key = o;
        o = up(o + 8 * (size_t)w);
        cz = o;
        o = up(o + 4 * (size_t)w);
        cd = o;  // dZ and the best atom of a column (the one-warp form's winner read)
        o = up(o + 4 * (size_t)w);
        ck = o;
        o = up(o + 4 * (size_t)w);
        zm = o;  // per column: bit k set when Z_k[t] != 0 (compile-time K <= 64)
        o = up(o + 8 * (size_t)w);
        nrm = o;
        o = up(o + 4 * (size_t)K);
        rnrm = o;
        o = up(o + 4 * (size_t)K);
        // staged tiles are column-major [jj][k]: with an odd row length K|1 lanes on
        // consecutive columns hit distinct banks (scalar accesses); the
        // compile-time-K kernels use vec_stride(K) for 128-bit accesses
        const size_t ks = vec ? (size_t)vec_stride(K) : (size_t)(K | 1);
        r = o;
        if (smem)
            o = up(o + 4 * ks * w);
        z = o;
        if (smem)
            o = up(o + 4 * ks * w);
        total = o;
    }
    __host__ __device__ static size_t up(size_t x) { return (x + 15) & ~(size_t)15; }
};

// KT > 0 fixes K at compile time (loops over atoms unroll, tile offsets
// become immediates); KT = 0 reads K from the parameters.
// One visit of segment m by the whole block (uniform control flow: every
// early exit is decided by thread 0 and broadcast).
template <bool SMEM, int MAXT, int KT>
__device__ __forceinline__ void visit_segment(const PhaseParams &pp, const int m, const int g,
                                              const int g_round)
{
    using Idx = typename std::conditional<SMEM, int, int64_t>::type;
    constexpr bool KFIX = KT > 0;
    constexpr int KPC = (KT + 3) & ~3;  // padded coefficient row, compile-time K
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_go;
    __shared__ double s_dec[32];
    // the block's best key of update i is reduced into s_best[i & 3] (a 64-bit
    // shared atomicMax per warp); slot (i + 2) & 3, last read in update i - 2,
    // is cleared during update i
    __shared__ unsigned long long s_best[4];

    // ---- early exits, decided by one thread so the block stays uniform ----
    // (total is being incremented by other blocks of this launch)
    if (threadIdx.x == 0) {
        int go = 1;
        if (*(volatile int *)pp.done) {
            go = 0;
        } else if (*(volatile long long *)pp.total >= pp.max_updates) {
            go = 0;  // out of budget: not a converged sweep, so done stays unset
        } else if (g - g_round >= pp.c) {
            // a full sweep (the previous c launches of this round) applied nothing
            long long sum = 0;
            for (int j = g - pp.c; j < g; j++)
                sum += *(volatile long long *)&pp.upd[j & (kPhaseRing - 1)];
            if (sum == 0) {
                *(volatile int *)pp.done = g + 1;  // same value from every block
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

    const int K = KFIX ? KT : pp.K, L = pp.L, W2 = 2 * L - 1;
    const int Kp = KFIX ? KPC : pp.Kp;
    // the segment's problem: its arrays, row stride, width and lambda
    const SigDesc *sdp = pp.sig + pp.seg_sig[m];
    float *const gr = sdp->r;
    float *const gz = sdp->Z;
    const int64_t ld = sdp->ld, Tz = sdp->Tz;
    const int seg_lo = sdp->seg0, seg_hi = sdp->seg0 + sdp->nseg;
    const int64_t s = pp.seg_s[m], e = pp.seg_e[m];
    const int w = (int)(e - s);
    // blockDim == MAXT, a power of two >= 2L-1 (see phase_config)
    constexpr int B = MAXT;
    constexpr int nwarps = B >> 5;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float lam = sdp->lam, tol = sdp->tol;

    constexpr int CST = vec_stride(KT);  // column stride of the vector layout (KFIX)
    constexpr int KQ = (KT + 3) / 4;      // float4 groups holding the KT atoms
    const Layout lay(K, pp.w_max, SMEM, KFIX);
    unsigned long long *ckey = reinterpret_cast<unsigned long long *>(smem_raw + lay.key);
    float *cz = reinterpret_cast<float *>(smem_raw + lay.cz);  // Z' of a column's key
    // one bit per atom of a column: 32 or 64 bits
    using Mask = typename std::conditional<(KT > 32), unsigned long long, unsigned>::type;
    static_assert(KT <= 64, "the masks of a column hold 64 atoms");
    Mask *zmask = reinterpret_cast<Mask *>(smem_raw + lay.zm);
    float *nrm = reinterpret_cast<float *>(smem_raw + lay.nrm);    // ||D_k||^2
    float *rnrm = reinterpret_cast<float *>(smem_raw + lay.rnrm);  // 1 / ||D_k||^2

    // own segment: element (k, jj = t - s) at rs[jj * cst + k * kst]
    //   staged (SMEM): column-major [jj][k], cst = K|1, kst = 1
    //   in place:      the problem's [k][ld] arrays, cst = 1, kst = ld
    float *rs;
    float *zs;
    Idx cst, kst;
    if (SMEM) {
        rs = reinterpret_cast<float *>(smem_raw + lay.r);
        zs = reinterpret_cast<float *>(smem_raw + lay.z);
        cst = (Idx)(KFIX ? CST : (K | 1));
        kst = 1;
        if constexpr (!KFIX) {
            for (int k = 0; k < K; k++) {
                const float *rsrc = gr + (int64_t)k * ld + s;
                const float *zsrc = gz + (int64_t)k * ld + s;
                for (int jj = tid; jj < w; jj += B) {
                    rs[jj * cst + k] = rsrc[jj];
                    zs[jj * cst + k] = zsrc[jj];
                }
            }
        }
        // (compile-time K: each thread stages its own columns below)
    } else {
        rs = gr + s;
        zs = gz + s;
        cst = 1;
        kst = (Idx)ld;
    }
    for (int k = tid; k < K; k += B) {
        nrm[k] = pp.norms[k];
        rnrm[k] = __frcp_rn(pp.norms[k]);
    }
    if (tid < 4)
        s_best[tid] = 0ull;
    __syncthreads();

    // best coordinate of own column jj from its r values (registers) and the
    // mask of entries that can move: z != 0 or |r| > lam (all others have
    // Z' = Sh(r, lam)/n = 0 = z exactly); compile-time K only
    // Only the set bits of need are visited (their r, z and norms re-read from
    // shared memory): an unrolled, predicated loop over all K atoms would issue
    // every atom's instructions whether its bit is set or not.
    auto col_finish = [&](int jj, Mask need) {
        float best = -1.f, bz = 0.f, bdz = 0.f;
        int bk = 0;
        const float *rc = rs + jj * cst;
        const float *zc = zs + jj * cst;
        // two set bits per round: their coordinate steps are independent, so
        // their latencies overlap (lower atom first: ties go to the lower k)
        for (Mask rest = need; rest;) {
            const int k1 = (sizeof(Mask) == 8 ? __ffsll((long long)rest) : __ffs((int)rest)) - 1;
            rest &= rest - 1;
            const bool two = rest != 0;
            const int k2 =
                two ? (sizeof(Mask) == 8 ? __ffsll((long long)rest) : __ffs((int)rest)) - 1 : k1;
            if (two)
                rest &= rest - 1;
            float zn1, d1, zn2, d2;
            coord_step(rc[k1 * kst], zc[k1 * kst], nrm[k1], rnrm[k1], lam, &zn1, &d1);
            coord_step(rc[k2 * kst], zc[k2 * kst], nrm[k2], rnrm[k2], lam, &zn2, &d2);
            if (fabsf(d1) > best) {
                best = fabsf(d1);
                bk = k1;
                bz = zn1;
                bdz = d1;
            }
            if (two && fabsf(d2) > best) {
                best = fabsf(d2);
                bk = k2;
                bz = zn2;
                bdz = d2;
            }
        }
        // segment-local index k << 17 | jj << 1: same order as k * Tz + t inside
        // the segment (jj < w_max < 2^16: the column caches live in shared
        // memory); bit 0 is the sign of dZ, so the key alone gives dZ exactly
        const unsigned flat = ((unsigned)bk << 17) | ((unsigned)jj << 1) | (bdz < 0.f ? 1u : 0u);
        ckey[jj] = best > 0.f ? ((unsigned long long)__float_as_uint(best) << 32) | (unsigned)(~flat)
                              : 0ull;
        cz[jj] = bz;
    };

    // best coordinate of own column jj over k
    auto col_eval = [&](int jj) {
        const float *rc = rs + jj * cst;
        const float *zc = zs + jj * cst;
        float best = -1.f, bz = 0.f, bdz = 0.f;
        int bk = 0;
        auto visit = [&](int k) {
            const float r = rc[k * kst], z = zc[k * kst];
            // inactive and inside the threshold: Z' = Sh(r, lam)/n = 0 = z exactly
            if (z == 0.f && fabsf(r) <= lam)
                return;
            float zn, d;
            coord_step(r, z, nrm[k], rnrm[k], lam, &zn, &d);
            const float ad = fabsf(d);
            if (ad > best) {
                best = ad;
                bk = k;
                bz = zn;
                bdz = d;
            }
        };
        if constexpr (KFIX) {
            Mask need = 0, zb = 0;
#pragma unroll
            for (int k = 0; k < KT; k++) {
                zb |= (Mask)(zc[k * kst] != 0.f ? 1 : 0) << k;
                need |= (Mask)(fabsf(rc[k * kst]) > lam ? 1 : 0) << k;
            }
            zmask[jj] = zb;
            col_finish(jj, need | zb);
            return;
        } else {
#pragma unroll 5
            for (int k = 0; k < K; k++)
                visit(k);
        }
        const unsigned flat = ((unsigned)bk << 17) | ((unsigned)jj << 1) | (bdz < 0.f ? 1u : 0u);
        ckey[jj] = best > 0.f ? ((unsigned long long)__float_as_uint(best) << 32) | (unsigned)(~flat)
                              : 0ull;
        cz[jj] = bz;
    };
    if constexpr (SMEM && KFIX) {
        // a column's KT values of r and of Z in one round trip of independent
        // loads (coalesced across the threads, one atom row at a time), stored
        // with 128-bit writes, screened from the registers
        for (int jj = tid; jj < w; jj += B) {
            Mask need = 0, zb = 0;
            // r, then Z (one array's column in registers at a time)
#pragma unroll
            for (int a = 0; a < 2; a++) {
                const float *src = (a == 0 ? gr : gz) + s + jj;
                float v[4 * KQ];
#pragma unroll
                for (int k = 0; k < 4 * KQ; k++)
                    v[k] = k < KT ? src[(int64_t)k * ld] : 0.f;
                float4 *dst = reinterpret_cast<float4 *>((a == 0 ? rs : zs) + jj * CST);
#pragma unroll
                for (int q = 0; q < KQ; q++)
                    dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
#pragma unroll
                for (int k = 0; k < KT; k++) {
                    if (a == 0)
                        need |= (Mask)(fabsf(v[k]) > lam ? 1 : 0) << k;
                    else
                        zb |= (Mask)(v[k] != 0.f ? 1 : 0) << k;
                }
            }
            zmask[jj] = zb;
            col_finish(jj, need | zb);
        }
    } else {
        for (int jj = tid; jj < w; jj += B)
            col_eval(jj);
    }
    // (no barrier needed: each thread reads back only its own columns)

    int nupd = 0;
    float decrease = 0.f;  // this thread's updates of the visit (at most u terms)
    int64_t tmin = Tz, tmax = -1;
    bool capped = false;
    for (int it = 0;; it++) {
        // ---- block argmax of the cached column keys ----------------------
        unsigned long long my = 0ull;
        for (int jj = tid; jj < w; jj += B) {
            const unsigned long long kk = ckey[jj];
            if (kk > my)
                my = kk;
        }
        const unsigned long long wm = warp_max_u64(my);
        if (lane == 0 && wm != 0ull)
            atomicMax(&s_best[it & 3], wm);
        if (tid == 0)
            s_best[(it + 2) & 3] = 0ull;
        __syncthreads();
        const unsigned long long bk = s_best[it & 3];
        const float adz = __uint_as_float((unsigned)(bk >> 32));
        if (!(adz >= tol))
            break;
        if (nupd >= pp.u) {
            capped = true;
            break;
        }
        // the winner (k0, column) and dZ = +-|dZ| from its key.  Only the
        // column's owner reads Z' from the column cache: the owner rewrites that
        // cache later in this update, and another thread's read would race it
        const unsigned flat = ~(unsigned)bk;
        const int k0 = (int)(flat >> 17), jw = (int)((flat >> 1) & 0xffffu);
        const float delta = (flat & 1u) ? -adz : adz;
        float znew = 0.f;
        const int64_t t0 = s + jw;

        // ---- Eq. beta_up (r form) on the window -------------------------
        const int64_t tlo = t0 - (L - 1);
        const int off = (tid - (int)(tlo - s)) & (B - 1);  // window position of this thread
        const int64_t t = tlo + off;
        if (off < W2 && t >= 0 && t < Tz) {
            const bool own = t >= s && t < e;
            const int jj = (int)(t - s);
            if (t == t0) {
                znew = cz[jw];
                // Prop. A.1 from the owner's r before this update touches it:
                // E(Z) - E(Z') = dZ (r - n dZ / 2) + lam (|z| - |u|), dZ = u - z
                const float n = nrm[k0], d = delta, u = znew, z = znew - delta;
                const float r0 = rs[jj * cst + k0 * kst];
                decrease += d * (r0 - 0.5f * n * d) + lam * (fabsf(z) - fabsf(u));
            }
            // the K coefficients S_{k,k0}[t-t0] of this lag: float4 group q of
            // (k0, lag) at Ct4[(k0 * Kp/4 + q) * W2 + lag], so that the threads of a
            // warp (consecutive lags) read consecutive 16-byte words; fetch them
            // first (independent vector loads, one L2 round trip), then apply
            const float4 *Ct4 = reinterpret_cast<const float4 *>(pp.Ct);
            const int64_t cbase = (int64_t)k0 * (Kp / 4) * W2 + off;
            float *rcol = rs + jj * cst;
            float *rg = gr + t;  // an idle neighbour's column (no other block touches it)
            auto apply = [&](int k, float cv) {
                if (own)
                    rcol[k * kst] = fmaf(-cv, delta, rcol[k * kst]);
                else
                    atomicAdd(rg + (int64_t)k * ld, -cv * delta);
            };
            if constexpr (KFIX) {
                // all K coefficients in one round trip (KPC/4 vector loads)
                float cv[KPC];
#pragma unroll
                for (int q = 0; q < KPC / 4; q++) {
                    const float4 v = __ldg(Ct4 + cbase + (int64_t)q * W2);
                    cv[4 * q] = v.x;
                    cv[4 * q + 1] = v.y;
                    cv[4 * q + 2] = v.z;
                    cv[4 * q + 3] = v.w;
                }
                if (own) {
                    // apply and screen in registers, then evaluate the movable entries
                    if (t == t0) {
                        zs[jj * cst + k0 * kst] = znew;
                        if constexpr (SMEM)
                            gz[(int64_t)k0 * ld + t0] = znew;  // (the write-back copies r only)
                        const Mask bit = (Mask)1 << k0;
                        zmask[jj] = znew != 0.f ? (zmask[jj] | bit) : (zmask[jj] & ~bit);
                    }
                    Mask need = 0;
                    if constexpr (SMEM) {
                        // 128-bit read-modify-write of the column (padded atoms stay 0:
                        // their coefficients are 0)
                        float4 *rc4 = reinterpret_cast<float4 *>(rcol);
#pragma unroll
                        for (int q = 0; q < KQ; q++) {
                            float4 v = rc4[q];
                            v.x = fmaf(-cv[4 * q], delta, v.x);
                            v.y = fmaf(-cv[4 * q + 1], delta, v.y);
                            v.z = fmaf(-cv[4 * q + 2], delta, v.z);
                            v.w = fmaf(-cv[4 * q + 3], delta, v.w);
                            rc4[q] = v;
                            const float rr[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int e = 0; e < 4; e++)
                                if (4 * q + e < KT)
                                    need |= (Mask)(fabsf(rr[e]) > lam ? 1 : 0) << (4 * q + e);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < KT; k++) {
                            const float r = fmaf(-cv[k], delta, rcol[k * kst]);
                            rcol[k * kst] = r;
                            need |= (Mask)(fabsf(r) > lam ? 1 : 0) << k;
                        }
                    }
                    col_finish(jj, need | zmask[jj]);
                } else {
#pragma unroll
                    for (int k = 0; k < KT; k++)
                        atomicAdd(rg + (int64_t)k * ld, -cv[k] * delta);
                }
            } else {
                const float *Ct1 = pp.Ct;
                for (int kb = 0; kb < K; kb += kCoefBatch) {
                    float cv[kCoefBatch];
#pragma unroll
                    for (int i = 0; i < kCoefBatch; i++) {
                        const int k = kb + i;
                        cv[i] = k < K ? __ldg(Ct1 + ((cbase + (int64_t)(k >> 2) * W2) << 2) + (k & 3))
                                      : 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < kCoefBatch; i++)
                        if (kb + i < K)
                            apply(kb + i, cv[i]);
                }
            }
            if (!KFIX && own) {
                if (t == t0) {
                    zs[jj * cst + k0 * kst] = znew;
                    if constexpr (SMEM)
                        gz[(int64_t)k0 * ld + t0] = znew;
                }
                col_eval(jj);
            }
        }
        nupd++;
        tmin = t0 < tmin ? t0 : tmin;
        tmax = t0 > tmax ? t0 : tmax;
    }

    // ---- write back, spill bookkeeping, trace ---------------------------
    // (Z changed only at the updated coordinates, each written to global
    // memory when it was applied: the write-back copies r)
    if (SMEM && nupd > 0) {
        if constexpr (KFIX) {
            // each thread writes back its own columns (128-bit shared reads;
            // the global stores of one atom row are coalesced across threads)
            for (int jj = tid; jj < w; jj += B) {
                const float4 *rc4 = reinterpret_cast<const float4 *>(rs + jj * CST);
#pragma unroll
                for (int q = 0; q < KQ; q++) {
                    const float4 a = rc4[q];
                    const float ra[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                    for (int e = 0; e < 4; e++)
                        if (4 * q + e < KT)
                            gr[(int64_t)(4 * q + e) * ld + s + jj] = ra[e];
                }
            }
        } else {
            for (int k = 0; k < K; k++) {
                float *rdst = gr + (int64_t)k * ld + s;
                for (int jj = tid; jj < w; jj += B)
                    rdst[jj] = rs[jj * cst + k];
            }
        }
    }
    // objective decrease of the visit: sum over the threads that owned t0
    for (int o = 16; o > 0; o >>= 1)
        decrease += __shfl_xor_sync(kFull, decrease, o);
    if (lane == 0)
        s_dec[warp] = (double)decrease;
    __syncthreads();
    if (tid == 0) {
        double dsum = 0.0;
        for (int i = 0; i < nwarps; i++)
            dsum += s_dec[i];
        pp.dirty[m] = capped ? 1 : 0;
        if (nupd > 0) {
            // neighbours whose r changed: segments meeting [tmin-L+1, tmax+L-1]
            const int64_t lo = tmin - (L - 1), hi = tmax + (L - 1);
            // (a problem's segments are consecutive and ordered by position);
            // they and this segment are also touched: r changed there
            for (int mm = m - 1; mm >= seg_lo && pp.seg_e[mm] > lo; mm--) {
                pp.dirty[mm] = 1;
                pp.touched[mm] = 1;
            }
            for (int mm = m + 1; mm < seg_hi && pp.seg_s[mm] <= hi; mm++) {
                pp.dirty[mm] = 1;
                pp.touched[mm] = 1;
            }
            pp.touched[m] = 1;
            const int slot = g & (kPhaseRing - 1);
            atomicAdd(reinterpret_cast<unsigned long long *>(&pp.upd[slot]),
                      (unsigned long long)nupd);
            atomicAdd(reinterpret_cast<unsigned long long *>(pp.total), (unsigned long long)nupd);
            atomicAdd(reinterpret_cast<unsigned long long *>(pp.visits), 1ull);
            atomicAdd(&pp.dec[slot], dsum);
            atomicMax(&pp.tend[slot], globaltimer_ns());
        }
    }
}

// One visit of segment m by one warp: the compile-time-K, shared-memory form
// for update windows of at most 128 columns (2L-1 <= 127).  Lane l owns the
// segment columns jj == l (mod 32) and handles, in an update, the window
// positions whose column is one of its own (up to four of them), so the
// argmax is a warp reduction, no barrier is needed between updates and the
// coefficients of all the lane's positions are loaded in one round trip.
// The arithmetic of an update is that of visit_segment (same coordinate
// step, same order per column, same tie-break), so both forms apply the
// same updates.
template <int KT>
__device__ __forceinline__ void visit_segment_warp(const PhaseParams &pp, const int m, const int g,
                                                   const int g_round)
{
    static_assert(KT > 0 && KT <= 64, "compile-time K");
    constexpr int KPC = (KT + 3) & ~3;
    constexpr int CST = vec_stride(KT);
    constexpr int KQ = (KT + 3) / 4;
    constexpr int NPOS = 4;  // window positions per lane: 2L-1 <= 4 * 32
    using Mask = typename std::conditional<(KT > 32), unsigned long long, unsigned>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;

    // ---- early exits, decided by lane 0 and broadcast ----
    int go = 1;
    if (lane == 0) {
        if (*(volatile int *)pp.done) {
            go = 0;
        } else if (*(volatile long long *)pp.total >= pp.max_updates) {
            go = 0;
        } else if (g - g_round >= pp.c) {
            long long sum = 0;
            for (int j = g - pp.c; j < g; j++)
                sum += *(volatile long long *)&pp.upd[j & (kPhaseRing - 1)];
            if (sum == 0) {
                *(volatile int *)pp.done = g + 1;
                go = 0;
            }
        }
        if (go && !*(volatile unsigned char *)&pp.dirty[m])
            go = 0;
    }
    if (!__shfl_sync(kFull, go, 0))
        return;

    const int K = KT, L = pp.L, W2 = 2 * L - 1, Kp = KPC;
    const SigDesc *sdp = pp.sig + pp.seg_sig[m];
    float *const gr = sdp->r;
    float *const gz = sdp->Z;
    const int64_t ld = sdp->ld, Tz = sdp->Tz;
    const int seg_lo = sdp->seg0, seg_hi = sdp->seg0 + sdp->nseg;
    const int64_t s = pp.seg_s[m], e = pp.seg_e[m];
    const int w = (int)(e - s);
    const float lam = sdp->lam, tol = sdp->tol;

    const Layout lay(K, pp.w_max, true, true);
    unsigned long long *ckey = reinterpret_cast<unsigned long long *>(smem_raw + lay.key);
    float *cz = reinterpret_cast<float *>(smem_raw + lay.cz);
    float *cd = reinterpret_cast<float *>(smem_raw + lay.cd);
    int *ck = reinterpret_cast<int *>(smem_raw + lay.ck);
    Mask *zmask = reinterpret_cast<Mask *>(smem_raw + lay.zm);
    float *nrm = reinterpret_cast<float *>(smem_raw + lay.nrm);
    float *rnrm = reinterpret_cast<float *>(smem_raw + lay.rnrm);
    float *rs = reinterpret_cast<float *>(smem_raw + lay.r);
    float *zs = reinterpret_cast<float *>(smem_raw + lay.z);
    for (int k = lane; k < K; k += 32) {
        nrm[k] = pp.norms[k];
        rnrm[k] = __frcp_rn(pp.norms[k]);
    }
    __syncwarp();

    // best coordinate of own column jj over the atoms whose bit is set in need
    auto col_finish = [&](int jj, Mask need) {
        float best = -1.f, bz = 0.f, bdz = 0.f;
        int bk = 0;
        const float *rc = rs + jj * CST;
        const float *zc = zs + jj * CST;
        for (Mask rest = need; rest; rest &= rest - 1) {
            const int k = (sizeof(Mask) == 8 ? __ffsll((long long)rest) : __ffs((int)rest)) - 1;
            float zn, d;
            coord_step(rc[k], zc[k], nrm[k], rnrm[k], lam, &zn, &d);
            const float ad = fabsf(d);
            if (ad > best) {
                best = ad;
                bk = k;
                bz = zn;
                bdz = d;
            }
        }
        const unsigned flat = (unsigned)bk * (unsigned)pp.w_max + (unsigned)jj;
        ckey[jj] = best > 0.f ? ((unsigned long long)__float_as_uint(best) << 32) | (unsigned)(~flat)
                              : 0ull;
        cz[jj] = bz;
        cd[jj] = bdz;
        ck[jj] = bk;
    };
    // stage the lane's columns (one round trip of independent loads each)
    for (int jj = lane; jj < w; jj += 32) {
        Mask need = 0, zb = 0;
#pragma unroll
        for (int a = 0; a < 2; a++) {
            const float *src = (a == 0 ? gr : gz) + s + jj;
            float v[4 * KQ];
#pragma unroll
            for (int k = 0; k < 4 * KQ; k++)
                v[k] = k < KT ? src[(int64_t)k * ld] : 0.f;
            float4 *dst = reinterpret_cast<float4 *>((a == 0 ? rs : zs) + jj * CST);
#pragma unroll
            for (int q = 0; q < KQ; q++)
                dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
#pragma unroll
            for (int k = 0; k < KT; k++) {
                if (a == 0)
                    need |= (Mask)(fabsf(v[k]) > lam ? 1 : 0) << k;
                else
                    zb |= (Mask)(v[k] != 0.f ? 1 : 0) << k;
            }
        }
        zmask[jj] = zb;
        col_finish(jj, need | zb);
    }
    __syncwarp();

    const float4 *Ct4 = reinterpret_cast<const float4 *>(pp.Ct);
    int nupd = 0;
    float decrease = 0.f;
    int64_t tmin = Tz, tmax = -1;
    bool capped = false;
    for (int it = 0;; it++) {
        // ---- warp argmax of the cached column keys ----------------------
        unsigned long long my = 0ull;
        int myj = 0;
        for (int jj = lane; jj < w; jj += 32) {
            const unsigned long long kk = ckey[jj];
            if (kk > my) {
                my = kk;
                myj = jj;
            }
        }
        const unsigned long long wm = warp_max_u64(my);
        const float adz = __uint_as_float((unsigned)(wm >> 32));
        if (!(adz >= tol))
            break;
        if (it >= pp.u) {
            capped = true;
            break;
        }
        const int src = __ffs(__ballot_sync(kFull, my == wm)) - 1;
        // the winning column is one of lane src's own: it reads its cached step
        float wz = 0.f, wd = 0.f;
        int wk = 0;
        if (lane == src) {
            wz = cz[myj];
            wd = cd[myj];
            wk = ck[myj];
        }
        const int jw = __shfl_sync(kFull, myj, src);
        const float znew = __shfl_sync(kFull, wz, src), delta = __shfl_sync(kFull, wd, src);
        const int k0 = __shfl_sync(kFull, wk, src);
        const int64_t t0 = s + jw;

        // ---- Eq. beta_up (r form) on the window -------------------------
        const int64_t tlo = t0 - (L - 1);
        const int base = (lane - (int)((tlo - s) & 31)) & 31;
        float cv[NPOS][KPC];
#pragma unroll
        for (int q = 0; q < NPOS; q++) {
            const int off = base + 32 * q;
            const int64_t t = tlo + off;
            const bool valid = off < W2 && t >= 0 && t < Tz;
            const int64_t cb = (int64_t)k0 * (Kp / 4) * W2 + (valid ? off : 0);
#pragma unroll
            for (int g4 = 0; g4 < KPC / 4; g4++) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (valid)
                    v = __ldg(Ct4 + cb + (int64_t)g4 * W2);
                cv[q][4 * g4] = v.x;
                cv[q][4 * g4 + 1] = v.y;
                cv[q][4 * g4 + 2] = v.z;
                cv[q][4 * g4 + 3] = v.w;
            }
        }
#pragma unroll
        for (int q = 0; q < NPOS; q++) {
            const int off = base + 32 * q;
            const int64_t t = tlo + off;
            if (!(off < W2 && t >= 0 && t < Tz))
                continue;
            const int jj = (int)(t - s);
            if (t >= s && t < e) {
                float *rcol = rs + jj * CST;
                if (t == t0) {
                    const float n = nrm[k0], u = znew, z = znew - delta;
                    decrease += delta * (rcol[k0] - 0.5f * n * delta) + lam * (fabsf(z) - fabsf(u));
                    zs[jj * CST + k0] = znew;
                    gz[(int64_t)k0 * ld + t0] = znew;  // (the write-back copies r only)
                    const Mask bit = (Mask)1 << k0;
                    zmask[jj] = znew != 0.f ? (zmask[jj] | bit) : (zmask[jj] & ~bit);
                }
                Mask need = 0;
                float4 *rc4 = reinterpret_cast<float4 *>(rcol);
#pragma unroll
                for (int g4 = 0; g4 < KQ; g4++) {
                    float4 v = rc4[g4];
                    v.x = fmaf(-cv[q][4 * g4], delta, v.x);
                    v.y = fmaf(-cv[q][4 * g4 + 1], delta, v.y);
                    v.z = fmaf(-cv[q][4 * g4 + 2], delta, v.z);
                    v.w = fmaf(-cv[q][4 * g4 + 3], delta, v.w);
                    rc4[g4] = v;
                    const float rr[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int c = 0; c < 4; c++)
                        if (4 * g4 + c < KT)
                            need |= (Mask)(fabsf(rr[c]) > lam ? 1 : 0) << (4 * g4 + c);
                }
                col_finish(jj, need | zmask[jj]);
            } else {
                // an idle neighbour's column (no other block touches it)
                float *rg = gr + t;
#pragma unroll
                for (int k = 0; k < KT; k++)
                    atomicAdd(rg + (int64_t)k * ld, -cv[q][k] * delta);
            }
        }
        __syncwarp();  // every lane's keys are updated before the next argmax
        nupd++;
        tmin = t0 < tmin ? t0 : tmin;
        tmax = t0 > tmax ? t0 : tmax;
    }

    // ---- write back, spill bookkeeping, trace ---------------------------
    if (nupd > 0) {
        for (int jj = lane; jj < w; jj += 32) {
            const float4 *rc4 = reinterpret_cast<const float4 *>(rs + jj * CST);
#pragma unroll
            for (int q = 0; q < KQ; q++) {
                const float4 a = rc4[q];
                const float ra[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                for (int c = 0; c < 4; c++)
                    if (4 * q + c < KT)
                        gr[(int64_t)(4 * q + c) * ld + s + jj] = ra[c];
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1)
        decrease += __shfl_xor_sync(kFull, decrease, o);
    if (lane == 0) {
        pp.dirty[m] = capped ? 1 : 0;
        if (nupd > 0) {
            const int64_t lo = tmin - (L - 1), hi = tmax + (L - 1);
            for (int mm = m - 1; mm >= seg_lo && pp.seg_e[mm] > lo; mm--) {
                pp.dirty[mm] = 1;
                pp.touched[mm] = 1;
            }
            for (int mm = m + 1; mm < seg_hi && pp.seg_s[mm] <= hi; mm++) {
                pp.dirty[mm] = 1;
                pp.touched[mm] = 1;
            }
            pp.touched[m] = 1;
            const int slot = g & (kPhaseRing - 1);
            atomicAdd(reinterpret_cast<unsigned long long *>(&pp.upd[slot]),
                      (unsigned long long)nupd);
            atomicAdd(reinterpret_cast<unsigned long long *>(pp.total), (unsigned long long)nupd);
            atomicAdd(reinterpret_cast<unsigned long long *>(pp.visits), 1ull);
            atomicAdd(&pp.dec[slot], (double)decrease);
            atomicMax(&pp.tend[slot], globaltimer_ns());
        }
    }
}

// Launch index and first index of the round: from the parameters, or, for
// launches replayed from a CUDA graph, offsets from counters in device memory.
__device__ __forceinline__ int launch_index(const PhaseParams &pp)
{
    return pp.g_dev ? *pp.g_dev + pp.g : pp.g;
}
__device__ __forceinline__ int round_index(const PhaseParams &pp)
{
    return pp.g_round_dev ? *pp.g_round_dev : pp.g_round;
}

// MAXT: the block size the instantiation is launched with.  Blocks of 128
// threads (atoms up to 64 samples) are compiled for 5 resident blocks per SM,
// so that the several hundred co-active segments of a phase fit in one wave;
// larger blocks get the full register file.
// One block per segment of the phase list.
template <bool SMEM, int MAXT, int KT>
__global__ void __launch_bounds__(MAXT, MAXT <= 128 ? 5 : 1) phase_kernel(PhaseParams pp)
{
    visit_segment<SMEM, MAXT, KT>(pp, pp.phase_list[blockIdx.x], launch_index(pp),
                                  round_index(pp));
}

// One warp (block) per segment of the phase list (K fixed, 2L-1 <= 127).
template <int KT>
__global__ void __launch_bounds__(32) phase_warp_kernel(PhaseParams pp)
{
    visit_segment_warp<KT>(pp, pp.phase_list[blockIdx.x], launch_index(pp), round_index(pp));
}

// The persistent form of the warp kernel (see phase_drain_kernel).
template <int KT>
__global__ void __launch_bounds__(32) phase_warp_drain_kernel(PhaseParams pp)
{
    const int n = *pp.qlen;
    const int g = launch_index(pp), g_round = round_index(pp);
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && lane == 0 && g - g_round >= pp.c && !*(volatile int *)pp.done) {
        long long sum = 0;
        for (int j = g - pp.c; j < g; j++)
            sum += *(volatile long long *)&pp.upd[j & (kPhaseRing - 1)];
        if (sum == 0)
            *(volatile int *)pp.done = g + 1;
    }
    for (;;) {
        int idx = 0;
        if (lane == 0)
            idx = atomicAdd(pp.qhead, 1);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= n)
            break;
        visit_segment_warp<KT>(pp, pp.queue[idx], g, g_round);
        __syncwarp();  // the next visit re-uses the shared memory
    }
}

// Persistent form: a grid of resident blocks drains the queue of this phase's
// segments that need a visit (built by compact_phase_kernel), so a phase with
// few dirty segments among very many costs its work, not a block per segment.
template <bool SMEM, int MAXT, int KT>
__global__ void __launch_bounds__(MAXT, MAXT <= 128 ? 5 : 1) phase_drain_kernel(PhaseParams pp)
{
    __shared__ int s_idx;
    const int n = *pp.qlen;
    const int g = launch_index(pp), g_round = round_index(pp);
    // an empty queue visits nothing, so the test for a full sweep without
    // updates (made at the start of every visit) is also made here once
    if (blockIdx.x == 0 && threadIdx.x == 0 && g - g_round >= pp.c &&
        !*(volatile int *)pp.done) {
        long long sum = 0;
        for (int j = g - pp.c; j < g; j++)
            sum += *(volatile long long *)&pp.upd[j & (kPhaseRing - 1)];
        if (sum == 0)
            *(volatile int *)pp.done = g + 1;
    }
    for (;;) {
        if (threadIdx.x == 0)
            s_idx = atomicAdd(pp.qhead, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();  // every thread has read s_idx before it is overwritten
        if (idx >= n)
            break;
        visit_segment<SMEM, MAXT, KT>(pp, pp.queue[idx], g, g_round);
        __syncthreads();  // the next visit re-uses the shared memory
    }
}

// The segments of a phase list that need a visit, in any order (co-active
// segments are independent, so the order of their visits changes nothing).
__global__ void compact_phase_kernel(const int *__restrict__ list, int count,
                                     const unsigned char *__restrict__ dirty,
                                     int *__restrict__ queue, int *__restrict__ qlen)
{
    const int lane = threadIdx.x & 31;
    for (int i0 = blockIdx.x * blockDim.x; i0 < count; i0 += gridDim.x * blockDim.x) {
        const int i = i0 + threadIdx.x;
        int m = 0;
        bool want = false;
        if (i < count) {
            m = list[i];
            want = dirty[m] != 0;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, want);
        int base = 0;
        if (lane == 0 && mask)
            base = atomicAdd(qlen, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (want)
            queue[base + __popc(mask & ((1u << lane) - 1u))] = m;
    }
}

}  // namespace

bool phase_warp_eligible(int K, int L, int wmax)
{
    return K == 25 && 2 * L - 1 <= 128 && Layout(K, wmax, true, true).total <= (size_t)kMaxSmem;
}

PhaseConfig phase_config(int K, int L, int wmax, int threads_per_segment)
{
    PhaseConfig cfg;
    if (threads_per_segment == 32 && phase_warp_eligible(K, L, wmax)) {
        // one warp per segment (visit_segment_warp)
        cfg.block = 32;
        cfg.tile_in_smem = true;
        cfg.smem = Layout(K, wmax, true, true).total;
        return cfg;
    }
    // An update touches the 2L-1 window columns: with at least that many threads
    // each of them goes to its own thread, however wide the segment; more threads
    // would idle in the update and only cost registers and occupancy.  The block
    // is a power of two (128, 512 or 1024) so that ownership is a mask.
    cfg.block = 2 * L - 1 <= 128 ? 128 : (2 * L - 1 <= 512 ? 512 : 1024);
    const bool vec = vec_layout(K, cfg.block);
    cfg.tile_in_smem = Layout(K, (int)wmax, true, vec).total <= (size_t)kMaxSmem;
    cfg.smem = Layout(K, (int)wmax, cfg.tile_in_smem, vec).total;
    return cfg;
}

namespace {

// Calls f with the phase-kernel instantiation (template) matching cfg and K.
template <template <bool, int, int> class Sel, class F>
cudaError_t dispatch(const PhaseConfig &cfg, int K, F &&f)
{
    // one warp per segment (phase_config checked K == 25 and the window)
    if (cfg.block == 32)
        return f(Sel<true, 32, 25>::fn());
    // the workloads' atom counts (25 and 64) are compiled with K fixed
    if (cfg.block == 128) {
        if (K == 25)
            return cfg.tile_in_smem ? f(Sel<true, 128, 25>::fn()) : f(Sel<false, 128, 25>::fn());
        if (K == 64)
            return cfg.tile_in_smem ? f(Sel<true, 128, 64>::fn()) : f(Sel<false, 128, 64>::fn());
        return cfg.tile_in_smem ? f(Sel<true, 128, 0>::fn()) : f(Sel<false, 128, 0>::fn());
    }
    if (cfg.block == 512) {
        if (K == 25)
            return cfg.tile_in_smem ? f(Sel<true, 512, 25>::fn()) : f(Sel<false, 512, 25>::fn());
        if (K == 64)
            return cfg.tile_in_smem ? f(Sel<true, 512, 64>::fn()) : f(Sel<false, 512, 64>::fn());
        return cfg.tile_in_smem ? f(Sel<true, 512, 0>::fn()) : f(Sel<false, 512, 0>::fn());
    }
    return cfg.tile_in_smem ? f(Sel<true, 1024, 0>::fn()) : f(Sel<false, 1024, 0>::fn());
}

// (block 32 selects the warp forms; A is then always true and C == 25)
template <bool A, int B, int C>
struct PerSegment {
    static auto fn()
    {
        if constexpr (B == 32)
            return phase_warp_kernel<C>;
        else
            return phase_kernel<A, B, C>;
    }
};
template <bool A, int B, int C>
struct Drain {
    static auto fn()
    {
        if constexpr (B == 32)
            return phase_warp_drain_kernel<C>;
        else
            return phase_drain_kernel<A, B, C>;
    }
};

cudaError_t check(const PhaseParams &pp, const PhaseConfig &cfg)
{
    if (cfg.smem > (size_t)kMaxSmem)
        return cudaErrorInvalidConfiguration;
    if (cfg.block == 32 ? 2 * pp.L - 1 > 128 : cfg.block < 2 * pp.L - 1)
        return cudaErrorInvalidConfiguration;  // window positions per thread: 1 (block), <= 4 (warp)
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_phase(const PhaseParams &pp, const PhaseConfig &cfg, int active,
                         cudaStream_t s)
{
    if (active == 0)
        return cudaSuccess;
    cudaError_t e = check(pp, cfg);
    if (e != cudaSuccess)
        return e;
    e = dispatch<PerSegment>(cfg, pp.K, [&](auto kern) -> cudaError_t {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)cfg.smem);
        if (r != cudaSuccess)
            return r;
        kern<<<active, cfg.block, cfg.smem, s>>>(pp);
        return cudaSuccess;
    });
    if (e != cudaSuccess)
        return e;
    return cudaGetLastError();
}

int phase_resident_blocks(const PhaseConfig &cfg, int K)
{
    int per_sm = 1, dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    dispatch<Drain>(cfg, K, [&](auto kern) -> cudaError_t {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, cfg.block, cfg.smem);
        return cudaSuccess;
    });
    cudaGetLastError();
    return nsm * (per_sm < 1 ? 1 : per_sm);
}

cudaError_t launch_phase_drain(const PhaseParams &pp, const PhaseConfig &cfg, int active,
                               int resident, cudaStream_t s)
{
    if (active == 0)
        return cudaSuccess;
    cudaError_t e = check(pp, cfg);
    if (e != cudaSuccess)
        return e;
    // queue length and head (two adjacent ints) start at 0
    e = cudaMemsetAsync(pp.qhead, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess)
        return e;
    const int cb = 256;
    const int cg = (active + cb - 1) / cb < 4096 ? (active + cb - 1) / cb : 4096;
    compact_phase_kernel<<<cg, cb, 0, s>>>(pp.phase_list, active, pp.dirty, pp.queue, pp.qhead + 1);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const int grid = resident < active ? resident : active;
    e = dispatch<Drain>(cfg, pp.K, [&](auto kern) -> cudaError_t {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)cfg.smem);
        if (r != cudaSuccess)
            return r;
        kern<<<grid, cfg.block, cfg.smem, s>>>(pp);
        return cudaSuccess;
    });
    if (e != cudaSuccess)
        return e;
    return cudaGetLastError();
}

}  // namespace csc
