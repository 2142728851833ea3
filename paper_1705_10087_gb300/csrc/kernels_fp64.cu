// The re-synchronisation of the solver state r = beta - n Z with its
// definition (Sec. 2.1), the objective E(Z) of Eq. sparse_code from the
// explicit residual (FP64, one value per problem), and per-problem lambda_max.
// Blocks work on tiles of one problem each (SigDesc, Tiles).
//
// Both exploit that Z is sparse: a block gathers the nonzeros of Z that can
// reach its tile (compacted in a fixed order, so results are deterministic)
// and every thread accumulates its outputs over that list in double-float
// (pairs of floats with error-free transformations), combined in FP64.
#include "csc_internal.cuh"

namespace csc {

namespace {

constexpr int kChunk = 64;  // Z columns scanned per compaction round
constexpr int kBucketBatch = 8;  // atom rows of Z a warp loads at once when listing nonzeros

struct NZ {
    int k;
    int t;  // column index in its problem (Tz < 2^31 is checked at init)
    float z;
};

// Ordered compaction of the nonzeros of Z[:, c0:c1) (k-major) into list.
// Returns the count (same value in every thread).  Block-wide barriers; each
// thread takes 4 consecutive elements per round (two barriers per 4*blockDim).
__device__ int compact_nonzeros(const float *__restrict__ Z, int K, int64_t ld, int64_t c0,
                                int64_t c1, NZ *list, int *warp_counts)
{
    const int tid = threadIdx.x, B = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = B >> 5;
    const int width = (int)(c1 - c0);
    const int n = K * width;
    int base = 0;
    for (int r0 = 0; r0 < n; r0 += 4 * B) {
        float z[4];
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int i = r0 + 4 * tid + q;
            z[q] = 0.f;
            if (i < n)
                z[q] = Z[(int64_t)(i / width) * ld + c0 + i % width];
            cnt += z[q] != 0.f;
        }
        // inclusive warp scan of the counts
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o)
                inc += v;
        }
        if (lane == 31)
            warp_counts[warp] = inc;
        __syncthreads();
        int off = base, tot = base;
        for (int q = 0; q < nw; q++) {
            const int wc = warp_counts[q];
            off += q < warp ? wc : 0;
            tot += wc;
        }
        int pos = off + inc - cnt;
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (z[q] != 0.f) {
                const int i = r0 + 4 * tid + q;
                list[pos++] = NZ{i / width, (int)(c0 + i % width), z[q]};
            }
        __syncthreads();
        base = tot;
    }
    return base;
}

constexpr int kResyncThreads = 256;
constexpr int kResyncGroups = kResyncThreads / kResyncCols;  // atom groups
constexpr int kListMax = 32 * kChunk;  // nonzeros a tile gathers from the lists at once
constexpr int kGatherBatch = 4;        // nonzeros whose coefficients are loaded together

// Whether r may have changed on the columns [c0, c0 + kResyncCols) of a
// problem since the last resync: every update window marks the segments it
// covers as touched, and every update marks its own segment.
__device__ __forceinline__ bool tile_touched(const SigDesc &sd, int64_t c0,
                                             const unsigned char *__restrict__ touched)
{
    if (!touched || sd.nseg <= 0)
        return true;
    // the problem's segments are the equal cut of seg_start
    const int64_t ce = c0 + kResyncCols < sd.Tz ? c0 + kResyncCols : sd.Tz;
    const int j1 = segment_of(sd.Tz, sd.nseg, ce - 1);
    for (int j = segment_of(sd.Tz, sd.nseg, c0); j <= j1; j++)
        if (touched[sd.seg0 + j])
            return true;
    return false;
}

// One warp per tile: the tile's nonzeros in (k, column) order (ballot
// compaction over 32 columns, one coalesced row of Z per atom).
__global__ void __launch_bounds__(256)
    nz_bucket_kernel(const SigDesc *__restrict__ sigs, Tiles tiles, int K,
                     const unsigned char *__restrict__ touched, NzLists lists)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (b >= tiles.n)
        return;
    const SigDesc sd = sigs[tiles.sig[b]];
    const int64_t c0 = tiles.start[b];
    // Z changed only in touched segments: the bucket of an untouched tile is
    // the one built at the previous resync over the same Z
    if (!tile_touched(sd, c0, touched))
        return;
    const int64_t t = c0 + lane;
    const bool in = t < sd.Tz;
    uint2 *__restrict__ out = lists.ent + b * kNzCap;
    int base = 0;
    for (int k0 = 0; k0 < K; k0 += kBucketBatch) {
        // kBucketBatch rows loaded together: one memory round trip
        float zv[kBucketBatch];
#pragma unroll
        for (int q = 0; q < kBucketBatch; q++)
            zv[q] = in && k0 + q < K ? sd.Z[(int64_t)(k0 + q) * sd.ld + t] : 0.f;
#pragma unroll
        for (int q = 0; q < kBucketBatch; q++) {
            const float z = zv[q];
            const unsigned m = __ballot_sync(0xffffffffu, z != 0.f);
            if (z != 0.f) {
                const int pos = base + __popc(m & ((1u << lane) - 1u));
                if (pos < kNzCap)
                    out[pos] = make_uint2((unsigned)((k0 + q) * kResyncCols + lane),
                                          __float_as_uint(z));
            }
            base += __popc(m);
        }
    }
    if (lane == 0)
        lists.count[b] = base;
}

// The refreshed r of coordinate (k, t) of problem sd from beta0 and the
// double-float sum (ah, al) of its S Z terms, and its share of the report:
// drift |r_old - r|, zero_excess, nonzero_gap, max |Delta Z| and the
// coord_step change on the float state (marking its segment dirty when that
// change is >= tol_mark, or the problem's tol when tol_mark < 0).
// (b0, rold, z, n: beta0, r, Z of the coordinate and ||D_k||^2, already loaded)
__device__ __forceinline__ void resync_finish_v(const SigDesc &sd, int64_t ix, int64_t t,
                                                float b0, float rold, float z, float n, float rn,
                                                float *__restrict__ rr, float ah, float al,
                                                float lam, int write_r,
                                                unsigned char *__restrict__ dirty, float tol_mark,
                                                float &drift, float &zex, float &nzg, float &all,
                                                float &dz32)
{
    const int64_t Tz = sd.Tz;
    // r = beta0 - (hi + lo), finished with TwoSum so that only the final
    // float rounding remains
    const float sm = __fsub_rn(b0, ah);
    const float bv = __fsub_rn(sm, b0);
    const float er = __fadd_rn(__fsub_rn(b0, __fsub_rn(sm, bv)), __fsub_rn(-ah, bv));
    const float r32 = __fadd_rn(sm, __fsub_rn(er, al));
    if (write_r)
        rr[ix] = r32;
    drift = fmaxf(drift, fabsf(rold - r32));
    // optimality in the r form (Theorem A.1): z = 0 needs |beta| = |r| <= lam;
    // otherwise |Z' - z| with Z' from Eq. pb_coord, without cancellation
    float gap;
    if (z == 0.f) {
        zex = fmaxf(zex, fabsf(r32) - lam);
        gap = soft_f(r32, lam) * rn;
    } else {
        const float sg = z > 0.f ? 1.f : -1.f;
        const float b = fmaf(n, z, r32);
        gap = b * sg > lam ? (r32 - lam * sg) * rn : soft_f(b, lam) * rn - z;
        nzg = fmaxf(nzg, fabsf(gap));
    }
    all = fmaxf(all, fabsf(gap));
    // the phase kernel's own test on the float state it will see
    float zn, d32;
    coord_step(write_r ? r32 : rold, z, n, rn, lam, &zn, &d32);
    dz32 = fmaxf(dz32, fabsf(d32));
    if (dirty && sd.nseg > 0 && fabsf(d32) >= (tol_mark < 0.f ? sd.tol : tol_mark))
        dirty[sd.seg0 + segment_of(Tz, sd.nseg, t)] = 1;
}

// resync_finish_v with its loads
__device__ __forceinline__ void resync_finish(const SigDesc &sd, int k, int64_t t,
                                              const float *__restrict__ b0p,
                                              float *__restrict__ rr,
                                              const float *__restrict__ zz,
                                              const float *__restrict__ norms, float ah, float al,
                                              float lam, int write_r,
                                              unsigned char *__restrict__ dirty, float tol_mark,
                                              float &drift, float &zex, float &nzg, float &all,
                                              float &dz32)
{
    const int64_t ix = (int64_t)k * sd.ld + t;
    const float n = norms[k];
    resync_finish_v(sd, ix, t, b0p[ix], rr[ix], zz[ix], n, __frcp_rn(n), rr, ah, al, lam, write_r,
                    dirty, tol_mark, drift, zex, nzg, all, dz32);
}

// KPT = 4 NG atoms per thread: thread group g (of kResyncGroups) owns the
// float4 groups of atoms g, g + kResyncGroups, ... of the by-lag table, so
// each listed nonzero costs one 16-byte coefficient load per group.
template <int KPT>
__global__ void __launch_bounds__(kResyncThreads, KPT <= 4 ? 3 : 1)
    resync_kernel(const SigDesc *__restrict__ sigs, Tiles tiles, const float *__restrict__ Ct,
                  const float *__restrict__ norms, int K, int L, int write_r,
                  unsigned long long *__restrict__ red, int red_stride,
                  unsigned char *__restrict__ dirty, float tol_mark,
                  const unsigned char *__restrict__ touched, float *__restrict__ rep,
                  NzLists lists)
{
    __shared__ NZ list[kListMax];
    __shared__ int warp_counts[32];
    __shared__ float bred[5][kResyncThreads / 32];
    __shared__ int s_off[2 * (kMaxL / kResyncCols) + 2];
    __shared__ int s_ok;
    const int isig = tiles.sig[blockIdx.x];
    const SigDesc sd = sigs[isig];
    const int64_t Tz = sd.Tz, ld = sd.ld;
    float *__restrict__ const rr = sd.r;
    const float *__restrict__ const zz = sd.Z;
    const float *__restrict__ const b0p = sd.beta0;
    const int W2 = 2 * L - 1;
    const int tid = threadIdx.x;
    const int col = tid % kResyncCols, grp = tid / kResyncCols;
    const int64_t c0 = tiles.start[blockIdx.x];
    const int64_t t = c0 + col;
    // columns this tile computes: [c0, tend)
    const int64_t tend = tiles.end && tiles.end[blockIdx.x] < Tz ? tiles.end[blockIdx.x] : Tz;
    float drift = 0.f, zex = 0.f, nzg = 0.f, all = 0.f, dz32 = 0.f;
    // r changed on this tile's columns only where an update window reached
    // them, and every window marks the segments it covers as touched
    const bool need = !(touched && rep) || tile_touched(sd, c0, touched);
    if (!need) {
        if (tid == 0) {  // the stored report of the unchanged tile (drift 0)
            zex = rep[5 * blockIdx.x + 1];
            nzg = rep[5 * blockIdx.x + 2];
            all = rep[5 * blockIdx.x + 3];
            dz32 = rep[5 * blockIdx.x + 4];
        }
    } else {
    float acc_hi[KPT], acc_lo[KPT];
#pragma unroll
    for (int i = 0; i < KPT; i++) {
        acc_hi[i] = 0.f;
        acc_lo[i] = 0.f;
    }

    // nonzeros that reach [c0, c0+cols): Z columns in [c0-(L-1), c0+cols+(L-1)),
    // i.e. the buckets of the tiles b-R .. b+R of the same problem
    const int R = (L - 1 + kResyncCols - 1) / kResyncCols;
    bool listed = false;
    if (lists.count) {
        if (tid <= 2 * R) {
            const int64_t bb = (int64_t)blockIdx.x - R + tid;
            int cnt = 0;
            if (bb >= 0 && bb < tiles.n && tiles.sig[bb] == isig &&
                tiles.start[bb] == c0 + (int64_t)(tid - R) * kResyncCols)
                cnt = lists.count[bb];
            s_off[tid + 1] = cnt;
        }
        __syncthreads();
        if (tid == 0) {
            int acc = 0, ok = 1;
            s_off[0] = 0;
            for (int j = 1; j <= 2 * R + 1; j++) {
                ok &= s_off[j] <= kNzCap;
                acc += s_off[j];
                s_off[j] = acc;
            }
            s_ok = ok && acc <= kListMax;
        }
        __syncthreads();
        listed = s_ok != 0;
    }
    if (listed) {
        // copy the 2R+1 buckets (in tile order) into the shared list
        const int warp = tid >> 5, lane = tid & 31;
        for (int j = warp; j <= 2 * R; j += kResyncThreads / 32) {
            const int n0 = s_off[j], cnt = s_off[j + 1] - n0;
            if (cnt == 0)
                continue;
            const int64_t bb = (int64_t)blockIdx.x - R + j;
            const int64_t cb = c0 + (int64_t)(j - R) * kResyncCols;
            const uint2 *src = lists.ent + bb * kNzCap;
            for (int i = lane; i < cnt; i += 32) {
                const uint2 v = src[i];
                list[n0 + i] = NZ{(int)(v.x / kResyncCols), (int)(cb + v.x % kResyncCols),
                                  __uint_as_float(v.y)};
            }
        }
        __syncthreads();
    }
    const int64_t lo = c0 - (L - 1) > 0 ? c0 - (L - 1) : 0;
    const int64_t hi = c0 + kResyncCols + (L - 1) < Tz ? c0 + kResyncCols + (L - 1) : Tz;
    const int chunk = listed ? (int)(hi - lo)
                             : ((32 * kChunk) / K < kChunk ? (32 * kChunk) / K : kChunk);
    for (int64_t a = lo; a < hi; a += chunk) {
        const int64_t b = a + chunk < hi ? a + chunk : hi;
        const int n = listed ? s_off[2 * R + 1] : compact_nonzeros(zz, K, ld, a, b, list, warp_counts);
        if (t < tend) {
            // NB nonzeros at a time: all their coefficients are loaded first
            // (one float4 per atom group, clamped to valid addresses), so that
            // one L2 round trip serves the batch; a nonzero out of the window
            // (or past n) adds the exact product 0 and leaves the sums unchanged
            // (fewer at a time for many atoms per thread: registers)
            constexpr int NG = KPT / 4;
            constexpr int NB = NG == 1 ? 2 * kGatherBatch : (NG == 2 ? kGatherBatch : (NG <= 4 ? 2 : 1));
            const int G = (K + 3) / 4;  // float4 groups of the table
            const float4 *Ct4 = reinterpret_cast<const float4 *>(Ct);
            for (int i0 = 0; i0 < n; i0 += NB) {
                float4 cv[NB][NG];
                float zv[NB];
#pragma unroll
                for (int b = 0; b < NB; b++) {
                    const int i = i0 + b < n ? i0 + b : n - 1;
                    const NZ e = list[i];
                    const int d = (int)(t - e.t) + (L - 1);
                    const bool in = i0 + b < n && d >= 0 && d < W2;
                    zv[b] = in ? e.z : 0.f;
                    const int64_t base = (int64_t)e.k * G * W2 + (in ? d : 0);
#pragma unroll
                    for (int gi = 0; gi < NG; gi++) {
                        const int g = grp + gi * kResyncGroups;
                        cv[b][gi] = g < G ? __ldg(Ct4 + base + (int64_t)g * W2)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int b = 0; b < NB; b++)
#pragma unroll
                    for (int gi = 0; gi < NG; gi++)
                        if (zv[b] != 0.f) {
                            df_add_prod(acc_hi[4 * gi], acc_lo[4 * gi], cv[b][gi].x, zv[b]);
                            df_add_prod(acc_hi[4 * gi + 1], acc_lo[4 * gi + 1], cv[b][gi].y, zv[b]);
                            df_add_prod(acc_hi[4 * gi + 2], acc_lo[4 * gi + 2], cv[b][gi].z, zv[b]);
                            df_add_prod(acc_hi[4 * gi + 3], acc_lo[4 * gi + 3], cv[b][gi].w, zv[b]);
                        }
            }
        }
        __syncthreads();
    }

    const float lam = sd.lam;
    if (t < tend) {
#pragma unroll
        for (int q = 0; q < KPT; q++) {
            const int k = 4 * (grp + (q / 4) * kResyncGroups) + (q % 4);
            if (k >= K)
                continue;
            resync_finish(sd, k, t, b0p, rr, zz, norms, acc_hi[q], acc_lo[q], lam, write_r, dirty,
                          tol_mark, drift, zex, nzg, all, dz32);
        }
    }
    }  // need
    // block reduce (max) and one atomic per block and quantity
    for (int off = 16; off > 0; off >>= 1) {
        drift = fmaxf(drift, __shfl_xor_sync(0xffffffffu, drift, off));
        zex = fmaxf(zex, __shfl_xor_sync(0xffffffffu, zex, off));
        nzg = fmaxf(nzg, __shfl_xor_sync(0xffffffffu, nzg, off));
        all = fmaxf(all, __shfl_xor_sync(0xffffffffu, all, off));
        dz32 = fmaxf(dz32, __shfl_xor_sync(0xffffffffu, dz32, off));
    }
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) {
        bred[0][warp] = drift;
        bred[1][warp] = zex;
        bred[2][warp] = nzg;
        bred[3][warp] = all;
        bred[4][warp] = dz32;
    }
    __syncthreads();
    if (tid == 0) {
        float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int w = 0; w < kResyncThreads / 32; w++)
            for (int q = 0; q < 5; q++)
                v[q] = fmaxf(v[q], bred[q][w]);
        if (need && rep)
            for (int q = 0; q < 5; q++)
                rep[5 * blockIdx.x + q] = v[q];
        unsigned long long *rd = red + (int64_t)isig * red_stride;
        for (int q = 0; q < 5; q++)
            atomicMax(&rd[q], (unsigned long long)__double_as_longlong((double)v[q]));
    }
}

// The resync with a few warps per tile (lane = column): the tiles of a long
// signal are many and each needs little arithmetic (a few nonzeros reach a
// 32-column tile at the optimum), so what bounds a tile is its chain of
// dependent memory round trips; small blocks keep many tiles in flight on an
// SM and need no barrier before the final reduction.  Block = WPT warps of
// one tile; warp q owns the float4 atom groups [q NG, (q+1) NG) of the
// by-lag table, and each lane loads the coefficients of NB nonzeros, and the
// state of its NG x 4 coordinates, in one round.  The nonzeros are read from
// the buckets in the same order as resync_kernel (bucket, then (k, column)),
// or, when a bucket overflowed or no lists are given, gathered from Z in that
// same order with ballots: results are identical either way.  Needs 2R+1 <=
// 32 buckets, R = ceil((L-1)/32) (L <= 481), and K <= 64 (at most 8 warps).
template <int NG>
__global__ void __launch_bounds__(256, 2)
    resync_warp_kernel(const SigDesc *__restrict__ sigs, Tiles tiles, const float *__restrict__ Ct,
                       const float *__restrict__ norms, int K, int L, int write_r,
                       unsigned long long *__restrict__ red, int red_stride,
                       unsigned char *__restrict__ dirty, float tol_mark,
                       const unsigned char *__restrict__ touched, float *__restrict__ rep,
                       NzLists lists)
{
    constexpr int KPT = 4 * NG;
    constexpr int NB = NG == 1 ? 8 : 4;  // nonzeros whose coefficients are loaded together
    constexpr unsigned kFullMask = 0xffffffffu;
    __shared__ float bred[5][32];
    __shared__ int s_need;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5, nwq = blockDim.x >> 5;
    const int64_t b = blockIdx.x;
    const int isig = tiles.sig[b];
    const SigDesc sd = sigs[isig];
    const int64_t Tz = sd.Tz, ld = sd.ld;
    float *__restrict__ const rr = sd.r;
    const float *__restrict__ const zz = sd.Z;
    const float *__restrict__ const b0p = sd.beta0;
    const int W2 = 2 * L - 1;
    const int G = (K + 3) / 4;  // float4 groups of the table
    const int g0 = wq * NG;     // this warp's first group
    const int64_t c0 = tiles.start[b];
    const int64_t t = c0 + lane;
    const int64_t tend = tiles.end && tiles.end[b] < Tz ? tiles.end[b] : Tz;
    const bool col_ok = t < tend;
    float drift = 0.f, zex = 0.f, nzg = 0.f, all = 0.f, dz32 = 0.f;
    // whether the tile must be recomputed: decided once per block (the
    // segment range of the tile takes two 64-bit divisions)
    if (threadIdx.x == 0)
        s_need = !(touched && rep) || tile_touched(sd, c0, touched);
    __syncthreads();
    const bool need = s_need != 0;
    if (!need) {
        if (lane == 0 && wq == 0) {  // the stored report of the unchanged tile (drift 0)
            zex = rep[5 * b + 1];
            nzg = rep[5 * b + 2];
            all = rep[5 * b + 3];
            dz32 = rep[5 * b + 4];
        }
    } else {
        // this lane's coordinates: its state first (one round trip for all)
        float b0v[KPT], rov[KPT], zv[KPT], nv[KPT];
        // 1 / ||D_k||^2 of the warp's KPT atoms: lane q computes atom q's
        const int kq = 4 * (g0 + (lane % KPT) / 4) + (lane % KPT) % 4;
        const float rn_lane = __frcp_rn(kq < K ? norms[kq] : 1.f);
#pragma unroll
        for (int q = 0; q < KPT; q++) {
            const int k = 4 * (g0 + q / 4) + (q % 4);
            const bool ok = col_ok && k < K;
            const int64_t ix = (int64_t)(ok ? k : 0) * ld + (ok ? t : 0);
            b0v[q] = ok ? b0p[ix] : 0.f;
            rov[q] = ok ? rr[ix] : 0.f;
            zv[q] = ok ? zz[ix] : 0.f;
            nv[q] = ok ? norms[k] : 1.f;
        }
        float acc_hi[KPT], acc_lo[KPT];
#pragma unroll
        for (int i = 0; i < KPT; i++) {
            acc_hi[i] = 0.f;
            acc_lo[i] = 0.f;
        }
        const float4 *Ct4 = reinterpret_cast<const float4 *>(Ct);
        // NB nonzeros (k, column, z) at a time: loads first, then the sums; a
        // nonzero out of this lane's window (z = 0 there) adds nothing
        // (column offsets relative to the tile start c0: 32-bit)
        auto add_batch = [&](const int (&kk)[NB], const int (&tc)[NB], const float (&z)[NB]) {
            float4 cv[NB][NG];
            float zz_[NB];
#pragma unroll
            for (int e = 0; e < NB; e++) {
                const int d = lane - tc[e] + (L - 1);
                const bool in = col_ok && z[e] != 0.f && d >= 0 && d < W2;
                zz_[e] = in ? z[e] : 0.f;
                const int base = (kk[e] * G + g0) * W2 + (in ? d : 0);
#pragma unroll
                for (int gi = 0; gi < NG; gi++)
                    cv[e][gi] = in && g0 + gi < G ? __ldg(Ct4 + base + gi * W2)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int e = 0; e < NB; e++)
                if (zz_[e] != 0.f) {
#pragma unroll
                    for (int gi = 0; gi < NG; gi++) {
                        df_add_prod(acc_hi[4 * gi], acc_lo[4 * gi], cv[e][gi].x, zz_[e]);
                        df_add_prod(acc_hi[4 * gi + 1], acc_lo[4 * gi + 1], cv[e][gi].y, zz_[e]);
                        df_add_prod(acc_hi[4 * gi + 2], acc_lo[4 * gi + 2], cv[e][gi].z, zz_[e]);
                        df_add_prod(acc_hi[4 * gi + 3], acc_lo[4 * gi + 3], cv[e][gi].w, zz_[e]);
                    }
                }
        };
        // buckets b-R .. b+R of the same problem: lane j holds bucket b-R+j
        const int R = (L - 1 + kResyncCols - 1) / kResyncCols;
        int cnt = 0;
        if (lists.count && lane <= 2 * R) {
            const int64_t bb = b - R + lane;
            const bool valid = bb >= 0 && bb < tiles.n && tiles.sig[bb] == isig &&
                               tiles.start[bb] == c0 + (int64_t)(lane - R) * kResyncCols;
            cnt = valid ? lists.count[bb] : 0;
        }
        const bool listed = lists.count && !__any_sync(kFullMask, cnt > kNzCap);
        if (listed) {
            // entries in bucket order: prefix of the counts over the lanes
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(kFullMask, incl, o);
                if (lane >= o)
                    incl += v;
            }
            const int total = __shfl_sync(kFullMask, incl, 31);
            const int excl = incl - cnt;
            for (int e0 = 0; e0 < total; e0 += 32) {
                // lane l fetches entry e0 + l: its bucket j is the last one with
                // excl_j <= e (empty buckets before it are passed over)
                const int e = e0 + lane;
                int j = 0;
                for (int q = 0; q <= 2 * R; q++)
                    if (e >= __shfl_sync(kFullMask, excl, q))
                        j = q;
                const int xj = __shfl_sync(kFullMask, excl, j);
                const uint2 v = e < total ? lists.ent[(b - R + j) * kNzCap + (e - xj)]
                                          : make_uint2(0u, 0u);
                // atom and column offset from c0 in one word: k << 16 | (offset + 1024)
                // (offsets lie in [-32 R, 32 R + 32), 2R + 1 <= 32)
                const int off = (j - R) * kResyncCols + (int)(v.x % kResyncCols);
                const unsigned pk = ((v.x / kResyncCols) << 16) | (unsigned)(off + 1024);
                const int m = total - e0 < 32 ? total - e0 : 32;
                for (int i0 = 0; i0 < m; i0 += NB) {
                    int kk[NB];
                    int tc[NB];
                    float z[NB];
#pragma unroll
                    for (int x = 0; x < NB; x++) {
                        const int src = i0 + x < m ? i0 + x : 0;
                        const unsigned px = __shfl_sync(kFullMask, pk, src);
                        const float zx = __uint_as_float(__shfl_sync(kFullMask, v.y, src));
                        kk[x] = (int)(px >> 16);
                        tc[x] = (int)(px & 0xffffu) - 1024;
                        z[x] = i0 + x < m ? zx : 0.f;
                    }
                    add_batch(kk, tc, z);
                }
            }
        } else {
            // from Z itself, bucket by bucket, (k, column) order by ballots;
            // every column of the problem counts here, also those no tile of
            // the table computes (a shard's halo)
            for (int q = 0; q <= 2 * R; q++) {
                const int64_t cb = c0 + (int64_t)(q - R) * kResyncCols;
                if (cb + kResyncCols <= 0 || cb >= Tz)
                    continue;
                const int64_t tq = cb + lane;
                const bool in = tq >= 0 && tq < Tz;
                for (int k = 0; k < K; k++) {
                    const float zq = in ? zz[(int64_t)k * ld + tq] : 0.f;
                    unsigned msk = __ballot_sync(kFullMask, zq != 0.f);
                    while (msk) {
                        int kk[NB];
                        int tc[NB];
                        float z[NB];
#pragma unroll
                        for (int x = 0; x < NB; x++) {
                            const int src = msk ? __ffs((int)msk) - 1 : 0;
                            const float zx = __shfl_sync(kFullMask, zq, src);
                            kk[x] = k;
                            tc[x] = (q - R) * kResyncCols + src;
                            z[x] = msk ? zx : 0.f;
                            msk &= msk - 1;
                        }
                        add_batch(kk, tc, z);
                    }
                }
            }
        }
        const float lam = sd.lam;
#pragma unroll
        for (int q = 0; q < KPT; q++) {
            const int k = 4 * (g0 + q / 4) + (q % 4);
            // every lane takes part in the shuffle (col_ok differs across the
            // lanes of a signal's last tile)
            const float rn = __shfl_sync(kFullMask, rn_lane, q);
            if (col_ok && k < K)
                resync_finish_v(sd, (int64_t)k * ld + t, t, b0v[q], rov[q], zv[q], nv[q], rn, rr,
                                acc_hi[q], acc_lo[q], lam, write_r, dirty, tol_mark, drift, zex,
                                nzg, all, dz32);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        drift = fmaxf(drift, __shfl_xor_sync(kFullMask, drift, off));
        zex = fmaxf(zex, __shfl_xor_sync(kFullMask, zex, off));
        nzg = fmaxf(nzg, __shfl_xor_sync(kFullMask, nzg, off));
        all = fmaxf(all, __shfl_xor_sync(kFullMask, all, off));
        dz32 = fmaxf(dz32, __shfl_xor_sync(kFullMask, dz32, off));
    }
    float v[5] = {drift, zex, nzg, all, dz32};
    if (nwq > 1) {
        if (lane == 0)
            for (int q = 0; q < 5; q++)
                bred[q][wq] = v[q];
        __syncthreads();
        if (wq == 0 && lane == 0)
            for (int w = 1; w < nwq; w++)
                for (int q = 0; q < 5; q++)
                    v[q] = fmaxf(v[q], bred[q][w]);
    }
    if (wq == 0 && lane == 0) {
        if (need && rep)
            for (int q = 0; q < 5; q++)
                rep[5 * b + q] = v[q];
        unsigned long long *rd = red + (int64_t)isig * red_stride;
        for (int q = 0; q < 5; q++)
            atomicMax(&rd[q], (unsigned long long)__double_as_longlong((double)v[q]));
    }
}

constexpr int kObjP = 8;    // channels accumulated per pass
constexpr int kObjCap = 64;  // nonzeros of one 32-column bucket held in shared memory
constexpr int kObjBuckets = kTile / 32 + (kMaxL - 1 + 31) / 32;

// acc[q] += D[q L] z for the channels q < np of a pass (double-float)
__device__ __forceinline__ void obj_add(float (&hi)[kObjP], float (&lo)[kObjP],
                                        const float *__restrict__ Dk, int np, int L, float z)
{
#pragma unroll
    for (int q = 0; q < kObjP; q++)
        if (q < np)
            df_add_prod(hi[q], lo[q], __ldg(Dk + q * L), z);
}

// Tile b (kTile samples of one problem): partials[2b] = sum over its samples of
// sum_p R[p][t]^2 with R = X - sum_k Z_k * D_k ((Z*D)[t] = sum_tau Z[t-tau] D[tau],
// Sec. 2), partials[2b+1] = sum of |Z| over its columns.  Without tables
// (sigs == NULL) the problem is `one` and tile b starts at b * kTile.
//
// The Z columns that reach the tile, [c0 - 32 R, c0 + kTile) with R =
// ceil((L-1)/32), are listed first in buckets of 32 columns (one warp per
// bucket, a ballot per atom row: entries in (k, column) order).  Warp w's
// samples [c0 + 32 w, c0 + 32 w + 32) are reached only by the columns of
// buckets w .. w + R, so each thread walks R + 1 buckets.  A bucket with more
// than kObjCap nonzeros is walked straight from Z in the same order.
// With lists (the buckets of the last resync, which saw this Z: same
// entries in the same order) a bucket inside the problem is copied from the
// resync tile starting at its first column, rtile_off[problem] + column / 32.
__global__ void __launch_bounds__(kTile, 5)
    objective_kernel(const float *__restrict__ D, const SigDesc *__restrict__ sigs, SigDesc one,
                     Tiles tiles, int K, int P, int L, const float *Zbase, const float *Zalt,
                     double *__restrict__ partials, NzLists lists,
                     const int64_t *__restrict__ rtile_off)
{
    static_assert(kObjCap == kNzCap && kResyncCols == 32, "resync buckets serve the objective");
    __shared__ uint2 ent[kObjBuckets][kObjCap];
    __shared__ int cnt[kObjBuckets];
    __shared__ double bsum[2][kTile / 32];
    const SigDesc sd = sigs ? sigs[tiles.sig[blockIdx.x]] : one;
    const float *Z = Zalt ? Zalt + (sd.Z - Zbase) : sd.Z;
    const int64_t Tz = sd.Tz, ld = sd.ld, T = Tz + L - 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c0 = sigs ? tiles.start[blockIdx.x] : (int64_t)blockIdx.x * kTile;
    int64_t c1 = c0 + kTile < T ? c0 + kTile : T;
    if (sigs && tiles.end && tiles.end[blockIdx.x] < c1)
        c1 = tiles.end[blockIdx.x];
    const int64_t t = c0 + tid;
    // Z columns that reach samples below c1 are below c1
    const int64_t zhi = c1 < Tz ? c1 : Tz;
    const int R = (L - 1 + 31) / 32;
    const int64_t cb0 = c0 - 32 * (int64_t)R;  // bucket j: columns [cb0 + 32 j, cb0 + 32 j + 32)
    const int nb = kTile / 32 + R;
    for (int j = warp; j < nb; j += kTile / 32) {
        const int64_t cbj = cb0 + 32 * (int64_t)j;
        if (lists.count && cbj >= 0 && cbj < zhi) {
            const int64_t rt = rtile_off[tiles.sig[blockIdx.x]] + cbj / kResyncCols;
            const int n = lists.count[rt];
            if (n <= kObjCap)
                for (int i = lane; i < n; i += 32)
                    ent[j][i] = lists.ent[rt * kNzCap + i];
            if (lane == 0)
                cnt[j] = n;
            continue;
        }
        const int64_t col = cbj + lane;
        const bool in = col >= 0 && col < zhi;
        int base = 0;
        for (int k0 = 0; k0 < K; k0 += kBucketBatch) {
            // kBucketBatch rows loaded together: one memory round trip
            float zv[kBucketBatch];
#pragma unroll
            for (int q = 0; q < kBucketBatch; q++)
                zv[q] = in && k0 + q < K ? Z[(int64_t)(k0 + q) * ld + col] : 0.f;
#pragma unroll
            for (int q = 0; q < kBucketBatch; q++) {
                const float z = zv[q];
                const unsigned m = __ballot_sync(0xffffffffu, z != 0.f);
                if (z != 0.f) {
                    const int pos = base + __popc(m & ((1u << lane) - 1u));
                    if (pos < kObjCap)
                        ent[j][pos] = make_uint2((unsigned)((k0 + q) * 32 + lane), __float_as_uint(z));
                }
                base += __popc(m);
            }
        }
        if (lane == 0)
            cnt[j] = base;
    }
    __syncthreads();

    // per thread: sum of squared residuals and of |Z| in double-float (the
    // FP64 pipe is narrow: only the per-warp totals are taken to FP64)
    float sq_h = 0.f, sq_l = 0.f, l1_h = 0.f, l1_l = 0.f;
    // |Z| of the tile's own columns [c0 + 32 w, ...) (bucket R + w), once each
    {
        const int j = R + warp;
        const int n = cnt[j];
        if (n <= kObjCap) {
            for (int i = lane; i < n; i += 32)
                df_add(l1_h, l1_l, fabsf(__uint_as_float(ent[j][i].y)));
        } else {
            const int64_t col = cb0 + 32 * (int64_t)j + lane;
            if (col >= 0 && col < zhi)
                for (int k = 0; k < K; k++)
                    df_add(l1_h, l1_l, fabsf(Z[(int64_t)k * ld + col]));
        }
    }
    for (int p0 = 0; p0 < P; p0 += kObjP) {
        float acc_hi[kObjP], acc_lo[kObjP];
#pragma unroll
        for (int q = 0; q < kObjP; q++) {
            acc_hi[q] = 0.f;
            acc_lo[q] = 0.f;
        }
        if (t < c1) {
            for (int j = warp; j <= warp + R; j++) {
                const int n = cnt[j];
                const int64_t cbj = cb0 + 32 * (int64_t)j;
                if (n <= kObjCap) {
                    for (int i = 0; i < n; i++) {
                        const uint2 v = ent[j][i];
                        const int tau = (int)(t - (cbj + (v.x & 31u)));
                        if (tau >= 0 && tau < L)
                            obj_add(acc_hi, acc_lo, D + ((int)(v.x >> 5) * P + p0) * L + tau,
                                    P - p0, L, __uint_as_float(v.y));
                    }
                } else {
                    for (int k = 0; k < K; k++)
                        for (int jj = 0; jj < 32; jj++) {
                            const int64_t tp = cbj + jj;
                            const int tau = (int)(t - tp);
                            if (tp < 0 || tp >= zhi || tau < 0 || tau >= L)
                                continue;
                            const float z = Z[(int64_t)k * ld + tp];
                            if (z != 0.f)
                                obj_add(acc_hi, acc_lo, D + (k * P + p0) * L + tau, P - p0, L, z);
                        }
                }
            }
#pragma unroll
            for (int q = 0; q < kObjP; q++)
                if (p0 + q < P)
                    df_add_sq_residual(sq_h, sq_l, sd.X[(int64_t)(p0 + q) * sd.ldx + t], acc_hi[q],
                                       acc_lo[q]);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const float a = __shfl_xor_sync(0xffffffffu, sq_h, off);
        const float b = __shfl_xor_sync(0xffffffffu, sq_l, off);
        const float c = __shfl_xor_sync(0xffffffffu, l1_h, off);
        const float e = __shfl_xor_sync(0xffffffffu, l1_l, off);
        df_add_df(sq_h, sq_l, a, b);
        df_add_df(l1_h, l1_l, c, e);
    }
    if (lane == 0) {
        bsum[0][warp] = (double)sq_h + (double)sq_l;
        bsum[1][warp] = (double)l1_h + (double)l1_l;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kTile / 32; w++) {
            a += bsum[0][w];
            b += bsum[1][w];
        }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

// Block i: fixed-order sum of problem i's tile partials, E_i = sq/2 + lam_i * l1
// (without tables: the one problem owns all ntiles tiles).
__global__ void objective_final_kernel(const double *__restrict__ partials,
                                       const int64_t *__restrict__ tile_off, int64_t ntiles,
                                       const SigDesc *__restrict__ sigs, double lam0,
                                       double *__restrict__ out)
{
    __shared__ double s[2][256];
    const int i = blockIdx.x;
    const int64_t j0 = tile_off ? tile_off[i] : 0, j1 = tile_off ? tile_off[i + 1] : ntiles;
    double a = 0.0, b = 0.0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        a += partials[2 * j];
        b += partials[2 * j + 1];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            s[0][threadIdx.x] += s[0][threadIdx.x + h];
            s[1][threadIdx.x] += s[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        out[i] = 0.5 * s[0][0] + (sigs ? sigs[i].lam_d : lam0) * s[1][0];
}

// max |beta0| over tile b's columns, into out[problem] (float bits).
__global__ void __launch_bounds__(kTile)
    signal_absmax_kernel(const SigDesc *__restrict__ sigs, Tiles tiles, int K,
                         unsigned int *__restrict__ out)
{
    const int i = tiles.sig[blockIdx.x];
    const SigDesc sd = sigs[i];
    const int64_t t = tiles.start[blockIdx.x] + threadIdx.x;
    float m = 0.f;
    if (t < sd.Tz)
        for (int k = 0; k < K; k++)
            m = fmaxf(m, fabsf(sd.beta0[(int64_t)k * sd.ld + t]));
    for (int off = 16; off > 0; off >>= 1)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0)
        atomicMax(&out[i], __float_as_uint(m));
}

__global__ void beta_from_r_kernel(const float *__restrict__ r, const float *__restrict__ Z,
                                   const float *__restrict__ norms, int K, int64_t Tz,
                                   float *__restrict__ out)
{
    const int64_t n = (int64_t)K * Tz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = fmaf(norms[i / Tz], Z[i], r[i]);
}

template <int KPT>
cudaError_t resync_launch(const SigDesc *sig, Tiles tiles, const float *Ct, const float *norms,
                          int K, int L, int write_r, unsigned long long *red, int red_stride,
                          unsigned char *dirty, float tol_mark, const unsigned char *touched,
                          float *rep, NzLists lists, cudaStream_t s)
{
    if (lists.count) {
        const int64_t blocks = (tiles.n + 7) / 8;
        nz_bucket_kernel<<<(unsigned)blocks, 256, 0, s>>>(sig, tiles, K, touched, lists);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    resync_kernel<KPT><<<(unsigned)tiles.n, kResyncThreads, 0, s>>>(
        sig, tiles, Ct, norms, K, L, write_r, red, red_stride, dirty, tol_mark, touched, rep,
        lists);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_resync(const SigDesc *sig, Tiles tiles, const float *Ct, const float *norms,
                          int K, int L, int write_r, unsigned long long *red, int red_stride,
                          unsigned char *dirty, float tol_mark, const unsigned char *touched,
                          float *rep, NzLists lists, cudaStream_t s)
{
    if (tiles.n <= 0)
        return cudaSuccess;
    const int G = (K + 3) / 4;  // float4 groups of atoms
    const int R = (L - 1 + kResyncCols - 1) / kResyncCols;
    if (2 * R + 1 <= 32 && G <= 16) {
        // a few warps per tile: NG groups per warp, ceil(G / NG) warps
        const int ng = G <= 1 ? 1 : 2;
        const int wpt = (G + ng - 1) / ng;
        if (lists.count) {
            const int64_t blocks = (tiles.n + 7) / 8;
            nz_bucket_kernel<<<(unsigned)blocks, 256, 0, s>>>(sig, tiles, K, touched, lists);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess)
                return e;
        }
#define CSC_RESYNC_W(N) \
    resync_warp_kernel<N><<<(unsigned)tiles.n, 32 * wpt, 0, s>>>(                            \
        sig, tiles, Ct, norms, K, L, write_r, red, red_stride, dirty, tol_mark, touched, rep, \
        lists);                                                                                \
    return cudaGetLastError()
        if (ng == 1) {
            CSC_RESYNC_W(1);
        }
        CSC_RESYNC_W(2);
#undef CSC_RESYNC_W
    }
    // float4 groups of atoms per thread group
    const int ngb = (G + kResyncGroups - 1) / kResyncGroups;
#define CSC_RESYNC(N) \
    return resync_launch<N>(sig, tiles, Ct, norms, K, L, write_r, red, red_stride, dirty, \
                            tol_mark, touched, rep, lists, s)
    if (ngb <= 1)
        CSC_RESYNC(4);
    if (ngb <= 2)
        CSC_RESYNC(8);
    if (ngb <= 4)
        CSC_RESYNC(16);
    if (ngb <= 8)  // K <= 256 (csc_setup, the server)
        CSC_RESYNC(32);
#undef CSC_RESYNC
    return cudaErrorInvalidValue;
}

cudaError_t launch_beta_from_r(const float *r, const float *Z, const float *norms, int K,
                               int64_t Tz, float *out, cudaStream_t s)
{
    const int64_t n = (int64_t)K * Tz;
    const int64_t grid = (n + 255) / 256;
    beta_from_r_kernel<<<(unsigned)(grid < 152 * 64 ? grid : 152 * 64), 256, 0, s>>>(r, Z, norms,
                                                                                   K, Tz, out);
    return cudaGetLastError();
}

cudaError_t launch_objective(const float *D, const SigDesc *sig, int n, Tiles tiles,
                             const int64_t *tile_off, int K, int P, int L, const float *Zbase,
                             const float *Zalt, double *partials, double *out, cudaStream_t s,
                             NzLists lists, const int64_t *rtile_off)
{
    if (tiles.n <= 0)
        return cudaSuccess;
    objective_kernel<<<(unsigned)tiles.n, kTile, 0, s>>>(D, sig, SigDesc{}, tiles, K, P, L, Zbase,
                                                         Zalt, partials, lists, rtile_off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    objective_final_kernel<<<n, 256, 0, s>>>(partials, tile_off, tiles.n, sig, 0.0, out);
    return cudaGetLastError();
}

cudaError_t launch_objective_single(const float *D, const SigDesc &one, int K, int P, int L,
                                    double *partials, double *out, cudaStream_t s)
{
    const int64_t ntiles = (one.Tz + L - 1 + kTile - 1) / kTile;
    objective_kernel<<<(unsigned)ntiles, kTile, 0, s>>>(D, nullptr, one, Tiles{nullptr, nullptr, 0},
                                                        K, P, L, nullptr, nullptr, partials,
                                                        NzLists{nullptr, nullptr}, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    objective_final_kernel<<<1, 256, 0, s>>>(partials, nullptr, ntiles, nullptr, one.lam_d, out);
    return cudaGetLastError();
}

cudaError_t launch_signal_absmax(const SigDesc *sig, Tiles tiles, int K, unsigned int *out,
                                 cudaStream_t s)
{
    if (tiles.n <= 0)
        return cudaSuccess;
    signal_absmax_kernel<<<(unsigned)tiles.n, kTile, 0, s>>>(sig, tiles, K, out);
    return cudaGetLastError();
}

}  // namespace csc
