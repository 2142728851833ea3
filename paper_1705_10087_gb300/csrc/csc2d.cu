// The 2-D variant (include/csc2d.h): images cut into row bands.
//
// The paper's conclusion names images cut along one direction as the way to
// keep the 1-D analysis: a band of rows has a neighbour above and one below,
// exactly as a 1-D segment has one on each side.  Every definition is that of
// Sec. 2.1 with 2-D lags.  With image X[P][H][W], atoms D[K][P][h][w] and
// activations Z[K][Hz][Wz] (Hz = H-h+1, Wz = W-w+1, "valid" placement):
//   beta0_k[i][j]  = sum_{p,u,v} D[k][p][u][v] X[p][i+u][j+v]            (Alg. 1 init)
//   C[k][k0][a][b] = sum_{p,u,v} D[k][p][u][v] D[k0][p][u+a-h+1][v+b-w+1] (S of Eq. beta_up)
// and the solver keeps r = beta - ||D_k||^2 Z as in 1-D (csc_internal.cuh):
// an update dZ of Z_k0[i0][j0] changes r_k[i][j] by -C[k][k0][i-i0+h-1][j-j0+w-1] dZ
// for every (k, i, j) of the (2h-1) x (2w-1) window, own coordinate included.
//
// Tiles: row band m of M covers rows [floor(m Hz / M), floor((m+1) Hz / M)),
// column block n of N the columns [floor(n Wz / N), floor((n+1) Wz / N)).
// Each axis gets the 1-D phase count (cr over rows, cc over columns, so that
// (cr-1) times the narrowest band is at least 2h-2 rows and likewise for the
// columns), and tile (m, n) runs in phase (m mod cr) cc + (n mod cc): two
// co-active tiles are separated by at least 2h-2 rows or 2w-2 columns, their
// windows never meet, and each phase equals a sequential run of its tiles.
// N = 1 is the paper's cut along one axis (bands only); more column blocks
// give more co-active tiles, which one GPU needs (a 512 x 512 image with
// 8 x 8 atoms has 18 co-active bands but 324 co-active tiles of 14 x 14).
// One thread block per active tile: it keeps, per position (i, j) of its
// tile, the best coordinate over k as a 64-bit key (|Delta Z| bits, ~flat
// index and the sign of Delta Z; ties to the lowest (k Hz + i) Wz + j) in
// shared memory, with r and Z of the tile staged there too when they fit, and
// repeats block argmax (a shared atomicMax per warp, one barrier) -> update
// -> re-evaluation of the window's positions, writing the window positions
// outside its tile (idle neighbours) with atomicAdd and each new Z value to
// global memory when it is applied.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "csc2d.h"
#include "csc_internal.cuh"
#include "host_util.cuh"

using namespace csc;

int csc_record_error(int code, const char *fmt, ...);

namespace {

#define C2_CUDA(expr)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return csc_record_error(e_ == cudaErrorMemoryAllocation ? CSC_ENOMEM : CSC_ECUDA, \
                                    "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),   \
                                    __FILE__, __LINE__);                                     \
    } while (0)

constexpr int kB2 = 256;        // threads of a tile block
// updates per tile visit by default: a launch lasts as long as its busiest
// tile, so short visits keep the 324 co-active tiles of a 512 x 512 image
// (8 x 8 atoms) in step (measured on an earlier build: 6.2 ms at 8, 6.6 at
// 16, 8.1 at 32, 23 ms when every visit runs to local convergence)
constexpr int kAutoVisit2d = 8;
constexpr int kSweepBatch = 4;  // tile sweeps launched per read-back of their update counts
constexpr int kMaxK2 = 64;      // atoms (one bit each in a 64-bit mask)
constexpr int kMaxWin = 4096;   // (2h-1)(2w-1) window positions
constexpr int kTile2 = 32;      // columns per resync / objective tile
constexpr int kList2 = 2048;    // nonzeros gathered per round

struct Dims {
    int K, P, h, w;
    int64_t H, W, Hz, Wz;
};

// ---------------------------------------------------------------- setup

// C (by lag, float4 groups of atoms): Ct[((k0 * KQ + q) * A + lag) * 4 + e] =
// C[k = 4q+e][k0][a][b], lag = a (2w-1) + b, A = (2h-1)(2w-1).  FP64 sums.
__global__ void dtd2d_kernel(const float *__restrict__ D, Dims d, int KQ, float *__restrict__ Ct,
                             float *__restrict__ norms)
{
    const int H2 = 2 * d.h - 1, W2 = 2 * d.w - 1, A = H2 * W2;
    const int64_t n = (int64_t)d.K * KQ * A * 4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(i & 3);
        const int64_t rest = i >> 2;
        const int lag = (int)(rest % A);
        const int64_t kq = rest / A;
        const int q = (int)(kq % KQ), k0 = (int)(kq / KQ);
        const int k = 4 * q + e;
        double acc = 0.0;
        if (k < d.K) {
            const int da = lag / W2 - (d.h - 1), db = lag % W2 - (d.w - 1);
            for (int p = 0; p < d.P; p++)
                for (int u = 0; u < d.h; u++) {
                    const int u2 = u + da;
                    if (u2 < 0 || u2 >= d.h)
                        continue;
                    for (int v = 0; v < d.w; v++) {
                        const int v2 = v + db;
                        if (v2 < 0 || v2 >= d.w)
                            continue;
                        acc += (double)D[(((int64_t)k * d.P + p) * d.h + u) * d.w + v] *
                               (double)D[(((int64_t)k0 * d.P + p) * d.h + u2) * d.w + v2];
                    }
                }
            if (k == k0 && lag == (d.h - 1) * W2 + (d.w - 1))
                norms[k] = (float)acc;
        }
        Ct[i] = (float)acc;
    }
}

// beta0 (and r = beta0 for Z = 0) in double-float sums rounded once (the
// FP64 pipe of GB300 is narrow); max |beta0| and sum X^2 (E(0) = sum X^2 / 2).
__global__ void dtx2d_kernel(const float *__restrict__ D, const float *__restrict__ X, Dims d,
                             float *__restrict__ beta0, float *__restrict__ r,
                             unsigned *__restrict__ absmax, double *__restrict__ x2)
{
    const int64_t n = (int64_t)d.K * d.Hz * d.Wz;
    float amax = 0.f;
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = o % d.Wz, i = (o / d.Wz) % d.Hz;
        const int k = (int)(o / (d.Wz * d.Hz));
        float hi = 0.f, lo = 0.f;
        for (int p = 0; p < d.P; p++)
            for (int u = 0; u < d.h; u++) {
                const float *xr = X + ((int64_t)p * d.H + i + u) * d.W + j;
                const float *dr = D + (((int64_t)k * d.P + p) * d.h + u) * d.w;
                for (int v = 0; v < d.w; v++)
                    df_add_prod(hi, lo, __ldg(dr + v), __ldg(xr + v));
            }
        const float b = __fadd_rn(hi, lo);
        beta0[o] = b;
        r[o] = b;
        amax = fmaxf(amax, fabsf(b));
    }
    double s = 0.0;
    const int64_t nx = (int64_t)d.P * d.H * d.W;
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < nx;
         o += (int64_t)gridDim.x * blockDim.x)
        s += (double)X[o] * (double)X[o];
    for (int off = 16; off > 0; off >>= 1) {
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
        s += __shfl_xor_sync(0xffffffffu, s, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(absmax, __float_as_uint(amax));
        atomicAdd(x2, s);
    }
}

// ---------------------------------------------------------------- phase

struct TileParams {
    float *r, *Z;
    const float *Ct, *norms;
    const int64_t *row_s;    // [Mr+1] first row of each row band
    const int64_t *col_s;    // [Mc+1] first column of each column block
    const int *list;         // tiles of this phase, m * Mc + n
    unsigned char *dirty;    // [Mr * Mc]
    long long *upd;          // [1] updates of this sweep
    double *dec;             // [1] objective decrease (Prop. A.1)
    Dims d;
    int Mr, Mc, KQ, u;
    int max_pos;             // positions of the largest tile (shared-memory layout)
    float lam, tol;
};

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
    unsigned hi = (unsigned)(v >> 32);
    const unsigned hmax = __reduce_max_sync(0xffffffffu, hi);
    unsigned lo = hi == hmax ? (unsigned)v : 0u;
    const unsigned lmax = __reduce_max_sync(0xffffffffu, lo);
    return ((unsigned long long)hmax << 32) | lmax;
}

// Shared-memory layout of a tile block (bytes, 16-aligned pieces): per
// position its cached key and candidate Z'; with STAGE also r
// and Z of the tile, position-major with an odd row of ks = K | 1 floats.
struct TileLayout {
    size_t key, cz, r, z, total;
    __host__ __device__ TileLayout(int K, int npos, bool stage)
    {
        size_t o = 0;
        key = o;
        o = up(o + 8 * (size_t)npos);
        cz = o;
        o = up(o + 4 * (size_t)npos);
        r = o;
        if (stage)
            o = up(o + 4 * (size_t)(K | 1) * npos);
        z = o;
        if (stage)
            o = up(o + 4 * (size_t)(K | 1) * npos);
        total = o;
    }
    __host__ __device__ static size_t up(size_t x) { return (x + 15) & ~(size_t)15; }
};

// One visit of a tile (row band m x column block n) per block.  Position
// (i, j) belongs to the thread (slot(i, j) mod kB2), slot(i, j) = (i mod
// (2h-1)) (2w-1) + (j mod (2w-1)): the (2h-1) x (2w-1) positions of an
// update window have distinct slots, so the window's positions go to
// distinct threads, and each position of the tile is only ever written, and
// its key re-evaluated, by its owner (no barrier between an update and the
// next argmax).  Positions of the window outside the tile belong to idle
// neighbours of this phase: their r is changed with atomicAdd.
// (three blocks per SM: the 324 co-active tiles of a 512 x 512 image with
// 8 x 8 atoms are resident at once, without spills)
template <bool STAGE>
__global__ void __launch_bounds__(kB2, 3) tile_kernel(TileParams tp)
{
    extern __shared__ __align__(16) unsigned char sm[];
    // the block's best key of update i is reduced into s_best[i & 3] (a 64-bit
    // shared atomicMax per warp); slot (i + 2) & 3, last read in update i - 2,
    // is cleared during update i
    __shared__ unsigned long long s_best[4];
    __shared__ float s_nrm[kMaxK2], s_rn[kMaxK2];
    __shared__ double s_dec[kB2 / 32];
    const int tile = tp.list[blockIdx.x];
    if (!tp.dirty[tile])
        return;  // uniform: every thread reads the same flag
    const int m = tile / tp.Mc, n = tile % tp.Mc;
    const Dims d = tp.d;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i_lo = tp.row_s[m], i_hi = tp.row_s[m + 1];
    const int64_t j_lo = tp.col_s[n], j_hi = tp.col_s[n + 1];
    const int th = (int)(i_hi - i_lo), tw = (int)(j_hi - j_lo);
    const int npos = th * tw;
    const int64_t Wz = d.Wz, HWz = d.Hz * d.Wz;
    const int K = d.K, ks = K | 1;
    const int H2 = 2 * d.h - 1, W2 = 2 * d.w - 1, A = H2 * W2;
    const TileLayout lay(K, tp.max_pos, STAGE);
    unsigned long long *key = reinterpret_cast<unsigned long long *>(sm + lay.key);
    float *cz = reinterpret_cast<float *>(sm + lay.cz);
    float *rs = reinterpret_cast<float *>(sm + lay.r);
    float *zs = reinterpret_cast<float *>(sm + lay.z);
    const float lam = tp.lam;
    for (int k = tid; k < K; k += kB2) {
        s_nrm[k] = tp.norms[k];
        s_rn[k] = __frcp_rn(tp.norms[k]);
    }
    if (tid < 4)
        s_best[tid] = 0ull;
    // element k of tile position p = (i - i_lo) tw + (j - j_lo)
    auto rref = [&](int p, int64_t i, int64_t j, int k) -> float & {
        return STAGE ? rs[p * ks + k] : tp.r[k * HWz + i * Wz + j];
    };
    auto zref = [&](int p, int64_t i, int64_t j, int k) -> float & {
        return STAGE ? zs[p * ks + k] : tp.Z[k * HWz + i * Wz + j];
    };
    if (STAGE)
        for (int p = tid; p < npos; p += kB2) {
            const int64_t i = i_lo + p / tw, j = j_lo + p % tw;
            for (int k = 0; k < K; k++) {
                rs[p * ks + k] = tp.r[k * HWz + i * Wz + j];
                zs[p * ks + k] = tp.Z[k * HWz + i * Wz + j];
            }
        }
    __syncthreads();
    // best coordinate over k of position p = (ii, jj) = (i - i_lo, j - j_lo),
    // cached as a key (|dZ| bits, ~(idx << 1 | sign of dZ)) with the bit fields
    // idx = k << (ib + jb) | ii << jb | jj (ib, jb: bits of th - 1 and tw - 1;
    // 6 + ib + jb < 32, checked by the host): ties go to the lowest (k, i, j),
    // i.e. the lowest (k Hz + i) Wz + j, and the key alone gives dZ exactly
    const int jbits = tw > 1 ? 32 - __clz(tw - 1) : 0;
    const int kshift = (th > 1 ? 32 - __clz(th - 1) : 0) + jbits;
    auto eval = [&](int p, int64_t i, int64_t j) {
        float best = -1.f, bz = 0.f, bd = 0.f;
        int bk = 0;
        for (int k = 0; k < K; k++) {
            const float r = rref(p, i, j, k), z = zref(p, i, j, k);
            if (z == 0.f && fabsf(r) <= lam)
                continue;
            float zn, dd;
            coord_step(r, z, s_nrm[k], s_rn[k], lam, &zn, &dd);
            if (fabsf(dd) > best) {
                best = fabsf(dd);
                bk = k;
                bz = zn;
                bd = dd;
            }
        }
        const unsigned idx = ((unsigned)bk << kshift) | ((unsigned)(i - i_lo) << jbits) | (unsigned)(j - j_lo);
        const unsigned flat = (idx << 1) | (bd < 0.f ? 1u : 0u);
        key[p] = best > 0.f ? ((unsigned long long)__float_as_uint(best) << 32) | (unsigned)(~flat)
                            : 0ull;
        cz[p] = bz;
    };
    // this thread's window slots q = tid, tid + kB2, ... < A as (a, b) =
    // (q / W2, q % W2), stepped without dividing
    const int a_step = kB2 / W2, b_step = kB2 - a_step * W2;
    auto for_slots = [&](auto &&f) {
        int a = tid / W2, b = tid - (tid / W2) * W2;
        for (int q = tid; q < A; q += kB2) {
            f(a, b);
            a += a_step;
            b += b_step;
            if (b >= W2) {
                b -= W2;
                a++;
            }
        }
    };
    // x mod m for x in [-m, 2m)
    auto wrap = [](int x, int m) { return x < 0 ? x + m : (x >= m ? x - m : x); };
    const int il = (int)(i_lo % H2), jl = (int)(j_lo % W2);
    // slot (a, b) holds the tile's rows i == a (mod H2) and columns j == b
    // (mod W2): ii from (a - i_lo) mod H2 in steps of H2, jj likewise
    auto for_positions = [&](int a, int b, auto &&f) {
        for (int ii = wrap(a - il, H2); ii < th; ii += H2)
            for (int jj = wrap(b - jl, W2); jj < tw; jj += W2)
                f(ii * tw + jj, i_lo + ii, j_lo + jj);
    };
    for_slots([&](int a, int b) { for_positions(a, b, eval); });
    int nupd = 0;
    int64_t imin = i_hi, imax = i_lo - 1, jmin = j_hi, jmax = j_lo - 1;
    float decrease = 0.f;
    bool capped = false;
    const float4 *Ct4 = reinterpret_cast<const float4 *>(tp.Ct);
    for (int it = 0;; it++) {
        unsigned long long my = 0ull;
        for_slots([&](int a, int b) {
            for_positions(a, b, [&](int p, int64_t, int64_t) {
                const unsigned long long kk = key[p];
                my = kk > my ? kk : my;
            });
        });
        const unsigned long long wm = warp_max_u64(my);
        if (lane == 0 && wm != 0ull)
            atomicMax(&s_best[it & 3], wm);
        if (tid == 0)
            s_best[(it + 2) & 3] = 0ull;
        __syncthreads();
        const unsigned long long bk = s_best[it & 3];
        const float adz = __uint_as_float((unsigned)(bk >> 32));
        if (!(adz >= tp.tol))
            break;
        if (it >= tp.u) {
            capped = true;
            break;
        }
        // the winner and dZ = +-|dZ| from its key.  Only the position's owner
        // reads Z' from the position cache: the owner rewrites that cache later
        // in this update, and another thread's read would race it
        const unsigned flat = ~(unsigned)bk, idx = flat >> 1;
        const float delta = (flat & 1u) ? -adz : adz;
        const int k0 = (int)(idx >> kshift);
        const int ii0 = (int)((idx & ((1u << kshift) - 1u)) >> jbits);
        const int jj0 = (int)(idx & ((1u << jbits) - 1u));
        const int64_t i0 = i_lo + ii0, j0 = j_lo + jj0;
        const int64_t ib = i0 - (d.h - 1), jb = j0 - (d.w - 1);
        // Eq. beta_up (r form) on the window: slot (a, b) holds the window
        // position ib + oi, jb + oj with oi = (a - ib) mod H2 = (a - i_lo +
        // h - 1 - ii0) mod H2 and oj likewise (ii0 < th <= H2 for the
        // automatic tiles: one wrap; larger tiles take a remainder)
        for_slots([&](int a, int b) {
            int oi = wrap(a - il + d.h - 1, H2) - ii0, oj = wrap(b - jl + d.w - 1, W2) - jj0;
            if (th > H2)
                oi %= H2;
            if (tw > W2)
                oj %= W2;
            oi = oi < 0 ? oi + H2 : oi;
            oj = oj < 0 ? oj + W2 : oj;
            const int64_t i = ib + oi, j = jb + oj;
            if (i < 0 || i >= d.Hz || j < 0 || j >= Wz)
                return;
            const int lag = oi * W2 + oj;
            const bool own = i >= i_lo && i < i_hi && j >= j_lo && j < j_hi;
            const int p = own ? (int)(i - i_lo) * tw + (int)(j - j_lo) : 0;
            if (own && i == i0 && j == j0) {
                // Prop. A.1 from the owner's r before this update touches it:
                // dZ (r - n dZ / 2) + lam (|z| - |u|)
                const float znew = cz[p], nk = s_nrm[k0], z = znew - delta;
                const float r0 = rref(p, i, j, k0);
                decrease += delta * (r0 - 0.5f * nk * delta) + lam * (fabsf(z) - fabsf(znew));
                zref(p, i, j, k0) = znew;
                if (STAGE)
                    tp.Z[k0 * HWz + i * Wz + j] = znew;  // (the write-back copies r only)
            }
            for (int g = 0; g < tp.KQ; g++) {
                const float4 c = __ldg(Ct4 + ((int64_t)k0 * tp.KQ + g) * A + lag);
                const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int k = 4 * g + e;
                    if (k >= K)
                        break;
                    if (own) {
                        float &rv = rref(p, i, j, k);
                        rv = fmaf(-cv[e], delta, rv);
                    } else {
                        atomicAdd(tp.r + k * HWz + i * Wz + j, -cv[e] * delta);
                    }
                }
            }
            if (own)
                eval(p, i, j);
        });
        nupd++;
        imin = i0 < imin ? i0 : imin;
        imax = i0 > imax ? i0 : imax;
        jmin = j0 < jmin ? j0 : jmin;
        jmax = j0 > jmax ? j0 : jmax;
    }
    if (STAGE && nupd > 0) {
        __syncthreads();  // every owner's last update is in shared memory
        for (int p = tid; p < npos; p += kB2) {
            const int64_t i = i_lo + p / tw, j = j_lo + p % tw;
            for (int k = 0; k < K; k++)
                tp.r[k * HWz + i * Wz + j] = rs[p * ks + k];
        }
    }
    for (int off = 16; off > 0; off >>= 1)
        decrease += __shfl_xor_sync(0xffffffffu, decrease, off);
    if (lane == 0)
        s_dec[warp] = (double)decrease;
    __syncthreads();
    if (tid == 0) {
        double dsum = 0.0;
        for (int q = 0; q < kB2 / 32; q++)
            dsum += s_dec[q];
        tp.dirty[tile] = capped ? 1 : 0;
        if (nupd > 0) {
            // tiles the windows reached need a visit again
            const int64_t rlo = imin - (d.h - 1), rhi = imax + (d.h - 1);
            const int64_t clo = jmin - (d.w - 1), chi = jmax + (d.w - 1);
            int m0 = m, m1 = m, n0 = n, n1 = n;
            while (m0 > 0 && tp.row_s[m0] > rlo)
                m0--;
            while (m1 + 1 < tp.Mr && tp.row_s[m1 + 1] <= rhi)
                m1++;
            while (n0 > 0 && tp.col_s[n0] > clo)
                n0--;
            while (n1 + 1 < tp.Mc && tp.col_s[n1 + 1] <= chi)
                n1++;
            for (int mm = m0; mm <= m1; mm++)
                for (int nn = n0; nn <= n1; nn++)
                    if (mm != m || nn != n)
                        tp.dirty[mm * tp.Mc + nn] = 1;
            atomicAdd(reinterpret_cast<unsigned long long *>(tp.upd), (unsigned long long)nupd);
            atomicAdd(tp.dec, dsum);
        }
    }
}

// ---------------------------------------------------------------- exact checks

// Nonzeros of Z in rows [r0, r1) x columns [c0, c1) (at most kList2
// elements: the callers cut their regions into column chunks that fit), in
// (k, row, column) order, compacted into list; returns the count (the same
// in every thread).  Block-wide barriers.  The exact checks use it where the
// nonzero buckets below cannot serve a region.
struct NZ2 {
    int k;
    int i, j;
    float z;
};

__device__ int compact2(const float *__restrict__ Z, const Dims &d, int64_t r0, int64_t r1,
                        int64_t c0, int64_t c1, NZ2 *list, int *wc)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int64_t rows = r1 - r0, cols = c1 - c0;
    const int64_t n = (int64_t)d.K * rows * cols;
    int base = 0;
    for (int64_t a = 0; a < n; a += blockDim.x) {
        const int64_t i = a + tid;
        float z = 0.f;
        int k = 0;
        int64_t ii = 0, jj = 0;
        if (i < n) {
            k = (int)(i / (rows * cols));
            ii = r0 + (i / cols) % rows;
            jj = c0 + i % cols;
            z = Z[((int64_t)k * d.Hz + ii) * d.Wz + jj];
        }
        const unsigned mask = __ballot_sync(0xffffffffu, z != 0.f);
        if (lane == 0)
            wc[warp] = __popc(mask);
        __syncthreads();
        int off = base, tot = base;
        for (int q = 0; q < nw; q++) {
            off += q < warp ? wc[q] : 0;
            tot += wc[q];
        }
        if (z != 0.f)
            list[off + __popc(mask & ((1u << lane) - 1u))] = NZ2{k, (int)ii, (int)jj, z};
        __syncthreads();
        base = tot;
    }
    return base;
}

// Nonzero buckets of Z per (row i, kTile2-column tile t), bucket b = i ntc + t:
// count[b] = the tile's nonzeros over all atoms (may exceed kBucket2), ent[b
// kBucket2 + e] the first kBucket2 of them in (k, column) order.  Built once
// per exact refresh; the final objective reads those of the last refresh (Z
// is the same).
constexpr int kBucket2 = 16;
constexpr int kGather2 = 256;  // buckets one block gathers at most
struct Buckets2 {
    const int *count;
    const NZ2 *ent;
    int64_t ntc;  // tiles per row, ceil(Wz / kTile2)
};

// One warp per bucket (blocks of whole warps: a warp exits as a whole).
__global__ void __launch_bounds__(256)
    bucket2d_kernel(const float *__restrict__ Z, Dims d, int64_t ntc, int *__restrict__ count,
                    NZ2 *__restrict__ ent)
{
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= d.Hz * ntc)
        return;
    const int64_t i = b / ntc, j = (b % ntc) * kTile2 + lane;
    int n = 0;
    for (int k = 0; k < d.K; k++) {
        const float z = j < d.Wz ? Z[((int64_t)k * d.Hz + i) * d.Wz + j] : 0.f;
        const unsigned m = __ballot_sync(0xffffffffu, z != 0.f);
        const int pos = n + __popc(m & ((1u << lane) - 1u));
        if (z != 0.f && pos < kBucket2)
            ent[b * kBucket2 + pos] = NZ2{k, (int)i, (int)j, z};
        n += __popc(m);
    }
    if (lane == 0)
        count[b] = n;
}

// Fills list with the nonzeros of the buckets of rows [r0, r1) and of the
// tiles holding columns [c0, c1) (r0 < r1, c0 < c1), in (row, tile, k,
// column) order: a superset of the region's nonzeros (callers skip what lies
// outside their windows).  Returns their count, or -1 when a bucket
// overflowed or the buckets are more than kGather2 or the nonzeros more than
// kList2; the same in every thread.  s_cnt [kGather2], s_off [kGather2 + 1],
// s_flag: shared scratch.  Block-wide barriers.
__device__ int gather2(const Buckets2 &bk, int64_t r0, int64_t r1, int64_t c0, int64_t c1,
                       NZ2 *list, int *s_cnt, int *s_off, int *s_flag)
{
    const int tid = threadIdx.x;
    const int64_t t0 = c0 / kTile2;
    const int nt = (int)((c1 - 1) / kTile2 + 1 - t0);
    if ((r1 - r0) * nt > kGather2)
        return -1;
    const int nb = (int)((r1 - r0) * nt);
    auto bucket = [&](int q) { return (r0 + q / nt) * bk.ntc + t0 + q % nt; };
    for (int q = tid; q < nb; q += blockDim.x)
        s_cnt[q] = bk.count[bucket(q)];
    __syncthreads();
    if (tid < 32) {
        // lane l takes buckets [l per, (l + 1) per): a sum, a warp scan, offsets
        const int per = (nb + 31) / 32, qa = min(nb, tid * per), qb = min(nb, qa + per);
        int sum = 0;
        bool over = false;
        for (int q = qa; q < qb; q++) {
            over |= s_cnt[q] > kBucket2;
            sum += s_cnt[q];
        }
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o)
                incl += v;
        }
        over = __any_sync(0xffffffffu, over);
        int run = incl - sum;
        for (int q = qa; q < qb; q++) {
            s_off[q] = run;
            run += s_cnt[q];
        }
        if (tid == 31) {
            s_off[nb] = incl;
            *s_flag = over || incl > kList2 ? 1 : 0;
        }
    }
    __syncthreads();
    if (*s_flag)
        return -1;
    const int total = s_off[nb];
    for (int q = tid; q < total; q += blockDim.x) {
        // the bucket of entry q: the last b with s_off[b] <= q
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= q)
                lo = mid;
            else
                hi = mid - 1;
        }
        list[q] = bk.ent[bucket(lo) * kBucket2 + (q - s_off[lo])];
    }
    __syncthreads();
    return total;
}

// r = beta0 - sum C Z (FP64 sums) on one row and kTile2 columns per block
// (threads: 32 columns x 8 atom groups), and the optimality report as in 1-D:
// red[0] drift, red[3] max |Delta Z| (no floor), red[4] the coordinate step on
// the refreshed state (with the float32 floor); write_r = 0 leaves r alone.
__global__ void __launch_bounds__(256)
    resync2d_kernel(const float *__restrict__ beta0, float *__restrict__ r,
                    const float *__restrict__ Z, const float *__restrict__ Ct,
                    const float *__restrict__ norms, Dims d, int KQ, float lam, int write_r,
                    Buckets2 bk, unsigned long long *__restrict__ red)
{
    __shared__ NZ2 list[kList2];
    __shared__ int wc[8];
    __shared__ float bred[3][8];
    __shared__ int s_cnt[kGather2], s_off[kGather2 + 1], s_flag;
    const int tid = threadIdx.x, col = tid & 31, grp = tid >> 5;
    const int64_t ntc = (d.Wz + kTile2 - 1) / kTile2;
    const int64_t i = blockIdx.x / ntc, j0 = (blockIdx.x % ntc) * kTile2, j = j0 + col;
    const int H2 = 2 * d.h - 1, W2 = 2 * d.w - 1, A = H2 * W2;
    const int64_t r0 = max((int64_t)0, i - (d.h - 1)), r1 = min(d.Hz, i + d.h);
    const int64_t c0 = max((int64_t)0, j0 - (d.w - 1)), c1 = min(d.Wz, j0 + kTile2 + d.w - 1);
    constexpr int kPer = (kMaxK2 + 7) / 8;
    float acc_hi[kPer], acc_lo[kPer];  // double-float sums of C z
#pragma unroll
    for (int q = 0; q < kPer; q++) {
        acc_hi[q] = 0.f;
        acc_lo[q] = 0.f;
    }
    // sum C z over the listed nonzeros whose window holds (i, j)
    auto accumulate = [&](int n) {
        if (j >= d.Wz)
            return;
        for (int q = 0; q < n; q++) {
            const NZ2 e = list[q];
            const int a = (int)(i - e.i) + (d.h - 1), b = (int)(j - e.j) + (d.w - 1);
            if (a < 0 || a >= H2 || b < 0 || b >= W2)
                continue;
            const int lag = a * W2 + b;
#pragma unroll
            for (int t = 0; t < kPer; t++) {
                const int k = grp + 8 * t;
                if (k < d.K)
                    df_add_prod(acc_hi[t], acc_lo[t],
                                __ldg(Ct + ((((int64_t)e.k * KQ + (k >> 2)) * A + lag) << 2) +
                                      (k & 3)),
                                e.z);
            }
        }
    };
    // the region's nonzeros from the buckets, else compacted from Z in column
    // chunks whose K x rows x chunk elements fit the list
    const int nl = bk.count ? gather2(bk, r0, r1, c0, c1, list, s_cnt, s_off, &s_flag) : -1;
    if (nl >= 0) {
        accumulate(nl);
    } else {
        const int64_t chunk = max((int64_t)1, (int64_t)kList2 / ((int64_t)d.K * (r1 - r0)));
        for (int64_t ca = c0; ca < c1; ca += chunk) {
            const int64_t cb = ca + chunk < c1 ? ca + chunk : c1;
            accumulate(compact2(Z, d, r0, r1, ca, cb, list, wc));
            __syncthreads();  // the list is rewritten by the next chunk
        }
    }
    float drift = 0.f, all = 0.f, dz32 = 0.f;
    if (j < d.Wz) {
#pragma unroll
        for (int t = 0; t < kPer; t++) {
            const int k = grp + 8 * t;
            if (k >= d.K)
                continue;
            const int64_t o = ((int64_t)k * d.Hz + i) * d.Wz + j;
            // r = beta0 - (hi + lo), finished with TwoSum: one final rounding
            float rn = beta0[o], rl = 0.f;
            df_add(rn, rl, -acc_hi[t]);
            df_add(rn, rl, -acc_lo[t]);
            rn = __fadd_rn(rn, rl);
            const float rold = r[o];
            if (write_r)
                r[o] = rn;
            drift = fmaxf(drift, fabsf(rold - rn));
            const float z = Z[o], nk = norms[k], rnk = __frcp_rn(nk);
            float gap;
            if (z == 0.f) {
                gap = soft_f(rn, lam) * rnk;
            } else {
                const float sg = z > 0.f ? 1.f : -1.f;
                const float b = fmaf(nk, z, rn);
                gap = b * sg > lam ? (rn - lam * sg) * rnk : soft_f(b, lam) * rnk - z;
            }
            all = fmaxf(all, fabsf(gap));
            float zn, dd;
            coord_step(rn, z, nk, rnk, lam, &zn, &dd);
            dz32 = fmaxf(dz32, fabsf(dd));
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        drift = fmaxf(drift, __shfl_xor_sync(0xffffffffu, drift, off));
        all = fmaxf(all, __shfl_xor_sync(0xffffffffu, all, off));
        dz32 = fmaxf(dz32, __shfl_xor_sync(0xffffffffu, dz32, off));
    }
    if (col == 0) {
        bred[0][grp] = drift;
        bred[1][grp] = all;
        bred[2][grp] = dz32;
    }
    __syncthreads();
    if (tid == 0) {
        float v[3] = {0.f, 0.f, 0.f};
        for (int g = 0; g < 8; g++)
            for (int q = 0; q < 3; q++)
                v[q] = fmaxf(v[q], bred[q][g]);
        atomicMax(&red[0], (unsigned long long)__double_as_longlong((double)v[0]));
        atomicMax(&red[3], (unsigned long long)__double_as_longlong((double)v[1]));
        atomicMax(&red[4], (unsigned long long)__double_as_longlong((double)v[2]));
    }
}

// Residual of one image row and kTile2 columns (all channels) per block, FP64:
// partial[2b] = sum over its pixels of R^2, partial[2b+1] = sum |Z| over the
// block's own activation positions (rows < Hz, columns < Wz).
__global__ void __launch_bounds__(256)
    objective2d_kernel(const float *__restrict__ D, const float *__restrict__ X,
                       const float *__restrict__ Z, Dims d, Buckets2 bk,
                       double *__restrict__ partial)
{
    __shared__ NZ2 list[kList2];
    __shared__ int wc[8];
    __shared__ double bsum[2][8];
    __shared__ int s_cnt[kGather2], s_off[kGather2 + 1], s_flag;
    const int tid = threadIdx.x, col = tid & 31, grp = tid >> 5;
    const int64_t ntc = (d.W + kTile2 - 1) / kTile2;
    const int64_t y = blockIdx.x / ntc, x0 = (blockIdx.x % ntc) * kTile2, x = x0 + col;
    // activations reaching pixel (y, x): rows [y-h+1, y], columns [x-w+1, x]
    const int64_t r0 = max((int64_t)0, y - (d.h - 1)), r1 = min(d.Hz, y + 1);
    const int64_t c0 = max((int64_t)0, x0 - (d.w - 1)), c1 = min(d.Wz, x0 + kTile2);
    // double-float per thread (the FP64 pipe is narrow); FP64 per warp
    float sq_h = 0.f, sq_l = 0.f, l1_h = 0.f, l1_l = 0.f;
    constexpr int kPm = 8;  // channels per thread group pass (P up to 64)
    float acc_hi[kPm], acc_lo[kPm];
#pragma unroll
    for (int t = 0; t < kPm; t++) {
        acc_hi[t] = 0.f;
        acc_lo[t] = 0.f;
    }
    // sum D z over the listed nonzeros whose atom covers (y, x)
    auto accumulate = [&](int n) {
        if (x >= d.W)
            return;
        for (int q = 0; q < n; q++) {
            const NZ2 e = list[q];
            const int64_t u = y - e.i, v = x - e.j;
            if (u < 0 || u >= d.h || v < 0 || v >= d.w)
                continue;
#pragma unroll
            for (int t = 0; t < kPm; t++) {
                const int p = grp + 8 * t;
                if (p < d.P)
                    df_add_prod(acc_hi[t], acc_lo[t],
                                __ldg(D + (((int64_t)e.k * d.P + p) * d.h + u) * d.w + v), e.z);
            }
        }
    };
    if (r0 < r1 && c0 < c1) {
        // from the buckets, else compacted from Z in column chunks
        const int nl = bk.count ? gather2(bk, r0, r1, c0, c1, list, s_cnt, s_off, &s_flag) : -1;
        if (nl >= 0) {
            accumulate(nl);
        } else {
            const int64_t chunk = max((int64_t)1, (int64_t)kList2 / ((int64_t)d.K * (r1 - r0)));
            for (int64_t ca = c0; ca < c1; ca += chunk) {
                const int64_t cb = ca + chunk < c1 ? ca + chunk : c1;
                accumulate(compact2(Z, d, r0, r1, ca, cb, list, wc));
                __syncthreads();
            }
        }
    }
    if (x < d.W)
#pragma unroll
        for (int t = 0; t < kPm; t++) {
            const int p = grp + 8 * t;
            if (p < d.P)
                df_add_sq_residual(sq_h, sq_l, X[((int64_t)p * d.H + y) * d.W + x], acc_hi[t],
                                   acc_lo[t]);
        }
    // |Z| of this block's own positions (row y, columns [x0, x0+32)), once
    if (grp == 0 && y < d.Hz && x < d.Wz)
        for (int k = 0; k < d.K; k++)
            df_add(l1_h, l1_l, fabsf(Z[((int64_t)k * d.Hz + y) * d.Wz + x]));
    for (int off = 16; off > 0; off >>= 1) {
        const float a = __shfl_xor_sync(0xffffffffu, sq_h, off);
        const float b = __shfl_xor_sync(0xffffffffu, sq_l, off);
        const float c = __shfl_xor_sync(0xffffffffu, l1_h, off);
        const float e = __shfl_xor_sync(0xffffffffu, l1_l, off);
        df_add_df(sq_h, sq_l, a, b);
        df_add_df(l1_h, l1_l, c, e);
    }
    if (col == 0) {
        bsum[0][grp] = (double)sq_h + (double)sq_l;
        bsum[1][grp] = (double)l1_h + (double)l1_l;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int g = 0; g < 8; g++) {
            a += bsum[0][g];
            b += bsum[1][g];
        }
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

__global__ void sum_partials_kernel(const double *__restrict__ partial, int64_t n, double lam,
                                    double *__restrict__ out)
{
    __shared__ double s[2][256];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int hh = blockDim.x / 2; hh > 0; hh >>= 1) {
        if ((int)threadIdx.x < hh) {
            s[0][threadIdx.x] += s[0][threadIdx.x + hh];
            s[1][threadIdx.x] += s[1][threadIdx.x + hh];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        out[0] = 0.5 * s[0][0] + lam * s[1][0];
}

int phases2(int64_t Hz, int M, int h)
{
    if (M <= 1)
        return 1;
    const int64_t hmin = Hz / M;
    const int64_t need = 2 * (int64_t)h - 2;
    const int64_t c = 1 + (need + hmin - 1) / hmin;
    return (int)(c > M ? M : c);
}

int auto_bands(int64_t Hz, int h)
{
    const int64_t bh = std::max<int64_t>(1, 2 * (int64_t)h - 2);
    return (int)std::max<int64_t>(1, std::min<int64_t>(Hz / bh, 1 << 20));
}

// Device buffers of one csc2d_solve call, carved from one allocation.
struct Dev2 {
    void *base = nullptr;
    float *D = nullptr, *X = nullptr, *Ct = nullptr, *norms = nullptr, *beta0 = nullptr,
          *r = nullptr, *Z = nullptr;
    int64_t *band_s = nullptr, *col_s = nullptr;
    int *list = nullptr;
    unsigned char *dirty = nullptr;
    long long *upd = nullptr;
    double *dec = nullptr, *x2 = nullptr, *partial = nullptr, *E = nullptr;
    unsigned *amax = nullptr;
    unsigned long long *red = nullptr;
    int *bcount = nullptr;  // nonzero buckets of Z (bucket2d_kernel)
    NZ2 *bent = nullptr;
    ~Dev2() { cudaFree(base); }
};

}  // namespace

extern "C" {

int csc2d_plan(int64_t Hz, int h, int M, int *M_out, int *phases, int64_t *starts)
{
    if (Hz < 1 || h < 1 || M < 0)
        return csc_record_error(CSC_EINVAL, "csc2d_plan: need Hz >= 1, h >= 1, M >= 0");
    if (M == 0)
        M = auto_bands(Hz, h);
    if (M > Hz)
        return csc_record_error(CSC_EINVAL, "csc2d_plan: M = %d exceeds Hz = %lld", M,
                                (long long)Hz);
    if (M_out)
        *M_out = M;
    if (phases)
        *phases = phases2(Hz, M, h);
    if (starts)
        for (int m = 0; m <= M; m++)
            starts[m] = (int64_t)m * Hz / M;
    return CSC_OK;
}

int csc2d_solve(const float *D, int K, int P, int h, int w, const float *X, int64_t H, int64_t W,
                double lambda, double tol, int64_t max_updates, int M, int N,
                int updates_per_visit, float *Z_out, double *objective, csc2d_stats *stats,
                void *stream)
{
    csc::TraceRange trace_("csc2d_solve");
    if (!D || !X)
        return csc_record_error(CSC_EINVAL, "csc2d_solve: null D or X");
    if (K < 1 || K > kMaxK2 || P < 1 || h < 1 || w < 1 || (2 * h - 1) * (2 * w - 1) > kMaxWin ||
        H < h || W < w)
        return csc_record_error(CSC_EINVAL,
                                "csc2d_solve: need 1 <= K <= %d, P >= 1, 1 <= h <= H, 1 <= w <= W, "
                                "(2h-1)(2w-1) <= %d",
                                kMaxK2, kMaxWin);
    if (!(lambda > 0.0) || !(tol > 0.0) || max_updates < 1 || updates_per_visit < 0 || N < 0)
        return csc_record_error(CSC_EINVAL, "csc2d_solve: need lambda > 0, tol > 0, "
                                            "max_updates >= 1, updates_per_visit >= 0, N >= 0");
    Dims d{K, P, h, w, H, W, H - h + 1, W - w + 1};
    if (d.K * d.Hz * d.Wz >= ((int64_t)1 << 31) || d.Hz * d.Wz >= ((int64_t)1 << 31) / 64)
        return csc_record_error(CSC_EINVAL, "csc2d_solve: image too large (flat indices)");
    // row bands and column blocks: the same cut and phase count per axis
    int Mb = 0, cr = 0, Nb = 0, cc = 0;
    int rc = csc2d_plan(d.Hz, h, M, &Mb, &cr, nullptr);
    if (rc != CSC_OK)
        return rc;
    rc = csc2d_plan(d.Wz, w, N, &Nb, &cc, nullptr);
    if (rc != CSC_OK)
        return rc;
    const int c = cr * cc;
    const int64_t ntiles = (int64_t)Mb * Nb;
    if (ntiles > (1 << 24))
        return csc_record_error(CSC_EINVAL, "csc2d_solve: %lld tiles (at most 2^24)",
                                (long long)ntiles);
    std::vector<int64_t> bs(Mb + 1), cs(Nb + 1);
    for (int m = 0; m <= Mb; m++)
        bs[m] = (int64_t)m * d.Hz / Mb;
    for (int q = 0; q <= Nb; q++)
        cs[q] = (int64_t)q * d.Wz / Nb;
    int64_t hmax = 0, wmax = 0;
    for (int m = 0; m < Mb; m++)
        hmax = std::max(hmax, bs[m + 1] - bs[m]);
    for (int q = 0; q < Nb; q++)
        wmax = std::max(wmax, cs[q + 1] - cs[q]);
    const int64_t max_pos = hmax * wmax;
    // a tile block's key index holds k (6 bits), the row and the column in
    // the tile and the sign of dZ in 32 bits
    auto bits = [](int64_t x) {
        int b = 0;
        while (b < 63 && ((int64_t)1 << b) <= x)
            b++;
        return b;
    };
    if (max_pos >= ((int64_t)1 << 31) / 64 || bits(hmax - 1) + bits(wmax - 1) > 25)
        return csc_record_error(CSC_EINVAL, "csc2d_solve: tiles too large");
    // a tile's r and Z are staged in shared memory when they fit
    const bool stage = TileLayout(K, (int)max_pos, true).total <= (size_t)kMaxSmem;
    const size_t smem = TileLayout(K, (int)max_pos, stage).total;
    if (smem > (size_t)kMaxSmem)
        return csc_record_error(CSC_EINVAL,
                                "csc2d_solve: a tile of %lld x %lld positions needs %zu bytes of "
                                "shared memory (more bands or column blocks)",
                                (long long)hmax, (long long)wmax, smem);
    // the exact checks gather the nonzeros of (2h-1) rows x K atoms one column
    // chunk at a time: one column must fit the list; the objective's
    // channels are spread over 8 thread groups, at most 8 passes each
    if ((int64_t)K * (2 * h - 1) > kList2 || P > 64)
        return csc_record_error(CSC_EINVAL, "csc2d_solve: need K (2h-1) <= %d and P <= 64",
                                kList2);
    int dev = 0;
    C2_CUDA(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    Dev2 g;
    const int KQ = (K + 3) / 4;
    const int64_t nz = (int64_t)K * d.Hz * d.Wz;
    const int A = (2 * h - 1) * (2 * w - 1);
    const int64_t ntile_o = H * ((W + kTile2 - 1) / kTile2);
    const int64_t ntc = (d.Wz + kTile2 - 1) / kTile2, nbk = d.Hz * ntc;
    {
        // one allocation, pieces on 256-byte boundaries
        size_t arena = 0;
        auto piece = [&arena](size_t bytes) {
            const size_t o = arena;
            arena += (bytes + 255) & ~(size_t)255;
            return o;
        };
        const size_t oD = piece(sizeof(float) * K * P * h * w), oX = piece(sizeof(float) * P * H * W),
                     oCt = piece(sizeof(float) * K * KQ * 4 * A), onorms = piece(sizeof(float) * K),
                     obeta0 = piece(sizeof(float) * nz), o_r = piece(sizeof(float) * nz),
                     oZ = piece(sizeof(float) * nz), oband = piece(sizeof(int64_t) * (Mb + 1)),
                     ocol = piece(sizeof(int64_t) * (Nb + 1)), olist = piece(sizeof(int) * ntiles),
                     odirty = piece((size_t)ntiles), oupd = piece(sizeof(long long) * kSweepBatch),
                     odec = piece(sizeof(double)), ox2 = piece(sizeof(double)),
                     oamax = piece(sizeof(unsigned)), ored = piece(sizeof(unsigned long long) * 8),
                     oE = piece(sizeof(double)), opart = piece(sizeof(double) * 2 * ntile_o),
                     obc = piece(sizeof(int) * nbk), obe = piece(sizeof(NZ2) * kBucket2 * nbk);
        C2_CUDA(cudaMalloc(&g.base, arena));
        char *b = static_cast<char *>(g.base);
        g.D = reinterpret_cast<float *>(b + oD);
        g.X = reinterpret_cast<float *>(b + oX);
        g.Ct = reinterpret_cast<float *>(b + oCt);
        g.norms = reinterpret_cast<float *>(b + onorms);
        g.beta0 = reinterpret_cast<float *>(b + obeta0);
        g.r = reinterpret_cast<float *>(b + o_r);
        g.Z = reinterpret_cast<float *>(b + oZ);
        g.band_s = reinterpret_cast<int64_t *>(b + oband);
        g.col_s = reinterpret_cast<int64_t *>(b + ocol);
        g.list = reinterpret_cast<int *>(b + olist);
        g.dirty = reinterpret_cast<unsigned char *>(b + odirty);
        g.upd = reinterpret_cast<long long *>(b + oupd);
        g.dec = reinterpret_cast<double *>(b + odec);
        g.x2 = reinterpret_cast<double *>(b + ox2);
        g.amax = reinterpret_cast<unsigned *>(b + oamax);
        g.red = reinterpret_cast<unsigned long long *>(b + ored);
        g.E = reinterpret_cast<double *>(b + oE);
        g.partial = reinterpret_cast<double *>(b + opart);
        g.bcount = reinterpret_cast<int *>(b + obc);
        g.bent = reinterpret_cast<NZ2 *>(b + obe);
    }
    int64_t launches = 0;
    C2_CUDA(copy_in(g.D, D, sizeof(float) * K * P * h * w, s));
    C2_CUDA(copy_in(g.X, X, sizeof(float) * P * H * W, s));
    // phase lists: phase pr cc + pc holds the tiles (m, n) with m == pr (mod
    // cr) and n == pc (mod cc), consecutive in the device list
    std::vector<int> list;
    std::vector<int> off(c + 1, 0);
    for (int pr = 0; pr < cr; pr++)
        for (int pc = 0; pc < cc; pc++) {
            off[pr * cc + pc] = (int)list.size();
            for (int m = pr; m < Mb; m += cr)
                for (int q = pc; q < Nb; q += cc)
                    list.push_back(m * Nb + q);
        }
    off[c] = (int)list.size();
    C2_CUDA(cudaMemcpyAsync(g.band_s, bs.data(), sizeof(int64_t) * (Mb + 1),
                            cudaMemcpyHostToDevice, s));
    C2_CUDA(cudaMemcpyAsync(g.col_s, cs.data(), sizeof(int64_t) * (Nb + 1),
                            cudaMemcpyHostToDevice, s));
    C2_CUDA(cudaMemcpyAsync(g.list, list.data(), sizeof(int) * ntiles, cudaMemcpyHostToDevice,
                            s));
    C2_CUDA(cudaMemsetAsync(g.amax, 0, sizeof(unsigned), s));
    C2_CUDA(cudaMemsetAsync(g.x2, 0, sizeof(double), s));
    C2_CUDA(cudaMemsetAsync(g.Z, 0, sizeof(float) * nz, s));
    C2_CUDA(cudaMemsetAsync(g.dirty, 1, ntiles, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    C2_CUDA(cudaEventCreate(&e0));
    C2_CUDA(cudaEventCreate(&e1));
    C2_CUDA(cudaEventRecord(e0, s));
    {
        const int64_t n = (int64_t)K * KQ * 4 * A;
        dtd2d_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(g.D, d, KQ,
                                                                                       g.Ct, g.norms);
        C2_CUDA(cudaGetLastError());
        dtx2d_kernel<<<(unsigned)std::min<int64_t>((nz + 255) / 256, 152 * 16), 256, 0, s>>>(
            g.D, g.X, d, g.beta0, g.r, g.amax, g.x2);
        C2_CUDA(cudaGetLastError());
        launches += 2;
    }
    auto tile_fn = stage ? tile_kernel<true> : tile_kernel<false>;
    C2_CUDA(cudaFuncSetAttribute(tile_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    TileParams tp;
    tp.r = g.r;
    tp.Z = g.Z;
    tp.Ct = g.Ct;
    tp.norms = g.norms;
    tp.row_s = g.band_s;
    tp.col_s = g.col_s;
    tp.dirty = g.dirty;
    tp.upd = g.upd;
    tp.dec = g.dec;
    tp.d = d;
    tp.Mr = Mb;
    tp.Mc = Nb;
    tp.KQ = KQ;
    tp.max_pos = (int)max_pos;
    tp.u = updates_per_visit > 0 ? updates_per_visit : kAutoVisit2d;
    tp.lam = (float)lambda;
    const int max_resyncs = 3;
    tp.tol = (float)(0.5 * tol);  // CD to tol/2, the exact check accepts at tol
    int64_t updates = 0, sweeps = 0;
    int resyncs = 0;
    bool converged = false;
    const unsigned rgrid = (unsigned)(d.Hz * ntc);
    const Buckets2 bk2{g.bcount, g.bent, ntc};
    double dz32 = 0.0, all = 0.0;
    for (;;) {
        bool settled = false;
        for (bool more = true; more;) {
            // kSweepBatch sweeps per read-back when neither limit can be reached
            // inside the batch (a visit applies at most u updates); after a
            // sweep without updates no tile is dirty and the rest do nothing
            const int64_t per_sweep = (int64_t)ntiles * tp.u;
            const int nb = updates + kSweepBatch * per_sweep < max_updates &&
                                   sweeps + kSweepBatch < 1000000
                               ? kSweepBatch
                               : 1;
            C2_CUDA(cudaMemsetAsync(g.upd, 0, sizeof(long long) * nb, s));
            for (int b = 0; b < nb; b++) {
                tp.upd = g.upd + b;
                for (int p = 0; p < c; p++) {
                    const int cnt = off[p + 1] - off[p];
                    if (cnt == 0)
                        continue;
                    tp.list = g.list + off[p];
                    tile_fn<<<cnt, kB2, smem, s>>>(tp);
                    C2_CUDA(cudaGetLastError());
                    launches++;
                }
            }
            long long u[kSweepBatch] = {};
            C2_CUDA(cudaMemcpyAsync(u, g.upd, sizeof(long long) * nb, cudaMemcpyDeviceToHost, s));
            C2_CUDA(cudaStreamSynchronize(s));
            for (int b = 0; b < nb && more; b++) {
                sweeps++;
                updates += u[b];
                if (u[b] == 0)
                    settled = true;
                if (settled || updates >= max_updates || sweeps >= 1000000)
                    more = false;
            }
        }
        // exact refresh of r from Z and the report
        C2_CUDA(cudaMemsetAsync(g.red, 0, sizeof(unsigned long long) * 8, s));
        bucket2d_kernel<<<(unsigned)((nbk * 32 + 255) / 256), 256, 0, s>>>(g.Z, d, ntc, g.bcount,
                                                                         g.bent);
        C2_CUDA(cudaGetLastError());
        resync2d_kernel<<<rgrid, 256, 0, s>>>(g.beta0, g.r, g.Z, g.Ct, g.norms, d, KQ,
                                              (float)lambda, 1, bk2, g.red);
        C2_CUDA(cudaGetLastError());
        launches += 2;
        unsigned long long red[8];
        C2_CUDA(cudaMemcpyAsync(red, g.red, sizeof red, cudaMemcpyDeviceToHost, s));
        C2_CUDA(cudaStreamSynchronize(s));
        std::memcpy(&dz32, &red[4], sizeof dz32);
        std::memcpy(&all, &red[3], sizeof all);
        if (!settled)
            break;  // max_updates or the sweep limit
        resyncs++;
        if (dz32 < tol) {
            converged = true;
            break;
        }
        if (resyncs > max_resyncs)
            break;
        C2_CUDA(cudaMemsetAsync(g.dirty, 1, ntiles, s));
    }
    C2_CUDA(cudaEventRecord(e1, s));
    const unsigned ogrid = (unsigned)ntile_o;
    objective2d_kernel<<<ogrid, 256, 0, s>>>(g.D, g.X, g.Z, d, bk2, g.partial);  // Z as refreshed
    C2_CUDA(cudaGetLastError());
    sum_partials_kernel<<<1, 256, 0, s>>>(g.partial, ntile_o, lambda, g.E);
    C2_CUDA(cudaGetLastError());
    launches += 2;
    double E = 0.0;
    C2_CUDA(cudaMemcpyAsync(&E, g.E, sizeof E, cudaMemcpyDeviceToHost, s));
    if (Z_out)
        C2_CUDA(copy_out(Z_out, g.Z, sizeof(float) * nz, s));
    C2_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    C2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (objective)
        *objective = E;
    if (stats) {
        stats->updates = updates;
        stats->sweeps = sweeps;
        stats->bands = Mb;
        stats->col_blocks = Nb;
        stats->phases = c;
        stats->resyncs = resyncs;
        stats->converged = converged ? 1 : 0;
        stats->objective = E;
        stats->max_delta_z = all;
        stats->solve_ms = ms;
        stats->kernel_launches = launches;
    }
    (void)dev;
    return converged ? CSC_OK : CSC_NOT_CONVERGED;
}

}  // extern "C"
