// beta0 = D~ * X (Alg. 1 initialisation) on the 5th-generation tensor cores.
//
// As a matrix product, beta0^T [Tz x K] = A [Tz x J] B [J x K] with the
// contraction index j = (p, tau), J = P * L16 (L padded to a multiple of 16),
// A[t][j] = X[p][t + tau] (a Hankel matrix per channel) and B[j][k] = D[k][p][tau].
// One CTA computes 128 consecutive t (the MMA's M) for all atoms (N = 32 or
// 64 >= K) with tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator in
// tensor memory), one instruction per 16 contraction indices.
//
// Precision: every X and D value is split into three BF16 terms,
// x = x_h + x_m + x_l (each term the BF16 rounding of what the previous ones
// left, so the split is exact to 2^-24 |x|), and the six products whose
// magnitude is at least 2^-16 of the leading one (hh, hm, mh, hl, lh, mm) are
// accumulated in FP32.  The dropped ones (ml, lm, ll) are below 2^-24 of it,
// so the result has the accuracy of an FP32 computation; with only the hh
// product (mode 2) it is a plain BF16 product, kept to measure that error.
//
// Operand layouts (no swizzle; a core matrix is 8 rows of 16 bytes):
//   A, MN-major (t contiguous): core matrix (m8, j8) holds rows j = 8 j8 + r,
//     each row X[p][t0 + 8 (m8 + j8) + r + 0..7].  It depends on m8 + j8 only,
//     so one run of 16 + L16/8 core matrices per channel and split serves the
//     whole tile, with equal leading and stride byte offsets (128 B): moving
//     one core matrix along M or along K is the same step in memory.
//   B, K-major (j contiguous): per 16-wide contraction step, the three
//     splits one after the other, each N/8 x 2 core matrices, K-adjacent at
//     128 B, N-adjacent at 256 B; row k of core matrix (n8, j8) of split
//     sigma holds term sigma of D[k = 8 n8 + r][p][tau = 16 s + 8 j8 + 0..7 -
//     p L16].  The splits of a step are thus one operand of 3N rows.
// Concatenated products (N = 32): per step one M x 3N product of the leading
// term of X with [D_h D_m D_l] (hh, hm, hl), one M x 2N product of its middle
// term with [D_h D_m] (mh, mm) and one M x N product of its last term with D_h
// (lh), into one accumulator of 3N columns: hh + mh + lh, hm + mm and hl,
// summed in the epilogue.  The tensor cores read each A run three times per
// step instead of six.  At N = 64 (K > 32) the six products go into one
// accumulator of N columns (3N columns twice would exceed the 256 a CTA
// allocates).  One warp issues the products while the others build operands
// and read accumulators out (dtx_tc_ws_kernel).  The accumulator lives in
// tensor memory (32-bit columns, lane = t); the warp of each lane quarter
// reads its 32 lanes with tcgen05.ld and writes beta0[k][t] coalesced along t.
//
// What bounds the products: the tensor cores read the operands from shared
// memory in this unswizzled layout (the Hankel runs of A overlap, which no
// swizzled layout allows); at N = 32 a step reads 18 KB (A three times, B
// once) for 0.4 M multiply-adds, so the operand reads, not the multipliers,
// set the pace of the products.
//
// Waits are bounded: a wait that gives up sets *err, the block stops issuing
// work, waits (again bounded) for the products already issued and releases
// tensor memory.
#include <cuda_bf16.h>
#include <stdint.h>

#include "csc_internal.cuh"

namespace csc {

namespace {

constexpr int kTcM = 128;        // time rows per tile
constexpr int kSplits = 3;
constexpr unsigned kWaitLimit = 1u << 22;
constexpr int kMaxSteps = 128;  // P * L16 / 16 contraction steps (B alone then needs >= 96 KB)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start address, leading and stride
// byte offsets (16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t mma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, A
// MN-major, B K-major, shape M x N.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// True once phase `parity` of the barrier has completed; false after `limit`
// unsuccessful polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned limit)
{
    for (unsigned n = 0; n < limit; n++)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

__device__ __forceinline__ void fence_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++)
        v[i] = __uint_as_float(r[i]);
}

// The three BF16 terms of x.
__device__ __forceinline__ void split3(float x, __nv_bfloat16 &h, __nv_bfloat16 &m,
                                       __nv_bfloat16 &l)
{
    h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    l = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

struct TcLayout {
    int L16, NQ, nsteps, xw;
    size_t a_off, b_off, pl_off, bar_off, total;
    __host__ __device__ TcLayout(int P, int L, int N)
    {
        L16 = (L + 15) & ~15;
        NQ = kTcM / 8 + L16 / 8;
        nsteps = P * L16 / 16;
        xw = kTcM + L16 + 8;  // staged samples per channel: 8 (NQ + 1)
        size_t o = 0;
        a_off = o;
        o += 2 * (size_t)kSplits * P * NQ * 128;  // two operand buffers
        b_off = o;
        o += (size_t)kSplits * nsteps * (N / 8) * 256;  // [step][split][n8][j8][r]
        pl_off = o;  // the three BF16 terms of the staged samples, [split][p][xw]
        o += (size_t)kSplits * P * xw * 2;
        o = (o + 15) & ~(size_t)15;
        bar_off = o;
        o += 16;  // two mbarriers
        total = o;
    }
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Barrier 1 among the n worker threads (the issuing warp does not take part).
__device__ __forceinline__ void workers_sync(int n)
{
    asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
}

// The same barrier, returning whether v was true in any of the n threads.
__device__ __forceinline__ bool workers_any(bool v, int n)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(n)
        : "memory");
    return r != 0;
}

// NW worker warps build the operands of tile i and read the accumulator of
// tile i-1 out while one more warp issues the products, so that the issue of
// a tile's products by one thread does not hold up the operand build and the
// read-out.  CAT (N = 32, mode 1): three concatenated products per step into
// an accumulator of 3N columns; otherwise one accumulator of N columns with
// the six products of mode 1 (N = 64, where 3N columns would not fit twice)
// or the hh product alone (mode 2).  The two sides meet only at mbarriers:
//   full[b]  the operands of the tile in buffer b are written (one arrival
//            per worker thread, after its proxy fence),
//   done[b]  the products into accumulator b have finished (tcgen05.commit),
//   free[b]  accumulator b has been read out (one arrival per worker thread).
// Tile i of the CTA uses operand buffer and accumulator b = i & 1; its use
// u = i >> 1 of them completes phase u of the three barriers of b, which is
// waited for with parity u & 1.  The workers share barrier 1 (plane buffer
// reuse, and the block's decision to give up after a wait ran out).
// (two CTAs per SM with four workers; the N = 64 form then keeps a few
// values in local memory, and still runs faster than with one CTA per SM)
template <int N, bool CAT, int NW>
__global__ void __launch_bounds__(32 * NW + 32, NW <= 4 ? 2 : 1)
    dtx_tc_ws_kernel(const float *__restrict__ D, const float *__restrict__ X, int K, int P,
                     int L, long long T, int mode, float *__restrict__ beta0,
                     float *__restrict__ r_out, unsigned int *__restrict__ absmax_bits,
                     double *__restrict__ x2sum, int *__restrict__ err, Dtx0Extras ex)
{
    static_assert(!CAT || N == 32, "concatenated products need N = 32 (3N + 3N <= 256 columns)");
    constexpr int NTW = 32 * NW;                   // worker threads
    constexpr int NTA = NTW + 32;                  // with the issuing warp
    constexpr int acc_cols = CAT ? 3 * N : N;      // CAT: hh+mh+lh | hm+mm | hl
    constexpr uint32_t tm_cols = CAT ? 256u : 2u * N;  // two accumulators (a power of two)
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint32_t s_taddr;
    __shared__ uint32_t s_aoff[kMaxSteps];
    __shared__ __align__(8) unsigned long long s_bar[6];  // full[2], done[2], free[2]
    const TcLayout lay(P, L, N);
    unsigned char *As = sm + lay.a_off;
    unsigned char *Bs = sm + lay.b_off;
    uint32_t *pl = reinterpret_cast<uint32_t *>(sm + lay.pl_off);
    const uint32_t full0 = smem_u32(&s_bar[0]), done0 = smem_u32(&s_bar[2]),
                   free0 = smem_u32(&s_bar[4]);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long Tz = T - L + 1;
    const long long ntiles = (Tz + kTcM - 1) / kTcM;

    if (warp == NW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_taddr)),
                     "r"(tm_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8u * b), "r"(NTW)
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done0 + 8u * b) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(free0 + 8u * b), "r"(NTW)
                         : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int st = tid; st < lay.nsteps; st += NTA) {
        const int p = (16 * st) / lay.L16, q0 = ((16 * st) % lay.L16) / 8;
        s_aoff[st] = (uint32_t)((p * lay.NQ + q0) * 128) >> 4;
    }
    // B: the three BF16 terms of D per contraction step.
    // element (sigma, s, n8, j8, r, e): D[k = 8 n8 + r][p][tau], j = 16 s + 8 j8 + e
    const int rows_b = lay.nsteps * (N / 8) * 2 * 8;
    for (int i = tid; i < rows_b; i += NTA) {
        const int r = i & 7, j8 = (i >> 3) & 1, n8 = (i >> 4) % (N / 8), s = (i >> 4) / (N / 8);
        const int k = 8 * n8 + r;
        uint32_t w[kSplits][4];
#pragma unroll
        for (int e2 = 0; e2 < 4; e2++) {
            __nv_bfloat16 h[2], m[2], l[2];
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int j = 16 * s + 8 * j8 + 2 * e2 + q;
                const int p = j / lay.L16, tau = j % lay.L16;
                const float v = (k < K && tau < L) ? D[((long long)k * P + p) * L + tau] : 0.f;
                split3(v, h[q], m[q], l[q]);
            }
            w[0][e2] = pack2(h[0], h[1]);
            w[1][e2] = pack2(m[0], m[1]);
            w[2][e2] = pack2(l[0], l[1]);
        }
#pragma unroll
        for (int sg = 0; sg < kSplits; sg++) {
            const size_t off =
                ((((size_t)s * kSplits + sg) * (N / 8) + n8) * 2 + j8) * 128 + (size_t)r * 16;
            *reinterpret_cast<uint4 *>(Bs + off) = make_uint4(w[sg][0], w[sg][1], w[sg][2], w[sg][3]);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t taddr = s_taddr;
    const size_t a_bytes = (size_t)kSplits * P * lay.NQ * 128;
    const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
    const long long cnt = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp < NW) {
        // ---------------- workers: operand build and read-out ----------------
        float amax = 0.f;
        int sig_c = -1;  // the batch problem of this thread's column in its last tile
        float x2h = 0.f, x2l = 0.f;  // sum of X^2 over the CTA's own samples (double-float)
        const int half = lay.xw / 2;
        constexpr int kPairs = 4;  // P = 7 at L = 64, or P = 1 at L = 200, fit
        const bool prefetched = P * half <= kPairs * NTW;
        float2 xr[kPairs];
        auto load_x = [&](long long tile) {
            const long long t0 = tile * kTcM;
#pragma unroll
            for (int q = 0; q < kPairs; q++) {
                const int i = tid + q * NTW;
                float2 v = make_float2(0.f, 0.f);
                if (i < P * half) {
                    const int p = i / half, j2 = i % half;
                    const long long t = t0 + 2 * j2;
                    const float *xp = X + (long long)p * T + t;
                    v.x = t < T ? xp[0] : 0.f;
                    v.y = t + 1 < T ? xp[1] : 0.f;
                }
                xr[q] = v;
            }
        };
        auto put_pair = [&](int i, float v0, float v1, bool own) {
            const int p = i / half, j2 = i % half;
            if (own || 2 * j2 < kTcM) {
                df_add_prod(x2h, x2l, v0, v0);
                df_add_prod(x2h, x2l, v1, v1);
            }
            __nv_bfloat16 h0, m0, l0, h1, m1, l1;
            split3(v0, h0, m0, l0);
            split3(v1, h1, m1, l1);
            pl[(0 * P + p) * half + j2] = pack2(h0, h1);
            pl[(1 * P + p) * half + j2] = pack2(m0, m1);
            pl[(2 * P + p) * half + j2] = pack2(l0, l1);
        };
        // operand runs of a tile into buffer buf.  Row (sigma, p, q, r) = split
        // sigma of X[p][t0 + 8 q + r + 0..7]: the BF16 words 4 q + r/2 .. 4 q +
        // r/2 + 4 of the plane, shifted by 16 bits when r is odd.  r = tid & 7 is
        // the same for all of a thread's rows, and the 8 lanes of one q write
        // 128 contiguous bytes (no bank conflict).
        auto build = [&](long long tile, int buf) {
            const long long t0 = tile * kTcM;
            const bool last = tile == ntiles - 1;
            if (prefetched) {
#pragma unroll
                for (int q = 0; q < kPairs; q++) {
                    const int i = tid + q * NTW;
                    if (i < P * half)
                        put_pair(i, xr[q].x, xr[q].y, last);
                }
            } else {
                for (int i = tid; i < P * half; i += NTW) {
                    const int p = i / half, j2 = i % half;
                    const long long t = t0 + 2 * j2;
                    const float *xp = X + (long long)p * T + t;
                    put_pair(i, t < T ? xp[0] : 0.f, t + 1 < T ? xp[1] : 0.f, last);
                }
            }
            workers_sync(NTW);
            unsigned char *Ab = As + (size_t)buf * a_bytes;
            const int rows_a = P * lay.NQ * 8;
            const int r = tid & 7, wa = r >> 1;
            const unsigned sh = (unsigned)(r & 1) * 16u;
            int q = (tid >> 3) % lay.NQ, p = (tid >> 3) / lay.NQ;
            for (int i = tid; i < rows_a; i += NTW) {
                const size_t off = ((size_t)p * lay.NQ + q) * 128 + (size_t)r * 16;
#pragma unroll
                for (int sg = 0; sg < kSplits; sg++) {
                    const uint32_t *w = pl + (size_t)(sg * P + p) * half + 4 * q + wa;
                    const uint32_t w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3], w4 = w[4];
                    *reinterpret_cast<uint4 *>(Ab + (size_t)sg * P * lay.NQ * 128 + off) =
                        make_uint4(__funnelshift_r(w0, w1, sh), __funnelshift_r(w1, w2, sh),
                                   __funnelshift_r(w2, w3, sh), __funnelshift_r(w3, w4, sh));
                }
                q += NTW / 8;
                while (q >= lay.NQ) {
                    q -= lay.NQ;
                    p++;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        };
        // accumulator buf (use parity par) -> beta0 columns of the tile; false
        // if the wait for its products ran out
        auto epilogue = [&](long long tile, int buf, uint32_t par) -> bool {
            // the warp reads tensor memory together (tcgen05.ld is warp-wide):
            // it reads only if every lane saw the products finish
            const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(done0 + 8u * (uint32_t)buf,
                                                                      par, kWaitLimit));
            if (got) {
                fence_after_sync();
                constexpr int CW = N / (NTW / 128);
                const int quarter = warp & 3, c_lo = (warp >> 2) * CW;
                const long long t = tile * kTcM + 32 * quarter + lane;
                const uint32_t lane_addr =
                    taddr + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(buf * acc_cols);
                float tmax = 0.f;  // this tile's largest |beta0| in the thread's column
                auto put = [&](int k, float v) {
                    if (k < K) {
                        beta0[(long long)k * Tz + t] = v;
                        if (r_out)
                            r_out[(long long)k * Tz + t] = v;
                        if (ex.z_out)
                            ex.z_out[(long long)k * Tz + t] = 0.f;
                        tmax = fmaxf(tmax, fabsf(v));
                    }
                };
                // 16 columns at a time (CAT: hl + (hm + mm) + (hh + mh + lh),
                // smallest first)
#pragma unroll
                for (int c = c_lo; c < c_lo + CW; c += 16) {
                    float v[16];
                    if constexpr (CAT) {
                        float u[16];
                        tmem_ld16(lane_addr + (uint32_t)(2 * N + c), v);
                        tmem_ld16(lane_addr + (uint32_t)(N + c), u);
#pragma unroll
                        for (int i = 0; i < 16; i++)
                            v[i] += u[i];
                        tmem_ld16(lane_addr + (uint32_t)c, u);
#pragma unroll
                        for (int i = 0; i < 16; i++)
                            v[i] += u[i];
                    } else {
                        tmem_ld16(lane_addr + (uint32_t)c, v);
                    }
                    if (t < Tz) {
#pragma unroll
                        for (int i = 0; i < 16; i++)
                            put(c + i, v[i]);
                    }
                }
                amax = fmaxf(amax, tmax);
                if (ex.lmax) {
                    // the problem of column t: the last i with a[i] <= t, if t
                    // is one of its columns (the L - 1 after it belong to none);
                    // a thread's columns only grow from tile to tile, so the
                    // search starts from the problem of its previous tile
                    int sig = -1;
                    if (t < Tz) {
                        if (sig_c < 0) {
                            int lo = 0, hi = ex.nsig;  // a[lo] <= t < a[hi]
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (ex.a[mid] <= t)
                                    lo = mid;
                                else
                                    hi = mid;
                            }
                            sig_c = lo;
                        }
                        while (sig_c + 1 < ex.nsig && ex.a[sig_c + 1] <= t)
                            sig_c++;
                        sig = t < ex.a[sig_c + 1] - L + 1 ? sig_c : -1;
                    }
                    // one atomic per warp where its 32 columns share a problem
                    const int s0 = __shfl_sync(0xffffffffu, sig, 0);
                    if (__all_sync(0xffffffffu, sig == s0)) {
                        float m = tmax;
                        for (int off = 16; off > 0; off >>= 1)
                            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
                        if (lane == 0 && s0 >= 0)
                            atomicMax(ex.lmax + s0, __float_as_uint(m));
                    } else if (sig >= 0) {
                        atomicMax(ex.lmax + sig, __float_as_uint(tmax));
                    }
                }
            }
            fence_before_sync();
            mbar_arrive(free0 + 8u * (uint32_t)buf);
            return got;
        };

        if (prefetched && cnt > 0)
            load_x(blockIdx.x);
        bool gave_up = false;
        for (long long i = 0; i < cnt; i++) {
            const int b = (int)(i & 1);
            build(blockIdx.x + i * gridDim.x, b);
            mbar_arrive(full0 + 8u * (uint32_t)b);
            // the next tile's samples are in flight while the products of tile i
            // run and the accumulator of tile i-1 is read out
            if (prefetched && i + 1 < cnt)
                load_x(blockIdx.x + (i + 1) * gridDim.x);
            bool got = true;
            if (i > 0)
                got = epilogue(blockIdx.x + (i - 1) * gridDim.x, (int)((i - 1) & 1),
                               (uint32_t)(((i - 1) >> 1) & 1));
            // every worker is done with the planes of tile i before the next
            // tile's samples overwrite them; a wait that ran out stops all of them
            if (workers_any(!got, NTW)) {
                gave_up = true;
                break;
            }
        }
        if (!gave_up && cnt > 0 &&
            !epilogue(blockIdx.x + (cnt - 1) * gridDim.x, (int)((cnt - 1) & 1),
                      (uint32_t)(((cnt - 1) >> 1) & 1)))
            gave_up = true;
        if (gave_up)
            atomicExch(err, 1);
        double x2 = (double)x2h + (double)x2l;
        for (int off = 16; off > 0; off >>= 1) {
            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
            x2 += __shfl_xor_sync(0xffffffffu, x2, off);
        }
        if (lane == 0) {
            atomicMax(absmax_bits, __float_as_uint(amax));
            atomicAdd(x2sum, x2);
        }
    } else {
        // ---------------- issuing warp (lane 0 issues) -----------------------
        const uint32_t idesc = mma_idesc(kTcM, N);
        const uint32_t idesc_cat2 = mma_idesc(kTcM, 2 * N), idesc_cat3 = mma_idesc(kTcM, 3 * N);
        const uint32_t a_split = (uint32_t)(P * lay.NQ * 128) >> 4;
        const uint32_t b_split = (uint32_t)((N / 8) * 256) >> 4;
        const uint64_t bd0 = mma_desc(b_base, 128, 256);
        long long issued = -1;
        for (long long i = 0; i < cnt; i++) {
            const int b = (int)(i & 1);
            const uint32_t par = (uint32_t)((i >> 1) & 1);
            bool ok = true;
            if (lane == 0) {
                ok = mbar_wait_bounded(full0 + 8u * (uint32_t)b, par, kWaitLimit);
                // accumulator b was read out (tile i-2)
                if (ok && i >= 2)
                    ok = mbar_wait_bounded(free0 + 8u * (uint32_t)b, par ^ 1u, kWaitLimit);
                if (ok) {
                    fence_after_sync();
                    const uint32_t d_acc = taddr + (uint32_t)(b * acc_cols);
                    const uint64_t ad0 = mma_desc(a_base + (uint32_t)(b * a_bytes), 128, 128);
                    for (int s = 0; s < lay.nsteps; s++) {
                        const uint64_t a_s = ad0 + s_aoff[s];
                        const uint64_t b_s = bd0 + ((uint32_t)(s * kSplits * (N / 8) * 256) >> 4);
                        const uint32_t acc = s > 0 ? 1u : 0u;
                        if constexpr (CAT) {
                            // hh|hm|hl (first: it covers all 3N columns), mh|mm, lh
                            mma_bf16(d_acc, a_s, b_s, idesc_cat3, acc);
                            mma_bf16(d_acc, a_s + 1 * a_split, b_s, idesc_cat2, 1u);
                            mma_bf16(d_acc, a_s + 2 * a_split, b_s, idesc, 1u);
                        } else if (mode == 2) {
                            mma_bf16(d_acc, a_s, b_s, idesc, acc);  // hh
                        } else {
                            // mm, lh, hl, mh, hm, hh: small terms first
                            mma_bf16(d_acc, a_s + 1 * a_split, b_s + 1 * b_split, idesc, acc);
                            mma_bf16(d_acc, a_s + 2 * a_split, b_s, idesc, 1u);
                            mma_bf16(d_acc, a_s, b_s + 2 * b_split, idesc, 1u);
                            mma_bf16(d_acc, a_s + 1 * a_split, b_s, idesc, 1u);
                            mma_bf16(d_acc, a_s, b_s + 1 * b_split, idesc, 1u);
                            mma_bf16(d_acc, a_s, b_s, idesc, 1u);
                        }
                    }
                    mma_commit(done0 + 8u * (uint32_t)b);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0)
                    atomicExch(err, 1);
                break;
            }
            issued = i;
        }
        // the last products issued (tcgen05.commit tracks all earlier ones) have
        // finished before tensor memory is released
        if (lane == 0 && issued >= 0 &&
            !mbar_wait_bounded(done0 + 8u * (uint32_t)(issued & 1), (uint32_t)((issued >> 1) & 1),
                               kWaitLimit))
            atomicExch(err, 1);
        __syncwarp();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == NW)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                     "r"(tm_cols)
                     : "memory");
}

// Failure-detection check of the bounded wait: one warp waits, with the
// wait the kernel above uses, on an mbarrier that nothing arrives at.  The
// wait gives up after `limit` polls, *gave_up is set, and the kernel returns.
__global__ void wait_selftest_kernel(unsigned limit, int *gave_up)
{
    __shared__ __align__(8) unsigned long long mb;
    const uint32_t bar = smem_u32(&mb);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool got = mbar_wait_bounded(bar, 0u, limit);
    if (__syncthreads_or(!got) && threadIdx.x == 0)
        atomicExch(gave_up, 1);
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned limit, int *gave_up, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 32, 0, s>>>(limit, gave_up);
    return cudaGetLastError();
}

size_t dtx_tc_smem(int K, int P, int L)
{
    const int N = K <= 32 ? 32 : 64;
    return TcLayout(P, L, N).total;
}

cudaError_t launch_dtx_tc(const float *D, const float *X, int K, int P, int L, int64_t T,
                          int mode, float *beta0, float *r_out, unsigned int *absmax_bits,
                          double *x2sum, int *err, cudaStream_t s, Dtx0Extras *ex)
{
    const Dtx0Extras extras = ex ? *ex : Dtx0Extras{};
    if (K > 64)
        return cudaErrorNotSupported;
    const size_t smem = dtx_tc_smem(K, P, L);
    if (smem > (size_t)kMaxSmem || (size_t)P * ((L + 15) / 16) > (size_t)kMaxSteps)
        return cudaErrorNotSupported;
    const int64_t Tz = T - L + 1;
    const int64_t ntiles = (Tz + kTcM - 1) / kTcM;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // max_per_sm: tensor-memory columns allow at most 512 / (columns per CTA)
    auto go = [&](auto kern, int max_per_sm) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess)
            return e;
        // one wave of persistent CTAs: as many per SM as its shared memory
        // (1 KB reserved per block) and register file hold at once, up to four
        // (at N <= 64 tensor-memory columns each they never ask an SM for more
        // than its 512 columns), each looping over its tiles
        int smem_sm = 0;
        cudaFuncAttributes fa;
        e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess)
            e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess)
            return e;
        const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
        // the block size the instantiation was compiled for (launch bounds)
        const int nt = fa.maxThreadsPerBlock;
        const int by_regs = 65536 / (fa.numRegs * nt > 0 ? fa.numRegs * nt : 1);
        int per_sm = by_smem < by_regs ? by_smem : by_regs;
        per_sm = per_sm < 1 ? 1 : (per_sm > max_per_sm ? max_per_sm : per_sm);
        // concatenated products where at most two CTAs share an SM: their
        // accumulators take 256 of its 512 tensor-memory columns each
        const int64_t cap = (int64_t)nsm * per_sm;
        const unsigned grid = (unsigned)(ntiles < cap ? ntiles : cap);
        kern<<<grid, nt, smem, s>>>(D, X, K, P, L, (long long)T, mode, beta0, r_out, absmax_bits,
                                   x2sum, err, extras);
        e = cudaGetLastError();
        if (e == cudaSuccess && ex)
            ex->done = true;
        return e;
    };
    // mode 1 at N = 32: concatenated products with a warp of their own, one
    // CTA per SM with eight worker warps or two with four (their accumulators
    // take 256 of the SM's 512 tensor-memory columns each)
    int smem_sm = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess)
        e = cudaFuncGetAttributes(&fa, dtx_tc_ws_kernel<32, true, 8>);
    if (e != cudaSuccess)
        return e;
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
    if (K > 32)
        return go(dtx_tc_ws_kernel<64, false, 4>, 2);
    if (mode == 1)
        return by_smem <= 1 ? go(dtx_tc_ws_kernel<32, true, 8>, 1)
                            : go(dtx_tc_ws_kernel<32, true, 4>, 2);
    return by_smem <= 1 ? go(dtx_tc_ws_kernel<32, false, 8>, 1)
                        : go(dtx_tc_ws_kernel<32, false, 4>, 2);
}

cudaError_t launch_dtx_any(const float *D, const float *X, int K, int P, int L, int64_t T,
                           int init_mode, float *beta0, float *r_out, unsigned int *absmax_bits,
                           double *x2sum, int *err, cudaStream_t s, Dtx0Extras *ex)
{
    int mode = init_mode;
    if (mode == 0)
        mode = dtx_tc_preferred(K, P, L) ? 1 : 3;
    if (mode == 1 || mode == 2) {
        const cudaError_t e =
            launch_dtx_tc(D, X, K, P, L, T, mode, beta0, r_out, absmax_bits, x2sum, err, s, ex);
        if (e != cudaErrorNotSupported)
            return e;
        cudaGetLastError();
    }
    return launch_dtx(D, X, K, P, L, T, beta0, r_out, absmax_bits, x2sum, s);
}

}  // namespace csc
