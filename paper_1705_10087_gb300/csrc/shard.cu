// One shard of a signal cut across processes (include/csc_shard.h): DICOD's
// partition of the signal into contiguous runs of segments, one run per
// worker (Sec. 2.2, Alg. 2), with the worker-to-worker messages of updates
// near a border replaced by a halo exchange between phases.
//
// A shard holds the columns it owns plus up to L-1 columns on each side (its
// halo).  During a phase its segments apply Eq. beta_up to every column of
// their update window, halo included; the halo's r entries start at 0 and so
// accumulate exactly the change the neighbour must apply to the columns it
// owns there.  Between phases the caller moves these accumulated changes to
// the neighbours (csc_shard_halo_out / csc_shard_halo_in).  The phase
// schedule is global (segment m runs in phase m mod c on whichever shard owns
// it), so a column never receives changes from two active segments in one
// phase and the exchanged changes land in segments that were idle: the
// sharded solve performs the single-process solve's arithmetic, with the
// border additions grouped per phase.  Before an exact resync and before the
// objective, the caller also moves the Z values within L-1 of each border
// (csc_shard_z_out / csc_shard_z_in), since both need Z over the window.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <vector>

#include "csc_internal.cuh"
#include "csc_shard.h"
#include "handle.cuh"
#include "host_util.cuh"

using namespace csc;

int csc_record_error(int code, const char *fmt, ...);

namespace {

#define SH_CUDA(expr)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return csc_record_error(e_ == cudaErrorMemoryAllocation ? CSC_ENOMEM : CSC_ECUDA, \
                                    "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),  \
                                    __FILE__, __LINE__);                                    \
    } while (0)

#define SH_ON_DEVICE(h)                                                                 \
    csc::DeviceGuard dev_guard_((h)->device);                                           \
    if (dev_guard_.err != cudaSuccess)                                                  \
        return csc_record_error(CSC_ECUDA, "cudaSetDevice(%d) failed: %s", (h)->device, \
                                cudaGetErrorString(dev_guard_.err))

int phases_of(int64_t Tz, int M, int L)
{
    if (M <= 1)
        return 1;
    const int64_t wmin = Tz / M;
    const int64_t need = 2 * (int64_t)L - 2;
    const int64_t c = 1 + (need + wmin - 1) / wmin;
    return (int)(c > M ? M : c);
}

// r[k][c0 + j] += in[k][j] for j < w (in: [K][w]); the segments of the shard
// whose columns receive a nonzero change become dirty (they must be visited).
__global__ void halo_add_kernel(float *__restrict__ r, int64_t ld, int K, int64_t c0, int64_t w,
                                const float *__restrict__ in, const int64_t *__restrict__ seg_s,
                                const int64_t *__restrict__ seg_e, int nseg,
                                unsigned char *__restrict__ dirty,
                                unsigned char *__restrict__ touched)
{
    const int64_t n = (int64_t)K * w;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / w, j = i % w;
        const float v = in[i];
        if (v == 0.f)
            continue;
        const int64_t t = c0 + j;
        r[k * ld + t] += v;
        // the shard's segments are few near a border: find the one holding t
        int lo = 0, hi = nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (seg_s[mid] <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        if (seg_s[lo] <= t && t < seg_e[lo]) {
            dirty[lo] = 1;
            touched[lo] = 1;
        }
    }
}

bool plan_equal(const csc_shard_plan &a, const csc_shard_plan &b)
{
    return std::memcmp(&a, &b, sizeof a) == 0;
}

// Device pointer for a caller's halo buffer of n <= K (L-1) floats: itself
// when it is device memory, else slot `slot` (0 or 1) of the handle's staging
// buffer, filled from it.
int staged(csc_handle_t h, const float *p, size_t n, size_t slot, float **out)
{
    if (is_device_pointer(p)) {
        *out = const_cast<float *>(p);
        return CSC_OK;
    }
    const size_t per = (size_t)h->K * (size_t)std::max(h->L - 1, 1);
    SH_CUDA(grow(&h->shard.stage, &h->shard.cap_stage, 2 * per));
    *out = h->shard.stage + slot * per;
    SH_CUDA(cudaMemcpyAsync(*out, p, sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
    return CSC_OK;
}

int require_shard(csc_handle_t h, const char *who)
{
    if (!h)
        return csc_record_error(CSC_EINVAL, "%s: null handle", who);
    if (!h->initialized || !h->shard.on)
        return csc_record_error(CSC_ESTATE, "%s: call csc_shard_init first", who);
    return CSC_OK;
}

}  // namespace

extern "C" {

int csc_shard_plan_make(int64_t T, int L, int M, int world, int rank, csc_shard_plan *pl)
{
    if (!pl || L < 1 || T < L || world < 1 || rank < 0 || rank >= world || M < 0)
        return csc_record_error(CSC_EINVAL, "csc_shard_plan_make: bad arguments");
    const int64_t Tz = T - L + 1;
    if (M == 0)
        M = (int)std::max<int64_t>(1, std::min<int64_t>(Tz / std::max(1, 2 * L - 2), 1 << 30));
    if (M > Tz || world > M)
        return csc_record_error(CSC_EINVAL,
                                "csc_shard_plan_make: need world <= M <= Tz (got %d, %d, %lld)",
                                world, M, (long long)Tz);
    const int64_t H = L - 1;
    // every shard must own at least L-1 columns, so that a halo is owned by
    // one neighbour only
    for (int q = 0; q < world; q++) {
        const int s0 = (int)((int64_t)q * M / world), s1 = (int)((int64_t)(q + 1) * M / world);
        if (seg_start(Tz, M, s1) - seg_start(Tz, M, s0) < std::max<int64_t>(H, 1))
            return csc_record_error(CSC_EINVAL,
                                    "csc_shard_plan_make: shard %d owns fewer than L-1 columns",
                                    q);
    }
    csc_shard_plan p;
    std::memset(&p, 0, sizeof p);
    p.T = T;
    p.Tz = Tz;
    p.L = L;
    p.M = M;
    p.phases = phases_of(Tz, M, L);
    p.world = world;
    p.rank = rank;
    p.seg_first = (int)((int64_t)rank * M / world);
    p.seg_count = (int)((int64_t)(rank + 1) * M / world) - p.seg_first;
    p.col_first = seg_start(Tz, M, p.seg_first);
    const int64_t col_end = seg_start(Tz, M, p.seg_first + p.seg_count);
    p.col_count = col_end - p.col_first;
    p.halo_left = std::min(H, p.col_first);
    p.halo_right = std::min(H, Tz - col_end);
    p.x_first = p.col_first - p.halo_left;
    p.x_count = col_end + p.halo_right - p.x_first + L - 1;
    *pl = p;
    return CSC_OK;
}

int csc_shard_init(csc_handle_t h, const csc_shard_plan *plan, const float *X, double lambda)
{
    if (!h || !plan || !X)
        return csc_record_error(CSC_EINVAL, "csc_shard_init: null argument");
    csc_shard_plan chk;
    if (csc_shard_plan_make(plan->T, plan->L, plan->M, plan->world, plan->rank, &chk) != CSC_OK ||
        !plan_equal(chk, *plan) || plan->L != h->L)
        return csc_record_error(CSC_EINVAL,
                                "csc_shard_init: the plan is not csc_shard_plan_make's for "
                                "this handle's atoms");
    int rc = csc_init(h, X, plan->x_count, lambda, nullptr);
    if (rc != CSC_OK)
        return rc;
    SH_ON_DEVICE(h);
    cudaStream_t s = h->stream;
    ShardState &sh = h->shard;
    sh.Tz_global = plan->Tz;
    sh.T_global = plan->T;
    sh.M_global = plan->M;
    sh.seg_first = plan->seg_first;
    sh.seg_count = plan->seg_count;
    sh.col_first = plan->col_first;
    sh.col_count = plan->col_count;
    sh.hl = plan->halo_left;
    sh.hr = plan->halo_right;
    sh.last = plan->col_first + plan->col_count == plan->Tz;
    sh.g = 0;
    const int L = h->L, c = plan->phases;
    // the owned segments in local columns, and the phase lists by global index
    std::vector<int64_t> seg_s(sh.seg_count), seg_e(sh.seg_count);
    std::vector<int> seg_sig(sh.seg_count, 0), list;
    std::vector<int> off(c + 1, 0);
    int w_max = 1;
    for (int i = 0; i < sh.seg_count; i++) {
        const int m = sh.seg_first + i;
        seg_s[i] = seg_start(plan->Tz, plan->M, m) - sh.col_first + sh.hl;
        seg_e[i] = seg_start(plan->Tz, plan->M, m + 1) - sh.col_first + sh.hl;
        w_max = std::max<int>(w_max, (int)(seg_e[i] - seg_s[i]));
    }
    for (int p = 0; p < c; p++) {
        off[p] = (int)list.size();
        for (int i = 0; i < sh.seg_count; i++)
            if ((sh.seg_first + i) % c == p)
                list.push_back(i);
    }
    off[c] = (int)list.size();
    SH_CUDA(upload(&h->d_seg_s, &h->cap_seg_s, seg_s, s));
    SH_CUDA(upload(&h->d_seg_e, &h->cap_seg_e, seg_e, s));
    SH_CUDA(upload(&h->d_seg_sig, &h->cap_seg_sig, seg_sig, s));
    SH_CUDA(upload(&h->d_phase_list, &h->cap_phase, list, s));
    SH_CUDA(grow(&h->dirty, &h->cap_dirty, (size_t)sh.seg_count));
    SH_CUDA(grow(&h->touched, &h->cap_touched, (size_t)sh.seg_count));
    SH_CUDA(cudaMemsetAsync(h->dirty, 1, (size_t)sh.seg_count, s));
    SH_CUDA(cudaMemsetAsync(h->touched, 1, (size_t)sh.seg_count, s));
    h->sigs[0].seg0 = 0;
    h->sigs[0].nseg = sh.seg_count;
    SH_CUDA(push_sigs(h, s));
    // resync tiles over the owned columns, objective tiles over the owned
    // samples (the last shard also owns the samples [Tz, T) of the signal)
    std::vector<int> rt_sig, ot_sig;
    std::vector<int64_t> rt_s, rt_e, ot_s, ot_e;
    const int64_t own_lo = sh.hl, own_hi = sh.hl + sh.col_count;
    for (int64_t t = own_lo; t < own_hi; t += kResyncCols) {
        rt_sig.push_back(0);
        rt_s.push_back(t);
        rt_e.push_back(own_hi);
    }
    const int64_t smp_hi = own_hi + (sh.last ? L - 1 : 0);
    for (int64_t t = own_lo; t < smp_hi; t += kTile) {
        ot_sig.push_back(0);
        ot_s.push_back(t);
        ot_e.push_back(smp_hi);
    }
    const std::vector<int64_t> ot_off{0, (int64_t)ot_s.size()};
    SH_CUDA(upload(&sh.d_rt_sig, &sh.cap_rt_sig, rt_sig, s));
    SH_CUDA(upload(&sh.d_rt_s, &sh.cap_rt_s, rt_s, s));
    SH_CUDA(upload(&sh.d_rt_e, &sh.cap_rt_e, rt_e, s));
    SH_CUDA(upload(&sh.d_ot_sig, &sh.cap_ot_sig, ot_sig, s));
    SH_CUDA(upload(&sh.d_ot_s, &sh.cap_ot_s, ot_s, s));
    SH_CUDA(upload(&sh.d_ot_e, &sh.cap_ot_e, ot_e, s));
    SH_CUDA(upload(&sh.d_ot_off, &sh.cap_ot_off, ot_off, s));
    sh.n_rt = (int64_t)rt_s.size();
    sh.n_ot = (int64_t)ot_s.size();
    SH_CUDA(grow(&h->partials, &h->cap_partials, 2 * (size_t)std::max<int64_t>(sh.n_ot, 1)));
    // the halo columns accumulate changes for the neighbours: start at 0
    const int64_t ld = h->Tz;
    if (sh.hl > 0)
        SH_CUDA(cudaMemset2DAsync(h->r, sizeof(float) * ld, 0, sizeof(float) * sh.hl, h->K, s));
    if (sh.hr > 0)
        SH_CUDA(cudaMemset2DAsync(h->r + own_hi, sizeof(float) * ld, 0, sizeof(float) * sh.hr,
                                  h->K, s));
    SH_CUDA(cudaMemsetAsync(h->sc, 0, offsetof(Scratch, red), s));  // trace ring, counters
    SH_CUDA(cudaStreamSynchronize(s));  // host tables outlive their uploads
    h->M = sh.seg_count;
    h->c = c;
    h->w_max = w_max;
    h->phase_off = off;
    h->plan_ok = false;  // csc_solve rebuilds an ordinary plan (and refuses shards)
    sh.on = true;
    h->z_is_zero = false;
    return CSC_OK;
}

int csc_shard_phase(csc_handle_t h, int p, double tol)
{
    int rc = require_shard(h, "csc_shard_phase");
    if (rc != CSC_OK)
        return rc;
    if (p < 0 || p >= h->c || !(tol > 0.0))
        return csc_record_error(CSC_EINVAL, "csc_shard_phase: need 0 <= p < phases, tol > 0");
    SH_ON_DEVICE(h);
    cudaStream_t s = h->stream;
    ShardState &sh = h->shard;
    if (h->sigs[0].tol != (float)tol) {
        h->sigs[0].tol = (float)tol;
        SH_CUDA(push_sigs(h, s));
        SH_CUDA(cudaStreamSynchronize(s));
    }
    const int cnt = h->phase_off[p + 1] - h->phase_off[p];
    const int64_t g = sh.g++;
    if (g >= kPhaseRing) {
        const int slot = (int)(g & (kPhaseRing - 1));
        SH_CUDA(cudaMemsetAsync(&h->sc->upd[slot], 0, sizeof(long long), s));
        SH_CUDA(cudaMemsetAsync(&h->sc->dec[slot], 0, sizeof(double), s));
        SH_CUDA(cudaMemsetAsync(&h->sc->tend[slot], 0, sizeof(unsigned long long), s));
    }
    if (cnt == 0)
        return CSC_OK;
    const PhaseConfig cfg = phase_config(h->K, h->L, h->w_max,
                                         h->opts.threads_per_segment == 32 ? 32 : 128);
    PhaseParams pp{};
    pp.sig = h->d_sig;
    pp.seg_sig = h->d_seg_sig;
    pp.C = h->C;
    pp.Ct = h->Ct;
    pp.norms = h->norms;
    pp.dirty = h->dirty;
    pp.touched = h->touched;
    pp.seg_s = h->d_seg_s;
    pp.seg_e = h->d_seg_e;
    pp.phase_list = h->d_phase_list + h->phase_off[p];
    pp.upd = h->sc->upd;
    pp.dec = h->sc->dec;
    pp.tend = h->sc->tend;
    pp.total = &h->sc->total;
    pp.visits = &h->sc->visits;
    pp.done = &h->sc->done;  // stays 0: convergence is decided across shards by the caller
    pp.max_updates = (long long)1 << 62;
    pp.M = h->M;
    pp.c = h->c;
    pp.p = p;
    pp.K = h->K;
    pp.Kp = coef_pad(h->K);
    pp.L = h->L;
    pp.g = (int)(g & 0x3fffffff);
    pp.g_round = pp.g;  // every launch starts a round: no in-kernel sweep test
    pp.u = h->opts.updates_per_visit ? h->opts.updates_per_visit : kDefaultMaxVisit;
    pp.w_max = h->w_max;
    SH_CUDA(launch_phase(pp, cfg, cnt, s));
    h->launches += 1;
    return CSC_OK;
}

int csc_shard_halo_out(csc_handle_t h, float *to_left, float *to_right)
{
    int rc = require_shard(h, "csc_shard_halo_out");
    if (rc != CSC_OK)
        return rc;
    ShardState &sh = h->shard;
    if ((sh.hl > 0 && !to_left) || (sh.hr > 0 && !to_right))
        return csc_record_error(CSC_EINVAL, "csc_shard_halo_out: null buffer for a halo");
    SH_ON_DEVICE(h);
    cudaStream_t s = h->stream;
    const size_t pitch = sizeof(float) * h->Tz;
    const int64_t right0 = sh.hl + sh.col_count;
    if (sh.hl > 0) {
        SH_CUDA(cudaMemcpy2DAsync(to_left, sizeof(float) * sh.hl, h->r, pitch,
                                  sizeof(float) * sh.hl, h->K, cudaMemcpyDefault, s));
        SH_CUDA(cudaMemset2DAsync(h->r, pitch, 0, sizeof(float) * sh.hl, h->K, s));
    }
    if (sh.hr > 0) {
        SH_CUDA(cudaMemcpy2DAsync(to_right, sizeof(float) * sh.hr, h->r + right0, pitch,
                                  sizeof(float) * sh.hr, h->K, cudaMemcpyDefault, s));
        SH_CUDA(cudaMemset2DAsync(h->r + right0, pitch, 0, sizeof(float) * sh.hr, h->K, s));
    }
    if ((sh.hl > 0 && !is_device_pointer(to_left)) || (sh.hr > 0 && !is_device_pointer(to_right)))
        SH_CUDA(cudaStreamSynchronize(s));
    return CSC_OK;
}

int csc_shard_halo_in(csc_handle_t h, const float *from_left, const float *from_right)
{
    int rc = require_shard(h, "csc_shard_halo_in");
    if (rc != CSC_OK)
        return rc;
    ShardState &sh = h->shard;
    if ((sh.hl > 0 && !from_left) || (sh.hr > 0 && !from_right))
        return csc_record_error(CSC_EINVAL, "csc_shard_halo_in: null buffer for a halo");
    SH_ON_DEVICE(h);
    cudaStream_t s = h->stream;
    const struct {
        const float *src;
        int64_t c0, w;
    } parts[2] = {{from_left, sh.hl, sh.hl},
                  {from_right, sh.hl + sh.col_count - sh.hr, sh.hr}};
    for (int i = 0; i < 2; i++) {
        if (parts[i].w == 0)
            continue;
        const size_t n = (size_t)h->K * parts[i].w;
        float *d = nullptr;
        rc = staged(h, parts[i].src, n, (size_t)i, &d);
        if (rc != CSC_OK)
            return rc;
        const int64_t blocks = std::min<int64_t>((int64_t)(n + 255) / 256, 1024);
        halo_add_kernel<<<(unsigned)blocks, 256, 0, s>>>(h->r, h->Tz, h->K, parts[i].c0,
                                                         parts[i].w, d, h->d_seg_s, h->d_seg_e,
                                                         sh.seg_count, h->dirty, h->touched);
        SH_CUDA(cudaGetLastError());
        h->launches += 1;
    }
    // the staging buffer is re-used by the next call
    SH_CUDA(cudaStreamSynchronize(s));
    return CSC_OK;
}

int csc_shard_z_out(csc_handle_t h, float *to_left, float *to_right)
{
    int rc = require_shard(h, "csc_shard_z_out");
    if (rc != CSC_OK)
        return rc;
    ShardState &sh = h->shard;
    if ((sh.hl > 0 && !to_left) || (sh.hr > 0 && !to_right))
        return csc_record_error(CSC_EINVAL, "csc_shard_z_out: null buffer for a halo");
    SH_ON_DEVICE(h);
    cudaStream_t s = h->stream;
    const size_t pitch = sizeof(float) * h->Tz;
    if (sh.hl > 0)
        SH_CUDA(cudaMemcpy2DAsync(to_left, sizeof(float) * sh.hl, h->Z + sh.hl, pitch,
                                  sizeof(float) * sh.hl, h->K, cudaMemcpyDefault, s));
    if (sh.hr > 0)
        SH_CUDA(cudaMemcpy2DAsync(to_right, sizeof(float) * sh.hr,
                                  h->Z + sh.hl + sh.col_count - sh.hr, pitch,
                                  sizeof(float) * sh.hr, h->K, cudaMemcpyDefault, s));
    SH_CUDA(cudaStreamSynchronize(s));
    return CSC_OK;
}

int csc_shard_z_in(csc_handle_t h, const float *from_left, const float *from_right)
{
    int rc = require_shard(h, "csc_shard_z_in");
    if (rc != CSC_OK)
        return rc;
    ShardState &sh = h->shard;
    if ((sh.hl > 0 && !from_left) || (sh.hr > 0 && !from_right))
        return csc_record_error(CSC_EINVAL, "csc_shard_z_in: null buffer for a halo");
    SH_ON_DEVICE(h);
    cudaStream_t s = h->stream;
    const size_t pitch = sizeof(float) * h->Tz;
    if (sh.hl > 0)
        SH_CUDA(cudaMemcpy2DAsync(h->Z, pitch, from_left, sizeof(float) * sh.hl,
                                  sizeof(float) * sh.hl, h->K, cudaMemcpyDefault, s));
    if (sh.hr > 0)
        SH_CUDA(cudaMemcpy2DAsync(h->Z + sh.hl + sh.col_count, pitch, from_right,
                                  sizeof(float) * sh.hr, sizeof(float) * sh.hr, h->K,
                                  cudaMemcpyDefault, s));
    SH_CUDA(cudaStreamSynchronize(s));
    return CSC_OK;
}

int csc_shard_updates(csc_handle_t h, int64_t *total)
{
    int rc = require_shard(h, "csc_shard_updates");
    if (rc != CSC_OK)
        return rc;
    if (!total)
        return csc_record_error(CSC_EINVAL, "csc_shard_updates: null argument");
    SH_ON_DEVICE(h);
    long long v = 0;
    SH_CUDA(cudaMemcpyAsync(&v, &h->sc->total, sizeof v, cudaMemcpyDeviceToHost, h->stream));
    SH_CUDA(cudaStreamSynchronize(h->stream));
    *total = v;
    return CSC_OK;
}

int csc_shard_resync(csc_handle_t h, double tol, double *max_dz)
{
    int rc = require_shard(h, "csc_shard_resync");
    if (rc != CSC_OK)
        return rc;
    if (!max_dz || !(tol > 0.0))
        return csc_record_error(CSC_EINVAL, "csc_shard_resync: need tol > 0 and an output");
    SH_ON_DEVICE(h);
    cudaStream_t s = h->stream;
    ShardState &sh = h->shard;
    SH_CUDA(cudaMemsetAsync(h->sc->red, 0, sizeof(h->sc->red), s));
    Tiles tiles{sh.d_rt_sig, sh.d_rt_s, sh.n_rt, sh.d_rt_e};
    // the owned columns only (the halo keeps the changes still to send); the
    // nonzeros are gathered by scanning Z, halo columns included
    SH_CUDA(launch_resync(h->d_sig, tiles, h->Ct, h->norms, h->K, h->L, 1, h->sc->red, 0, nullptr,
                          0.f, nullptr, nullptr, NzLists{nullptr, nullptr}, s));
    h->launches += 1;
    // every owned segment is visited again in the next round
    SH_CUDA(cudaMemsetAsync(h->dirty, 1, (size_t)sh.seg_count, s));
    unsigned long long red[8];
    SH_CUDA(cudaMemcpyAsync(red, h->sc->red, sizeof red, cudaMemcpyDeviceToHost, s));
    SH_CUDA(cudaStreamSynchronize(s));
    if (int rc = finish_init(h))  // (beta0 came before this resync in the stream)
        return rc;
    double v[5];
    std::memcpy(v, red, sizeof v);
    max_dz[0] = v[4];
    return CSC_OK;
}

int csc_shard_objective(csc_handle_t h, double *out)
{
    int rc = require_shard(h, "csc_shard_objective");
    if (rc != CSC_OK)
        return rc;
    if (!out)
        return csc_record_error(CSC_EINVAL, "csc_shard_objective: null argument");
    SH_ON_DEVICE(h);
    cudaStream_t s = h->stream;
    ShardState &sh = h->shard;
    Tiles tiles{sh.d_ot_sig, sh.d_ot_s, sh.n_ot, sh.d_ot_e};
    SH_CUDA(launch_objective(h->D, h->d_sig, 1, tiles, sh.d_ot_off, h->K, h->P, h->L, h->Z,
                             nullptr, h->partials, h->d_E, s));
    h->launches += 2;
    SH_CUDA(cudaMemcpyAsync(out, h->d_E, sizeof(double), cudaMemcpyDeviceToHost, s));
    SH_CUDA(cudaStreamSynchronize(s));
    return CSC_OK;
}

int csc_shard_get_z(csc_handle_t h, float *Z_out)
{
    int rc = require_shard(h, "csc_shard_get_z");
    if (rc != CSC_OK)
        return rc;
    if (!Z_out)
        return csc_record_error(CSC_EINVAL, "csc_shard_get_z: null argument");
    SH_ON_DEVICE(h);
    ShardState &sh = h->shard;
    SH_CUDA(cudaMemcpy2DAsync(Z_out, sizeof(float) * sh.col_count, h->Z + sh.hl,
                              sizeof(float) * h->Tz, sizeof(float) * sh.col_count, h->K,
                              cudaMemcpyDefault, h->stream));
    SH_CUDA(cudaStreamSynchronize(h->stream));
    return CSC_OK;
}

}  // extern "C"
