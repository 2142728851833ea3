// C ABI entry points (include/csc.h) and the host-side orchestration of the
// solver: handle state, pointer-kind detection, signal tables and segment
// plans, the phase loop with its convergence polls and resync rounds.
//
// A problem is a batch of n >= 1 signals concatenated in time (csc_init is the
// n = 1 case).  Each signal is described to the kernels by a SigDesc pointing
// into the concatenated arrays (row stride = the concatenation's width), so
// the kernels solve n separate problems; the L-1 columns after each signal's
// last valid column belong to none of them and Z stays 0 there.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "csc_internal.cuh"
#include "handle.cuh"
#include "host_util.cuh"

using namespace csc;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CSC_CUDA(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? CSC_ENOMEM : CSC_ECUDA,        \
                        "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                       \
    } while (0)

// Switches to the handle's device for the rest of the calling scope (the
// caller's device is restored on return) and fails if the switch fails.
#define CSC_ON_DEVICE(dev)                                                               \
    csc::DeviceGuard dev_guard_(dev);                                                    \
    if (dev_guard_.err != cudaSuccess)                                                   \
        return fail(CSC_ECUDA, "cudaSetDevice(%d) failed: %s", (int)(dev),                \
                    cudaGetErrorString(dev_guard_.err))

// Phases of the schedule for one signal: co-active segments m, m' (m == m'
// mod c) must leave at least 2L-2 samples between them, (c-1) w_min >= 2L-2.
int phase_count_host(int64_t Tz, int M, int L)
{
    if (M <= 1)
        return 1;
    const int64_t wmin = Tz / M;
    if (wmin < 1)
        return -1;
    const int64_t need = 2 * (int64_t)L - 2;
    int64_t c = 1 + (need + wmin - 1) / wmin;
    return (int)(c > M ? M : c);
}

int64_t auto_width(int L)
{
    return 2 * (int64_t)L - 2 > 1 ? 2 * (int64_t)L - 2 : 1;
}

// Threads per segment when the options leave it automatic: a block (the
// one-warp form measured 2.2x slower per phase launch on the long signal,
// 94.8 vs 43.7 us: its lanes apply up to four window columns each in turn,
// which costs more than the block barrier it saves; csc_autotune tries both).
constexpr int kAutoThreadsPerSegment = 128;

int auto_segments(int64_t Tz, int L)
{
    int64_t M = Tz / auto_width(L);
    if (M < 1)
        M = 1;
    if (M > (1 << 30))
        M = 1 << 30;
    return (int)M;
}

}  // namespace

// Error recording for entry points defined in other translation units.
int csc_record_error(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

namespace {

int threads_per_segment(csc_handle_t h)
{
    return h->opts.threads_per_segment ? h->opts.threads_per_segment : kAutoThreadsPerSegment;
}

// Segments of every signal, their lambdas and the per-phase lists.
int build_plan(csc_handle_t h)
{
    if (h->plan_ok)
        return CSC_OK;
    cudaStream_t s = h->stream;
    const int L = h->L;
    if (h->M > 0 && h->plan_a == h->a && h->plan_L == L &&
        h->plan_segments == h->opts.segments && h->plan_width == h->opts.segment_width) {
        // same signals and options: the device tables are still those of this plan
        for (int i = 0; i < h->n; i++) {
            h->sigs[i].seg0 = h->plan_seg0[i];
            h->sigs[i].nseg = h->plan_nseg[i];
        }
        CSC_CUDA(push_sigs(h, s));
        h->plan_ok = true;
        return CSC_OK;
    }
    std::vector<int64_t> seg_s, seg_e;
    std::vector<int> seg_sig;
    std::vector<int> local;
    int c = 1;
    for (int i = 0; i < h->n; i++) {
        const int64_t Tzi = h->a[i + 1] - h->a[i] - L + 1;
        int Mi;
        if (h->n == 1 && h->opts.segments > 0) {
            Mi = h->opts.segments;
            if (Mi > Tzi)
                return fail(CSC_EINVAL, "csc_solve: %d segments exceed Tz = %lld", Mi,
                            (long long)Tzi);
        } else {
            const int64_t w = h->opts.segment_width > 0 ? h->opts.segment_width : auto_width(L);
            Mi = (int)std::max<int64_t>(1, Tzi / w);
        }
        c = std::max(c, phase_count_host(Tzi, Mi, L));
        h->sigs[i].seg0 = (int)seg_s.size();
        h->sigs[i].nseg = Mi;
        for (int m = 0; m < Mi; m++) {
            // columns local to the signal
            seg_s.push_back(seg_start(Tzi, Mi, m));
            seg_e.push_back(seg_start(Tzi, Mi, m + 1));
            seg_sig.push_back(i);
            local.push_back(m);
        }
    }
    const int M = (int)seg_s.size();
    int w_max = 1;
    for (int m = 0; m < M; m++)
        w_max = std::max<int>(w_max, (int)(seg_e[m] - seg_s[m]));
    std::vector<int> list;
    std::vector<int> off(c + 1, 0);
    for (int p = 0; p < c; p++) {
        off[p] = (int)list.size();
        for (int m = 0; m < M; m++)
            if (local[m] % c == p)
                list.push_back(m);
    }
    off[c] = (int)list.size();
    CSC_CUDA(upload(&h->d_seg_s, &h->cap_seg_s, seg_s, s));
    CSC_CUDA(upload(&h->d_seg_e, &h->cap_seg_e, seg_e, s));
    CSC_CUDA(upload(&h->d_seg_sig, &h->cap_seg_sig, seg_sig, s));
    CSC_CUDA(push_sigs(h, s));
    CSC_CUDA(upload(&h->d_phase_list, &h->cap_phase, list, s));
    CSC_CUDA(grow(&h->dirty, &h->cap_dirty, (size_t)M));
    CSC_CUDA(grow(&h->touched, &h->cap_touched, (size_t)M));
    {
        int most = 0;
        for (int p = 0; p < c; p++)
            most = std::max(most, off[p + 1] - off[p]);
        CSC_CUDA(grow(&h->d_queue, &h->cap_queue, (size_t)most));
    }
    CSC_CUDA(grow(&h->tile_rep, &h->cap_tile_rep, 5 * (size_t)h->nrtiles));
    // the host vectors must outlive the asynchronous copies
    CSC_CUDA(cudaStreamSynchronize(s));
    h->M = M;
    h->c = c;
    h->w_max = w_max;
    h->phase_off = off;
    h->plan_a = h->a;
    h->plan_L = L;
    h->plan_segments = h->opts.segments;
    h->plan_width = h->opts.segment_width;
    h->plan_seg0.resize(h->n);
    h->plan_nseg.resize(h->n);
    for (int i = 0; i < h->n; i++) {
        h->plan_seg0[i] = h->sigs[i].seg0;
        h->plan_nseg[i] = h->sigs[i].nseg;
    }
    h->plan_ok = true;
    return CSC_OK;
}

// Per-signal objectives of Zd into pinned h->E_pin, not waited for;
// lists_current: the resync bucket lists describe Zd (no change since).
int objectives_async(csc_handle_t h, const float *Zd, bool lists_current)
{
    cudaStream_t s = h->stream;
    if (h->cap_E_pin < (size_t)h->n) {
        CSC_CUDA(cudaStreamSynchronize(s));  // (the old block may still be written)
        if (h->E_pin)
            cudaFreeHost(h->E_pin);
        h->E_pin = nullptr;
        h->cap_E_pin = 0;
        CSC_CUDA(cudaHostAlloc(&h->E_pin, sizeof(double) * h->n, cudaHostAllocDefault));
        h->cap_E_pin = (size_t)h->n;
    }
    const bool lists = lists_current && Zd == h->Z;
    CSC_CUDA(launch_objective(h->D, h->d_sig, h->n, h->obj_tiles(), h->d_tile_off, h->K, h->P,
                              h->L, h->Z, Zd == h->Z ? nullptr : Zd, h->partials, h->d_E, s,
                              lists ? h->nz_lists() : NzLists{nullptr, nullptr},
                              lists ? h->d_rtile_off : nullptr));
    h->launches += 2;
    CSC_CUDA(cudaMemcpyAsync(h->E_pin, h->d_E, sizeof(double) * h->n, cudaMemcpyDeviceToHost, s));
    return CSC_OK;
}

// h->E_sig from E_pin (after the stream has been waited for), and their sum.
double objectives_done(csc_handle_t h)
{
    double t = 0.0;
    for (int i = 0; i < h->n; i++) {
        h->E_sig[i] = h->E_pin[i];
        t += h->E_pin[i];
    }
    return t;
}

// Per-signal objectives into h->E_sig (and their sum).
int objectives(csc_handle_t h, const float *Zd, double *sum)
{
    cudaStream_t s = h->stream;
    CSC_CUDA(launch_objective(h->D, h->d_sig, h->n, h->obj_tiles(), h->d_tile_off, h->K, h->P,
                              h->L, h->Z, Zd == h->Z ? nullptr : Zd, h->partials, h->d_E, s));
    h->launches += 2;
    CSC_CUDA(cudaMemcpyAsync(h->E_sig.data(), h->d_E, sizeof(double) * h->n,
                             cudaMemcpyDeviceToHost, s));
    CSC_CUDA(cudaStreamSynchronize(s));
    double t = 0.0;
    for (double v : h->E_sig)
        t += v;
    *sum = t;
    return CSC_OK;
}

template <class T>
void append_bytes(std::vector<unsigned char> &v, const T &x)
{
    const unsigned char *b = reinterpret_cast<const unsigned char *>(&x);
    v.insert(v.end(), b, b + sizeof(T));
}

// One poll batch, S sweeps of the c phases, as direct launches with the given
// launch indices (gp.g_dev == NULL) or, while capturing, with indices offset
// from the device counters.
int issue_batch(csc_handle_t h, PhaseParams gp, const PhaseConfig &cfg, int S, int resident,
                int64_t g0, int64_t g_round, cudaStream_t s)
{
    const int c = h->c;
    for (int i = 0; i < S; i++)
        for (int p = 0; p < c; p++) {
            const int64_t g = g0 + (int64_t)i * c + p;
            gp.p = p;
            gp.g = (int)g;
            gp.g_round = (int)g_round;
            gp.phase_list = h->d_phase_list + h->phase_off[p];
            const int cnt = h->phase_off[p + 1] - h->phase_off[p];
            if (cnt > 4 * resident) {
                CSC_CUDA(launch_phase_drain(gp, cfg, cnt, resident, s));
                h->launches += 2;
            } else {
                CSC_CUDA(launch_phase(gp, cfg, cnt, s));
                h->launches += 1;
            }
        }
    return CSC_OK;
}

// The graph of a CD round for these parameters: a while loop over poll
// batches (S sweeps of the c phases), each ended by launch_round_step, which
// stops the loop on the round's stopping rules (the limits in
// Scratch::round_lim), so that the host waits once per round instead of once
// per batch.  Captured the second time a plan is solved and re-used while
// nothing it depends on changes (same buffers, plan, options).
int batch_graph(csc_handle_t h, const PhaseParams &pp, const PhaseConfig &cfg, int S,
                int resident, int *gctr, cudaGraphExec_t *out)
{
    PhaseParams gp = pp;
    gp.g_dev = gctr;
    gp.g_round_dev = gctr + 1;
    gp.g = 0;
    gp.g_round = 0;
    gp.p = 0;
    gp.phase_list = nullptr;
    std::vector<unsigned char> key;
    append_bytes(key, gp);
    append_bytes(key, cfg.block);
    append_bytes(key, cfg.smem);
    append_bytes(key, cfg.tile_in_smem);
    append_bytes(key, S);
    append_bytes(key, resident);
    append_bytes(key, h->c);
    for (int o : h->phase_off)
        append_bytes(key, o);
    if (h->gexec && key == h->gkey) {
        *out = h->gexec;
        return CSC_OK;
    }
    // a plan is captured the second time it is solved: a one-off plan (a new
    // signal length every solve) runs direct launches and pays no capture
    if (key != h->gkey_seen) {
        h->gkey_seen = key;
        *out = nullptr;
        return CSC_OK;
    }
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
        h->gkey.clear();
    }
    const int64_t launches = h->launches;
    if (!h->cap_stream)
        CSC_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaStream_t s = h->cap_stream;
    cudaGraph_t graph = nullptr;
    CSC_CUDA(cudaGraphCreate(&graph, 0));
    // while (cond) { one poll batch; launch_round_step }, cond = 1 at each launch
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess)
        e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    int rc = CSC_OK;
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = issue_batch(h, gp, cfg, S, resident, 0, 0, s);
            cudaError_t e2 = cudaSuccess;
            if (rc == CSC_OK)
                e2 = launch_round_step(cond, gctr, S * h->c, &h->sc->done, &h->sc->total,
                                       h->sc->round_lim, s);
            cudaGraph_t captured = nullptr;
            e = cudaStreamEndCapture(s, &captured);
            if (e == cudaSuccess)
                e = e2;
        }
    }
    h->launches = launches;  // captured, not launched
    if (rc != CSC_OK || e != cudaSuccess) {
        cudaGraphDestroy(graph);
        if (rc != CSC_OK)
            return rc;
        CSC_CUDA(e);
    }
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    CSC_CUDA(e);
    h->gkey = key;
    *out = h->gexec;
    return CSC_OK;
}

int set_lambdas(csc_handle_t h, const double *lambda, bool push)
{
    for (int i = 0; i < h->n; i++)
        if (!(lambda[i] > 0.0) || !std::isfinite(lambda[i]))
            return fail(CSC_EINVAL, "lambda[%d] must be positive and finite", i);
    h->lam.assign(lambda, lambda + h->n);
    for (int i = 0; i < h->n; i++) {
        h->sigs[i].lam = (float)h->lam[i];
        h->sigs[i].lam_d = h->lam[i];
    }
    if (push)
        CSC_CUDA(push_sigs(h, h->stream));
    return CSC_OK;
}

}  // namespace

// Completes csc_init's asynchronous read-back: lambda_max per signal, the
// beta0 kernel's time and its give-up flag (an error surfaces here).
int finish_init(csc_handle_t h)
{
    if (!h->init_pending)
        return CSC_OK;
    CSC_CUDA(cudaEventSynchronize(h->ev_init));
    h->init_pending = false;
    if (h->init_pin[0]) {
        h->initialized = false;
        return fail(CSC_ETIMEOUT, "csc_init: the tensor-core beta0 kernel gave up waiting");
    }
    for (int i = 0; i < h->n; i++) {
        float v;
        std::memcpy(&v, &h->init_pin[1 + i], sizeof v);
        h->lmax[i] = v;
    }
    h->init_ms = -1.0;
    if (h->opts.time_kernels) {
        float ms = 0.f;
        CSC_CUDA(cudaEventElapsedTime(&ms, h->ev_i0, h->ev_i1));
        h->init_ms = ms;
    }
    return CSC_OK;
}

extern "C" {

const char *csc_last_error_string(void)
{
    return g_err.c_str();
}

void csc_default_opts(csc_opts *o)
{
    if (!o)
        return;
    std::memset(o, 0, sizeof *o);
    o->max_resyncs = -1;
}

int csc_plan(int64_t Tz, int L, int M, int *M_out, int *phases, int64_t *starts)
{
    if (Tz < 1 || L < 1 || M < 0)
        return fail(CSC_EINVAL, "csc_plan: need Tz >= 1, L >= 1, M >= 0");
    if (M == 0)
        M = auto_segments(Tz, L);
    if (M > Tz)
        return fail(CSC_EINVAL, "csc_plan: M = %d exceeds Tz = %lld", M, (long long)Tz);
    if (M_out)
        *M_out = M;
    if (phases)
        *phases = phase_count_host(Tz, M, L);
    if (starts)
        for (int m = 0; m <= M; m++)
            starts[m] = seg_start(Tz, M, m);
    return CSC_OK;
}

int csc_destroy(csc_handle_t h)
{
    if (!h)
        return CSC_OK;
    CSC_ON_DEVICE(h->device);
    if (h->stream)
        cudaStreamSynchronize(h->stream);
    void *bufs[] = {h->D,          h->C,          h->Ct,         h->norms,      h->X,
                    h->r,          h->beta0,      h->Z,          h->partials,   h->dirty,
                    h->tmpZ,       h->tmpB,       h->sc,         h->d_sig,      h->d_tile_s,
                    h->d_tile_off, h->d_tile_sig, h->d_rtile_s,  h->d_rtile_sig, h->d_rtile_off,
                    h->d_sig_a,    h->d_E,
                    h->d_lmax,     h->d_seg_s,    h->d_seg_e,    h->d_seg_sig,  h->d_phase_list,
                    h->touched,    h->tile_rep,   h->d_queue,    h->d_sig_alt,
                    h->nz_count,   h->nz_ent,     h->shard.d_rt_sig, h->shard.d_ot_sig,
                    h->shard.d_rt_s, h->shard.d_rt_e, h->shard.d_ot_s, h->shard.d_ot_e,
                    h->shard.d_ot_off, h->shard.stage};
    for (void *p : bufs)
        cudaFree(p);
    if (h->poll)
        cudaFreeHost(h->poll);
    if (h->init_pin)
        cudaFreeHost(h->init_pin);
    if (h->fin)
        cudaFreeHost(h->fin);
    if (h->E_pin)
        cudaFreeHost(h->E_pin);
    if (h->ev_init)
        cudaEventDestroy(h->ev_init);
    if (h->ev_copy)
        cudaEventDestroy(h->ev_copy);
    if (h->ev0)
        cudaEventDestroy(h->ev0);
    if (h->ev1)
        cudaEventDestroy(h->ev1);
    if (h->ev_i0)
        cudaEventDestroy(h->ev_i0);
    if (h->ev_i1)
        cudaEventDestroy(h->ev_i1);
    if (h->ev_r0)
        cudaEventDestroy(h->ev_r0);
    if (h->ev_r1)
        cudaEventDestroy(h->ev_r1);
    for (int i = 0; i < h->n_kev; i++)
        cudaEventDestroy(h->kev[i]);
    delete[] h->kev;
    if (h->gexec)
        cudaGraphExecDestroy(h->gexec);
    if (h->cap_stream)
        cudaStreamDestroy(h->cap_stream);
    delete h;
    return CSC_OK;
}

int csc_setup(csc_handle_t *hp, const float *D, int K, int P, int L, const csc_opts *opts,
              void *stream)
{
    csc::TraceRange trace_("csc_setup");
    if (!hp || !D)
        return fail(CSC_EINVAL, "csc_setup: null handle pointer or D");
    if (K < 1 || K > 256 || P < 1 || L < 1 || L > kMaxL)
        return fail(CSC_EINVAL, "csc_setup: need 1 <= K <= 256, P >= 1, 1 <= L <= %d (got %d,%d,%d)",
                    kMaxL, K, P, L);
    csc_opts o;
    csc_default_opts(&o);
    if (opts) {
        o = *opts;
        if (o.segments < 0 || o.updates_per_visit < 0 || o.max_resyncs < -1 ||
            o.sweeps_per_poll < 0 || o.max_sweeps < 0 || o.time_kernels < 0 ||
            o.time_kernels > 1 || o.segment_width < 0 || o.init_mode < 0 || o.init_mode > 3 ||
            o.launch_mode < 0 || o.launch_mode > 1 ||
            (o.threads_per_segment != 0 && o.threads_per_segment != 32 &&
             o.threads_per_segment != 128))
            return fail(CSC_EINVAL, "csc_setup: invalid options");
    }
    csc_handle_t h = *hp;
    bool fresh = false;
    if (!h) {
        h = new (std::nothrow) csc_handle_s();
        if (!h)
            return fail(CSC_ENOMEM, "csc_setup: host allocation failed");
        fresh = true;
        if (cudaGetDevice(&h->device) != cudaSuccess) {
            delete h;
            return fail(CSC_ECUDA, "csc_setup: no CUDA device");
        }
    }
    const int dev = h->device;
    csc::DeviceGuard dev_guard_(dev);
    if (dev_guard_.err != cudaSuccess) {
        if (fresh)
            delete h;
        return fail(CSC_ECUDA, "csc_setup: cudaSetDevice(%d) failed: %s", dev,
                    cudaGetErrorString(dev_guard_.err));
    }
    h->stream = (cudaStream_t)stream;
    h->opts = o;
    h->K = K;
    h->P = P;
    h->L = L;
    h->initialized = false;
    h->plan_ok = false;
    h->shard.on = false;
    auto body = [&]() -> int {
        CSC_CUDA(grow(&h->D, &h->cap_D, (size_t)K * P * L));
        CSC_CUDA(grow(&h->C, &h->cap_C, (size_t)K * K * (2 * L - 1)));
        CSC_CUDA(grow(&h->Ct, &h->cap_Ct, (size_t)K * (2 * L - 1) * coef_pad(K)));
        CSC_CUDA(grow(&h->norms, &h->cap_n, (size_t)K));
        if (!h->sc)
            CSC_CUDA(cudaMalloc(&h->sc, sizeof(Scratch)));
        if (!h->poll)
            CSC_CUDA(cudaHostAlloc(&h->poll, sizeof(Poll), cudaHostAllocDefault));
        if (!h->fin)
            CSC_CUDA(cudaHostAlloc(&h->fin, sizeof(Fin), cudaHostAllocDefault));
        if (!h->ev0)
            CSC_CUDA(cudaEventCreate(&h->ev0));
        if (!h->ev1)
            CSC_CUDA(cudaEventCreate(&h->ev1));
        if (!h->ev_copy)
            CSC_CUDA(cudaEventCreateWithFlags(&h->ev_copy, cudaEventDisableTiming));
        CSC_CUDA(copy_in(h->D, D, sizeof(float) * K * P * L, h->stream));
        CSC_CUDA(cudaEventRecord(h->ev_copy, h->stream));
        CSC_CUDA(launch_dtd(h->D, K, P, L, h->C, h->norms, h->stream));
        CSC_CUDA(launch_coef_by_lag(h->C, K, L, h->Ct, h->stream));
        h->launches += 2;
        // D may be reused once this returns (a copy from pinned host memory
        // is asynchronous: wait for it; the kernels run on)
        if (is_pinned_host(D))
            CSC_CUDA(cudaEventSynchronize(h->ev_copy));
        return CSC_OK;
    };
    int rc = body();
    if (rc != CSC_OK) {
        if (fresh)
            csc_destroy(h);
        return rc;
    }
    *hp = h;
    return CSC_OK;
}

int csc_init_batch(csc_handle_t h, const float *X, const int64_t *T, int n, const double *lambda,
                   const float *Z0)
{
    csc::TraceRange trace_("csc_init");
    if (!h || !X || !T || !lambda)
        return fail(CSC_EINVAL, "csc_init: null argument");
    if (n < 1)
        return fail(CSC_EINVAL, "csc_init: need at least one signal");
    int64_t Ttot = 0;
    for (int i = 0; i < n; i++) {
        if (T[i] < h->L)
            return fail(CSC_EINVAL, "csc_init: T[%d] = %lld < L = %d", i, (long long)T[i], h->L);
        Ttot += T[i];
    }
    const int64_t Tz = Ttot - h->L + 1;
    if (Tz >= ((int64_t)1 << 31) - 1)
        return fail(CSC_EINVAL, "csc_init: T - L + 1 must be below 2^31 - 1 columns");
    h->shard.on = false;  // csc_shard_init sets it again after this
    CSC_ON_DEVICE(h->device);
    if (h->init_pending) {
        // superseded by this call; its read-back buffer is about to be reused
        CSC_CUDA(cudaEventSynchronize(h->ev_init));
        h->init_pending = false;
    }
    h->initialized = false;
    h->plan_ok = false;
    cudaStream_t s = h->stream;
    h->n = n;
    h->T = Ttot;
    h->Tz = Tz;
    h->a.assign(n + 1, 0);
    for (int i = 0; i < n; i++)
        h->a[i + 1] = h->a[i] + T[i];
    const size_t nz = (size_t)h->K * Tz;
    CSC_CUDA(grow(&h->X, &h->cap_X, (size_t)h->P * Ttot));
    CSC_CUDA(grow(&h->r, &h->cap_r, nz));
    CSC_CUDA(grow(&h->beta0, &h->cap_beta0, nz));
    CSC_CUDA(grow(&h->Z, &h->cap_Z, nz));
    // descriptors into the concatenation and the tiles over each signal (the
    // stopping threshold of the previous solve is kept: unchanged descriptors
    // are not uploaded again)
    std::vector<float> tol_prev;
    for (const SigDesc &d : h->sigs)
        tol_prev.push_back(d.tol);
    h->sigs.assign(n, SigDesc{});
    for (int i = 0; i < n && i < (int)tol_prev.size(); i++)
        h->sigs[i].tol = tol_prev[i];
    // tiles over each signal: the objective's (kTile samples) and the
    // resync's (kResyncCols columns); the host keeps only the first tile of
    // each signal, the device expands the tables from it
    std::vector<int64_t> rtile_off(n + 1, 0);
    h->tile_off.assign(n + 1, 0);
    for (int i = 0; i < n; i++) {
        SigDesc &d = h->sigs[i];
        d.r = h->r + h->a[i];
        d.Z = h->Z + h->a[i];
        d.beta0 = h->beta0 + h->a[i];
        d.X = h->X + h->a[i];
        d.ld = Tz;
        d.ldx = Ttot;
        d.Tz = T[i] - h->L + 1;
        h->tile_off[i + 1] = h->tile_off[i] + (T[i] + kTile - 1) / kTile;
        rtile_off[i + 1] = rtile_off[i] + (d.Tz + kResyncCols - 1) / kResyncCols;
    }
    h->ntiles = h->tile_off[n];
    h->nrtiles = rtile_off[n];
    h->E_sig.assign(n, 0.0);
    h->lmax.assign(n, 0.0);
    if (h->tiles_a != h->a || h->tiles_L != h->L) {
        CSC_CUDA(upload(&h->d_tile_off, &h->cap_tile_off, h->tile_off, s));
        CSC_CUDA(upload(&h->d_rtile_off, &h->cap_rtile_off, rtile_off, s));
        CSC_CUDA(upload(&h->d_sig_a, &h->cap_sig_a, h->a, s));
        CSC_CUDA(grow(&h->d_tile_s, &h->cap_tile_s, (size_t)h->ntiles));
        CSC_CUDA(grow(&h->d_tile_sig, &h->cap_tile_sig, (size_t)h->ntiles));
        CSC_CUDA(grow(&h->d_rtile_s, &h->cap_rtile_s, (size_t)h->nrtiles));
        CSC_CUDA(grow(&h->d_rtile_sig, &h->cap_rtile_sig, (size_t)h->nrtiles));
        CSC_CUDA(launch_expand_tiles(h->d_tile_off, n, kTile, h->ntiles, h->d_tile_s,
                                     h->d_tile_sig, s));
        CSC_CUDA(launch_expand_tiles(h->d_rtile_off, n, kResyncCols, h->nrtiles, h->d_rtile_s,
                                     h->d_rtile_sig, s));
        h->launches += 2;
        h->tiles_a = h->a;
        h->tiles_L = h->L;
    }
    CSC_CUDA(grow(&h->d_E, &h->cap_E, (size_t)n));
    CSC_CUDA(grow(&h->d_lmax, &h->cap_lmax, (size_t)n));
    CSC_CUDA(grow(&h->partials, &h->cap_partials, 2 * (size_t)h->ntiles));
    CSC_CUDA(grow(&h->nz_count, &h->cap_nz_count, (size_t)h->nrtiles));
    CSC_CUDA(grow(&h->nz_ent, &h->cap_nz_ent, (size_t)h->nrtiles * kNzCap));
    {
        // d_sig is read by every kernel on the handle's problems (csc_objective
        // and csc_kkt may follow without a solve); unchanged descriptors are
        // not uploaded again
        int rc = set_lambdas(h, lambda, true);
        if (rc != CSC_OK)
            return rc;
    }
    if (h->cap_init_pin < (size_t)n + 1) {
        if (h->init_pin)
            cudaFreeHost(h->init_pin);
        h->init_pin = nullptr;
        h->cap_init_pin = 0;
        CSC_CUDA(cudaHostAlloc(&h->init_pin, sizeof(unsigned) * (n + 1), cudaHostAllocDefault));
        h->cap_init_pin = (size_t)n + 1;
    }
    if (!h->ev_init)
        CSC_CUDA(cudaEventCreateWithFlags(&h->ev_init, cudaEventDisableTiming));
    if (!h->ev_copy)
        CSC_CUDA(cudaEventCreateWithFlags(&h->ev_copy, cudaEventDisableTiming));
    CSC_CUDA(copy_in(h->X, X, sizeof(float) * h->P * Ttot, s));
    CSC_CUDA(cudaEventRecord(h->ev_copy, s));  // the caller's X has been read
    // x2, lmax_bits and tc_err (adjacent in Scratch) cleared in one memset
    static_assert(offsetof(Scratch, lmax_bits) == offsetof(Scratch, x2) + sizeof(double) &&
                      offsetof(Scratch, tc_err) == offsetof(Scratch, lmax_bits) + sizeof(unsigned),
                  "x2, lmax_bits, tc_err adjacent");
    CSC_CUDA(cudaMemsetAsync(&h->sc->x2, 0, offsetof(Scratch, tc_err) + sizeof(int) -
                                              offsetof(Scratch, x2), s));
    const bool timed = h->opts.time_kernels != 0;
    if (timed && !h->ev_i0) {
        CSC_CUDA(cudaEventCreate(&h->ev_i0));
        CSC_CUDA(cudaEventCreate(&h->ev_i1));
    }
    // a cold start (Z = 0) has r = beta0: the kernel writes both, and the
    // tensor-core kernel also zeroes Z and, for a batch, takes the per-signal
    // maxima (the kernel's overall maximum also covers the columns between
    // signals, which belong to no problem)
    Dtx0Extras ex;
    if (!Z0)
        ex.z_out = h->Z;
    if (n > 1) {
        CSC_CUDA(cudaMemsetAsync(h->d_lmax, 0, sizeof(unsigned) * n, s));
        ex.a = h->d_sig_a;
        ex.nsig = n;
        ex.lmax = h->d_lmax;
    }
    if (timed)
        CSC_CUDA(cudaEventRecord(h->ev_i0, s));
    CSC_CUDA(launch_dtx_any(h->D, h->X, h->K, h->P, h->L, Ttot, h->opts.init_mode, h->beta0,
                            Z0 ? nullptr : h->r, &h->sc->lmax_bits, &h->sc->x2, &h->sc->tc_err,
                            s, &ex));
    if (timed)
        CSC_CUDA(cudaEventRecord(h->ev_i1, s));
    h->launches += 1;
    if (n > 1 && !ex.done) {
        CSC_CUDA(launch_signal_absmax(h->d_sig, h->obj_tiles(), h->K, h->d_lmax, s));
        h->launches += 1;
    }
    if (Z0) {
        h->launches += 2;  // bucket lists + resync
        CSC_CUDA(copy_in(h->Z, Z0, sizeof(float) * nz, s));
        CSC_CUDA(cudaEventRecord(h->ev_copy, s));
        // the columns between signals belong to no problem: 0
        for (int i = 0; i + 1 < n; i++)
            CSC_CUDA(cudaMemset2DAsync(h->Z + h->a[i + 1] - h->L + 1, sizeof(float) * Tz, 0,
                                       sizeof(float) * (h->L - 1), h->K, s));
        CSC_CUDA(cudaMemsetAsync(h->sc->red, 0, sizeof(h->sc->red), s));
        CSC_CUDA(launch_resync(h->d_sig, h->resync_tiles(), h->Ct, h->norms, h->K, h->L, 1,
                               h->sc->red, 0, nullptr, 0.f, nullptr, nullptr, h->nz_lists(), s));
    } else if (!ex.done) {
        CSC_CUDA(cudaMemsetAsync(h->Z, 0, sizeof(float) * nz, s));
    }
    // read back without waiting (finish_init completes it): the stream goes
    // on to the solve while beta0 is computed
    CSC_CUDA(cudaMemcpyAsync(h->init_pin + 1, n > 1 ? h->d_lmax : &h->sc->lmax_bits,
                             sizeof(unsigned) * n, cudaMemcpyDeviceToHost, s));
    CSC_CUDA(cudaMemcpyAsync(h->init_pin, &h->sc->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CSC_CUDA(cudaEventRecord(h->ev_init, s));
    h->init_pending = true;
    // the inputs may be reused once this returns (a copy from pinned host
    // memory is asynchronous): wait for the copies, not for the kernels
    if (is_pinned_host(X) || (Z0 && is_pinned_host(Z0)))
        CSC_CUDA(cudaEventSynchronize(h->ev_copy));
    h->z_is_zero = Z0 == nullptr;
    h->initialized = true;
    return CSC_OK;
}

int csc_init(csc_handle_t h, const float *X, int64_t T, double lambda, const float *Z0)
{
    return csc_init_batch(h, X, &T, 1, &lambda, Z0);
}

int csc_set_lambda(csc_handle_t h, const double *lambda)
{
    if (!h || !lambda)
        return fail(CSC_EINVAL, "csc_set_lambda: null argument");
    if (!h->initialized)
        return fail(CSC_ESTATE, "csc_set_lambda: call csc_init first");
    CSC_ON_DEVICE(h->device);
    return set_lambdas(h, lambda, true);
}

int csc_lambda_max(csc_handle_t h, double *out)
{
    if (!h || !out)
        return fail(CSC_EINVAL, "csc_lambda_max: null argument");
    if (!h->initialized)
        return fail(CSC_ESTATE, "csc_lambda_max: call csc_init first");
    CSC_ON_DEVICE(h->device);
    if (int rc = finish_init(h))
        return rc;
    *out = *std::max_element(h->lmax.begin(), h->lmax.end());
    return CSC_OK;
}

int csc_lambda_max_batch(csc_handle_t h, double *out)
{
    if (!h || !out)
        return fail(CSC_EINVAL, "csc_lambda_max_batch: null argument");
    if (!h->initialized)
        return fail(CSC_ESTATE, "csc_lambda_max_batch: call csc_init first");
    CSC_ON_DEVICE(h->device);
    if (int rc = finish_init(h))
        return rc;
    std::copy(h->lmax.begin(), h->lmax.end(), out);
    return CSC_OK;
}

int csc_get_objectives(csc_handle_t h, double *out)
{
    if (!h || !out)
        return fail(CSC_EINVAL, "csc_get_objectives: null argument");
    if (!h->initialized)
        return fail(CSC_ESTATE, "csc_get_objectives: call csc_init first");
    std::copy(h->E_sig.begin(), h->E_sig.end(), out);
    return CSC_OK;
}

int csc_solve(csc_handle_t h, double tol, int64_t max_updates, float *Z_out, double *objective,
              csc_stats *stats)
{
    csc::TraceRange trace_("csc_solve");
    if (!h)
        return fail(CSC_EINVAL, "csc_solve: null handle");
    if (!h->initialized)
        return fail(CSC_ESTATE, "csc_solve: call csc_init first");
    if (!(tol > 0.0) || max_updates < 1)
        return fail(CSC_EINVAL, "csc_solve: need tol > 0 and max_updates >= 1");
    if (h->shard.on)
        return fail(CSC_ESTATE, "csc_solve: the handle holds a shard (use the csc_shard_* calls)");
    CSC_ON_DEVICE(h->device);
    cudaStream_t s = h->stream;
    const int64_t Tz = h->Tz;
    {
        int rc = build_plan(h);
        if (rc != CSC_OK)
            return rc;
    }
    const int M = h->M, c = h->c;
    const PhaseConfig cfg = phase_config(h->K, h->L, h->w_max, threads_per_segment(h));
    const int S = h->opts.sweeps_per_poll ? h->opts.sweeps_per_poll : 4;
    const int64_t max_sweeps = h->opts.max_sweeps ? h->opts.max_sweeps : 1000000;
    const int max_resyncs = h->opts.max_resyncs < 0 ? 3 : h->opts.max_resyncs;
    const bool timed = h->opts.time_kernels != 0;
    Scratch *sc = h->sc;
    const int64_t launches0 = h->launches;

    if (timed && h->n_kev < 2 * S * c) {
        for (int i = 0; i < h->n_kev; i++)
            cudaEventDestroy(h->kev[i]);
        delete[] h->kev;
        h->n_kev = 0;
        h->kev = new (std::nothrow) cudaEvent_t[2 * S * c];
        if (!h->kev)
            return fail(CSC_ENOMEM, "csc_solve: host allocation failed");
        for (int i = 0; i < 2 * S * c; i++) {
            CSC_CUDA(cudaEventCreate(&h->kev[i]));
            h->n_kev = i + 1;
        }
    }

    if (timed && !h->ev_r0) {
        CSC_CUDA(cudaEventCreate(&h->ev_r0));
        CSC_CUDA(cudaEventCreate(&h->ev_r1));
    }
    double resync_ms = 0.0, objective_ms = 0.0;
    // device time between ev_r0 and ev_r1 (recorded around one resync or objective)
    auto span_ms = [&](double *acc) -> int {
        float ms = 0.f;
        CSC_CUDA(cudaEventElapsedTime(&ms, h->ev_r0, h->ev_r1));
        *acc += ms;
        return CSC_OK;
    };
    CSC_CUDA(cudaEventRecord(h->ev0, s));
    // trace ring, counters and red zeroed (Scratch up to x2), every segment
    // dirty and, so that the first resync of the solve recomputes every tile,
    // touched; the start stamped
    CSC_CUDA(launch_solve_begin(reinterpret_cast<unsigned long long *>(sc),
                                (int64_t)(offsetof(Scratch, x2) / sizeof(unsigned long long)),
                                h->dirty, h->touched, M, &sc->tstart, s));
    h->launches += 1;
    const bool cold = h->z_is_zero;
    double E0 = 0.0;
    if (!cold) {
        int rc = objectives(h, h->Z, &E0);
        if (rc != CSC_OK)
            return rc;
    }
    h->z_is_zero = false;

    PhaseParams pp{};
    pp.C = h->C;
    pp.Ct = h->Ct;
    pp.Kp = coef_pad(h->K);
    pp.norms = h->norms;
    pp.dirty = h->dirty;
    pp.touched = h->touched;
    pp.qhead = sc->qhead;
    pp.qlen = sc->qhead + 1;
    pp.queue = h->d_queue;
    // phases with many more segments than resident blocks are drained from a
    // queue of the segments that need a visit by persistent blocks
    const int resident = phase_resident_blocks(cfg, h->K);
    pp.seg_s = h->d_seg_s;
    pp.seg_e = h->d_seg_e;
    pp.sig = h->d_sig;
    pp.seg_sig = h->d_seg_sig;
    pp.upd = sc->upd;
    pp.dec = sc->dec;
    pp.tend = sc->tend;
    pp.total = &sc->total;
    pp.visits = &sc->visits;
    pp.done = &sc->done;
    pp.max_updates = max_updates;
    pp.M = M;
    pp.c = c;
    pp.K = h->K;
    pp.L = h->L;
    pp.u = h->opts.updates_per_visit ? h->opts.updates_per_visit : kDefaultMaxVisit;
    // CD runs to tol/2 and a resync accepts at tol: coordinates left just under
    // the inner tolerance then stay under tol after the exact refresh, instead
    // of bouncing back above it round after round
    const float tol_inner = (float)(max_resyncs > 0 ? 0.5 * tol : tol);
    for (SigDesc &d : h->sigs)
        d.tol = tol_inner;
    CSC_CUDA(push_sigs(h, s));
    pp.w_max = h->w_max;

    int status = CSC_OK;
    bool converged = false, report_fresh = false;
    int resyncs = 0;
    int64_t drift_resyncs = 0;
    double drift = 0.0, phase_ms = 0.0;
    int64_t g = 0, effective = 0, phase_launches = 0;
    // a poll batch is replayed from a CUDA graph (launch indices from device
    // counters) while its indices stay inside the trace ring
    cudaGraphExec_t gexec = nullptr;
    if (h->opts.launch_mode == 0) {
        int rc = batch_graph(h, pp, cfg, S, resident, sc->gctr, &gexec);
        if (rc != CSC_OK)
            return rc;
        // (the launch counter gctr[0] starts at 0: solve_begin)
    }
    for (;;) {
        const int64_t g_round = g;
        // done cleared, the round's first launch index and the stopping rules
        // tested on the device (launch_round_step) set
        CSC_CUDA(launch_round_begin(&sc->done, sc->gctr, (int)g_round, sc->round_lim, max_updates,
                                    max_resyncs > 0 ? (long long)kDriftSweeps * c : 0,
                                    (long long)max_sweeps * c, kPhaseRing, s));
        h->launches += 1;
        bool round_done = false, forced = false;
        for (;;) {
            int nb = 0;  // launches in this poll batch
            const bool graphed = gexec && g + (int64_t)S * c <= kPhaseRing;
            if (graphed) {
                // the round runs on the device, batch after batch, until one of
                // the stopping rules tested below holds (launch_round_step)
                if (timed)
                    CSC_CUDA(cudaEventRecord(h->kev[0], s));
                CSC_CUDA(cudaGraphLaunch(gexec, s));
                if (timed)
                    CSC_CUDA(cudaEventRecord(h->kev[1], s));
                // (the graph's launches are counted after the poll)
            } else {
                for (int i = 0; i < S; i++)
                    for (int p = 0; p < c; p++) {
                        if (g >= kPhaseRing) {
                            const int slot = (int)(g & (kPhaseRing - 1));
                            CSC_CUDA(cudaMemsetAsync(&sc->upd[slot], 0, sizeof(long long), s));
                            CSC_CUDA(cudaMemsetAsync(&sc->dec[slot], 0, sizeof(double), s));
                            CSC_CUDA(cudaMemsetAsync(&sc->tend[slot], 0, sizeof(unsigned long long), s));
                        }
                        if (timed)
                            CSC_CUDA(cudaEventRecord(h->kev[2 * nb], s));
                        pp.phase_list = nullptr;
                        // one launch: S = 1 sweep restricted to phase p
                        PhaseParams one = pp;
                        one.p = p;
                        one.g = (int)g;
                        one.g_round = (int)g_round;
                        one.phase_list = h->d_phase_list + h->phase_off[p];
                        const int cnt = h->phase_off[p + 1] - h->phase_off[p];
                        if (cnt > 4 * resident) {
                            CSC_CUDA(launch_phase_drain(one, cfg, cnt, resident, s));
                            h->launches += 2;
                        } else {
                            CSC_CUDA(launch_phase(one, cfg, cnt, s));
                            h->launches += 1;
                        }
                        if (timed)
                            CSC_CUDA(cudaEventRecord(h->kev[2 * nb + 1], s));
                        nb++;
                        g++;
                    }
            }
            // total, done and the next launch index in one copy
            CSC_CUDA(cudaMemcpyAsync(h->poll, &sc->total, sizeof(Poll), cudaMemcpyDeviceToHost, s));
            CSC_CUDA(cudaStreamSynchronize(s));
            if (int rc = finish_init(h))  // (beta0 came before this poll in the stream)
                return rc;
            if (graphed) {
                // batches the device loop ran, each S sweeps of the c phases
                // and one round_step launch
                nb = (int)(h->poll->g_next - g);
                g = h->poll->g_next;
                int per_batch = 1;
                for (int p = 0; p < c; p++)
                    per_batch += S * ((h->phase_off[p + 1] - h->phase_off[p] > 4 * resident) ? 2 : 1);
                h->launches += (int64_t)(nb / (S * c)) * per_batch;
            }
            phase_launches += nb;
            if (timed) {
                const int pairs = graphed ? 1 : nb;
                for (int i = 0; i < pairs; i++) {
                    float ms = 0.f;
                    CSC_CUDA(cudaEventElapsedTime(&ms, h->kev[2 * i], h->kev[2 * i + 1]));
                    phase_ms += ms;
                }
            }
            if (h->poll->total >= max_updates && !h->poll->done) {
                status = CSC_NOT_CONVERGED;
                break;
            }
            if (h->poll->done) {
                // done = 1 + index of the launch that saw a full sweep without
                // updates: launches [g_round, done-1) did the work of this round
                effective += (h->poll->done - 1) - g_round;
                round_done = true;
                break;
            }
            if (g / c >= max_sweeps) {
                status = CSC_NOT_CONVERGED;
                break;
            }
            if (max_resyncs > 0 && g - g_round >= (int64_t)kDriftSweeps * c) {
                forced = true;
                break;
            }
        }
        if (!round_done && !forced) {
            effective += g - g_round;
            break;
        }
        if (forced)
            effective += g - g_round;
        // the loop settled after the last resync allowed: one more exact
        // refresh decides the status (no further CD round follows it)
        const bool last = round_done && resyncs >= max_resyncs;
        if (last && max_resyncs == 0) {
            converged = true;  // no resync requested: the float32 loop's own test
            break;
        }
        CSC_CUDA(cudaMemsetAsync(sc->red, 0, sizeof(sc->red), s));
        // segments come back dirty only where the refreshed state has a
        // coordinate at or above the inner tolerance (a round cut short keeps
        // the segments it still had to visit)
        if (round_done && !last)
            CSC_CUDA(cudaMemsetAsync(h->dirty, 0, (size_t)M, s));
        if (timed)
            CSC_CUDA(cudaEventRecord(h->ev_r0, s));
        CSC_CUDA(launch_resync(h->d_sig, h->resync_tiles(), h->Ct, h->norms, h->K, h->L, 1,
                               sc->red, 0, last ? nullptr : h->dirty, tol_inner, h->touched,
                               h->tile_rep, h->nz_lists(), s));
        if (timed)
            CSC_CUDA(cudaEventRecord(h->ev_r1, s));
        CSC_CUDA(cudaMemsetAsync(h->touched, 0, (size_t)M, s));
        h->launches += 2;
        unsigned long long red[8];
        CSC_CUDA(cudaMemcpyAsync(red, sc->red, sizeof red, cudaMemcpyDeviceToHost, s));
        CSC_CUDA(cudaStreamSynchronize(s));
        if (timed) {
            const int rc = span_ms(&resync_ms);
            if (rc != CSC_OK)
                return rc;
        }
        if (round_done)
            resyncs++;
        else
            drift_resyncs++;
        double d0, dz32;
        std::memcpy(&d0, &red[0], sizeof d0);
        std::memcpy(&dz32, &red[4], sizeof dz32);
        drift = d0 > drift ? d0 : drift;
        if (dz32 < tol || last) {
            // the exact check: every coordinate's change on the refreshed state
            // is below tol, or (after the last resync allowed) it is not
            converged = dz32 < tol;
            report_fresh = true;
            break;
        }
    }
    if (!report_fresh) {
        // optimality report against a fresh r, leaving r unchanged
        CSC_CUDA(cudaMemsetAsync(sc->red, 0, sizeof(sc->red), s));
        if (timed)
            CSC_CUDA(cudaEventRecord(h->ev_r0, s));
        CSC_CUDA(launch_resync(h->d_sig, h->resync_tiles(), h->Ct, h->norms, h->K, h->L, 0,
                               sc->red, 0, nullptr, 0.f, h->touched, h->tile_rep, h->nz_lists(), s));
        if (timed) {
            CSC_CUDA(cudaEventRecord(h->ev_r1, s));
            CSC_CUDA(cudaEventSynchronize(h->ev_r1));
            const int rc = span_ms(&resync_ms);
            if (rc != CSC_OK)
                return rc;
        }
        h->launches += 2;
    }
    CSC_CUDA(cudaEventRecord(h->ev1, s));
    // the objective, the copy of Z and the counters, then one wait
    if (timed)
        CSC_CUDA(cudaEventRecord(h->ev_r0, s));
    // (the last resync listed the nonzeros of this Z: the objective re-uses them)
    if (int rc = objectives_async(h, h->Z, true))
        return rc;
    if (timed)
        CSC_CUDA(cudaEventRecord(h->ev_r1, s));
    if (Z_out)
        CSC_CUDA(copy_out(Z_out, h->Z, sizeof(float) * h->K * Tz, s));
    Fin *fin = h->fin;
    CSC_CUDA(cudaMemcpyAsync(fin, &sc->total, sizeof(Fin), cudaMemcpyDeviceToHost, s));
    CSC_CUDA(cudaStreamSynchronize(s));
    const double E = objectives_done(h);
    if (timed) {
        const int rc = span_ms(&objective_ms);
        if (rc != CSC_OK)
            return rc;
    }
    unsigned long long red[8];
    std::memcpy(red, fin->red, sizeof red);
    const double x2 = fin->x2;
    const long long total = fin->total, visits = fin->visits;
    float ms = 0.f;
    CSC_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->g_used = g;
    h->E_start = cold ? 0.5 * x2 : E0;
    if (objective)
        *objective = E;
    if (stats) {
        double v[5];
        std::memcpy(v, red, sizeof v);
        stats->updates = total;
        stats->sweeps = (effective + c - 1) / c;
        stats->segments = M;
        stats->phases = c;
        stats->resyncs = resyncs;
        stats->converged = converged ? 1 : 0;
        stats->objective = E;
        stats->max_drift = drift;
        stats->kkt_zero_excess = v[1];
        stats->kkt_nonzero_gap = v[2];
        stats->max_delta_z = v[3];
        stats->solve_ms = ms;
        stats->phase_ms = phase_ms;
        stats->phase_launches = phase_launches;
        stats->visits = visits;
        stats->kernel_launches = h->launches - launches0;
        stats->drift_resyncs = drift_resyncs;
        stats->resync_ms = resync_ms;
        stats->objective_ms = objective_ms;
    }
    return status != CSC_OK ? status : (converged ? CSC_OK : CSC_NOT_CONVERGED);
}

int csc_autotune(csc_handle_t h, double tol, int64_t max_updates, csc_tune_result *out)
{
    csc::TraceRange trace_("csc_autotune");
    if (!h)
        return fail(CSC_EINVAL, "csc_autotune: null handle");
    if (!h->initialized)
        return fail(CSC_ESTATE, "csc_autotune: call csc_init first");
    if (!(tol > 0.0) || max_updates < 1)
        return fail(CSC_EINVAL, "csc_autotune: need tol > 0 and max_updates >= 1");
    CSC_ON_DEVICE(h->device);
    if (int rc = finish_init(h))
        return rc;
    cudaStream_t s = h->stream;
    const size_t nz = (size_t)h->K * h->Tz;
    // the starting point every candidate solves from
    const bool cold = h->z_is_zero;
    if (!cold) {
        CSC_CUDA(grow(&h->tmpZ, &h->cap_tmpZ, nz));
        CSC_CUDA(grow(&h->tmpB, &h->cap_tmpB, nz));
        CSC_CUDA(cudaMemcpyAsync(h->tmpZ, h->Z, sizeof(float) * nz, cudaMemcpyDeviceToDevice, s));
        CSC_CUDA(cudaMemcpyAsync(h->tmpB, h->r, sizeof(float) * nz, cudaMemcpyDeviceToDevice, s));
    }
    auto restore = [&]() -> int {
        if (cold) {
            CSC_CUDA(cudaMemsetAsync(h->Z, 0, sizeof(float) * nz, s));
            CSC_CUDA(cudaMemcpyAsync(h->r, h->beta0, sizeof(float) * nz, cudaMemcpyDeviceToDevice,
                                     s));
            h->z_is_zero = true;
        } else {
            CSC_CUDA(cudaMemcpyAsync(h->Z, h->tmpZ, sizeof(float) * nz, cudaMemcpyDeviceToDevice,
                                     s));
            CSC_CUDA(cudaMemcpyAsync(h->r, h->tmpB, sizeof(float) * nz, cudaMemcpyDeviceToDevice,
                                     s));
        }
        return CSC_OK;
    };
    const csc_opts saved = h->opts;
    const int L = h->L;
    int ncand = 0;
    double best_ms = 1e300, default_ms = -1.0;
    int best_w = 0, best_u = 0, best_c = 0;
    auto trial = [&](int w, int u, double *ms) -> int {
        h->opts.segments = 0;
        h->opts.segment_width = w;
        h->opts.updates_per_visit = u;
        h->plan_ok = false;
        csc_stats st;
        int rc = csc_solve(h, tol, max_updates, nullptr, nullptr, &st);
        if (rc < 0)
            return rc;
        ncand++;
        *ms = rc == CSC_OK ? st.solve_ms : 1e300;  // a candidate that did not converge loses
        if (*ms < best_ms) {
            best_ms = *ms;
            best_w = w;
            best_u = u;
            best_c = st.phases;
        }
        return restore();
    };
    // stage 1: segment width (and with it the number of phases) at the given u
    const int u0 = saved.updates_per_visit ? saved.updates_per_visit : 24;
    const int widths[] = {std::max(1, L - 1), std::max(1, 2 * L - 2), std::max(1, 3 * L - 3),
                          std::max(1, 4 * L - 4), std::max(1, 6 * L - 6)};
    int rc = CSC_OK;
    for (int i = 0; i < 5 && rc == CSC_OK; i++) {
        if (i > 0 && widths[i] == widths[i - 1])
            continue;
        double ms;
        rc = trial(widths[i], u0, &ms);
        if (rc == CSC_OK && widths[i] == std::max(1, 2 * L - 2))
            default_ms = ms;
    }
    // stage 2: updates per visit at the chosen width
    const int w1 = best_w;
    const int us[] = {8, 24, 64, 0};
    for (int i = 0; i < 4 && rc == CSC_OK; i++) {
        if (us[i] == u0)
            continue;
        double ms;
        rc = trial(w1, us[i], &ms);
    }
    // stage 3: threads per segment (one warp or a block) at that width and u
    int best_t = saved.threads_per_segment;
    if (rc == CSC_OK && phase_warp_eligible(h->K, h->L, 2 * std::max(best_w, 1))) {
        const int tps[] = {32, 128};
        const int t0 = saved.threads_per_segment ? saved.threads_per_segment
                                                 : kAutoThreadsPerSegment;
        best_t = t0;
        for (int i = 0; i < 2 && rc == CSC_OK; i++) {
            if (tps[i] == t0)
                continue;
            const double before = best_ms;
            double ms;
            h->opts.threads_per_segment = tps[i];
            rc = trial(best_w, best_u, &ms);
            h->opts.threads_per_segment = saved.threads_per_segment;
            if (best_ms < before)
                best_t = tps[i];
        }
    }
    if (rc != CSC_OK) {
        h->opts = saved;
        h->plan_ok = false;
        return rc;
    }
    h->opts = saved;
    h->opts.segments = 0;
    h->opts.segment_width = best_w;
    h->opts.updates_per_visit = best_u;
    h->opts.threads_per_segment = best_t;
    h->plan_ok = false;
    if (out) {
        out->segment_width = best_w;
        out->updates_per_visit = best_u;
        out->phases = best_c;
        out->candidates = ncand;
        out->best_ms = best_ms;
        out->default_ms = default_ms;
        out->threads_per_segment = best_t ? best_t : kAutoThreadsPerSegment;
    }
    return CSC_OK;
}

int csc_check_wait_timeout(int64_t polls)
{
    if (polls < 1 || polls > (int64_t)1 << 22)
        return fail(CSC_EINVAL, "csc_check_wait_timeout: polls must be in [1, 2^22]");
    int *d = nullptr;
    CSC_CUDA(cudaMalloc(&d, sizeof(int)));
    int gave_up = 0;
    cudaError_t e = cudaMemset(d, 0, sizeof(int));
    if (e == cudaSuccess)
        e = launch_wait_selftest((unsigned)polls, d, 0);
    if (e == cudaSuccess)
        e = cudaMemcpy(&gave_up, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess)
        return fail(CSC_ECUDA, "csc_check_wait_timeout: %s", cudaGetErrorString(e));
    if (gave_up)
        return fail(CSC_ETIMEOUT, "csc_check_wait_timeout: the bounded wait gave up after %lld polls",
                    (long long)polls);
    return CSC_OK;
}

int csc_init_time(csc_handle_t h, double *beta0_ms)
{
    if (!h || !beta0_ms)
        return fail(CSC_EINVAL, "csc_init_time: null argument");
    if (!h->initialized)
        return fail(CSC_ESTATE, "csc_init_time: call csc_init first");
    CSC_ON_DEVICE(h->device);
    if (int rc = finish_init(h))
        return rc;
    *beta0_ms = h->init_ms;
    return CSC_OK;
}

int csc_kernel_launches(csc_handle_t h, int64_t *out)
{
    if (!h || !out)
        return fail(CSC_EINVAL, "csc_kernel_launches: null argument");
    *out = h->launches;
    return CSC_OK;
}

int csc_get_beta(csc_handle_t h, float *beta_out)
{
    if (!h || !beta_out)
        return fail(CSC_EINVAL, "csc_get_beta: null argument");
    if (!h->initialized)
        return fail(CSC_ESTATE, "csc_get_beta: call csc_init first");
    CSC_ON_DEVICE(h->device);
    if (int rc = finish_init(h))
        return rc;
    const size_t nz = (size_t)h->K * h->Tz;
    // beta = r + ||D_k||^2 Z (the kernels keep r)
    if (is_device_pointer(beta_out)) {
        CSC_CUDA(launch_beta_from_r(h->r, h->Z, h->norms, h->K, h->Tz, beta_out, h->stream));
    } else {
        CSC_CUDA(grow(&h->tmpB, &h->cap_tmpB, nz));
        CSC_CUDA(launch_beta_from_r(h->r, h->Z, h->norms, h->K, h->Tz, h->tmpB, h->stream));
        CSC_CUDA(cudaMemcpyAsync(beta_out, h->tmpB, sizeof(float) * nz, cudaMemcpyDeviceToHost,
                                 h->stream));
    }
    h->launches += 1;
    CSC_CUDA(cudaStreamSynchronize(h->stream));
    return CSC_OK;
}

int csc_get_dtd(csc_handle_t h, float *dtd_out, float *norms_out)
{
    if (!h)
        return fail(CSC_EINVAL, "csc_get_dtd: null handle");
    CSC_ON_DEVICE(h->device);
    if (dtd_out)
        CSC_CUDA(copy_out(dtd_out, h->C, sizeof(float) * h->K * h->K * (2 * h->L - 1), h->stream));
    if (norms_out)
        CSC_CUDA(copy_out(norms_out, h->norms, sizeof(float) * h->K, h->stream));
    CSC_CUDA(cudaStreamSynchronize(h->stream));
    return CSC_OK;
}

int csc_objective(csc_handle_t h, const float *Z, double *out)
{
    csc::TraceRange trace_("csc_objective");
    if (!h || !Z || !out)
        return fail(CSC_EINVAL, "csc_objective: null argument");
    if (!h->initialized)
        return fail(CSC_ESTATE, "csc_objective: call csc_init first");
    CSC_ON_DEVICE(h->device);
    if (int rc = finish_init(h))
        return rc;
    cudaStream_t s = h->stream;
    const size_t nz = (size_t)h->K * h->Tz;
    const float *Zd = Z;
    if (!is_device_pointer(Z)) {
        CSC_CUDA(grow(&h->tmpZ, &h->cap_tmpZ, nz));
        CSC_CUDA(cudaMemcpyAsync(h->tmpZ, Z, sizeof(float) * nz, cudaMemcpyHostToDevice, s));
        Zd = h->tmpZ;
    }
    return objectives(h, Zd, out);
}

int csc_kkt(csc_handle_t h, const float *Z, double *out)
{
    csc::TraceRange trace_("csc_kkt");
    if (!h || !Z || !out)
        return fail(CSC_EINVAL, "csc_kkt: null argument");
    if (!h->initialized)
        return fail(CSC_ESTATE, "csc_kkt: call csc_init first");
    CSC_ON_DEVICE(h->device);
    if (int rc = finish_init(h))
        return rc;
    cudaStream_t s = h->stream;
    const size_t nz = (size_t)h->K * h->Tz;
    const float *Zd = Z;
    if (!is_device_pointer(Z)) {
        CSC_CUDA(grow(&h->tmpZ, &h->cap_tmpZ, nz));
        CSC_CUDA(cudaMemcpyAsync(h->tmpZ, Z, sizeof(float) * nz, cudaMemcpyHostToDevice, s));
        Zd = h->tmpZ;
    }
    // the problems' descriptors with Z moved to the caller's array (same
    // layout as the handle's Z); r is only read (write_r = 0), and no segment
    // flags or stored tile reports are used or changed
    std::vector<SigDesc> alt(h->sigs);
    for (SigDesc &d : alt)
        d.Z = const_cast<float *>(Zd) + (d.Z - h->Z);
    CSC_CUDA(upload(&h->d_sig_alt, &h->cap_sig_alt, alt, s));
    CSC_CUDA(cudaMemsetAsync(h->sc->red, 0, sizeof(h->sc->red), s));
    CSC_CUDA(launch_resync(h->d_sig_alt, h->resync_tiles(), h->Ct, h->norms, h->K, h->L, 0,
                           h->sc->red, 0, nullptr, 0.f, nullptr, nullptr, h->nz_lists(), s));
    h->launches += 2;
    unsigned long long red[8];
    CSC_CUDA(cudaMemcpyAsync(red, h->sc->red, sizeof red, cudaMemcpyDeviceToHost, s));
    CSC_CUDA(cudaStreamSynchronize(s));
    double v[5];
    std::memcpy(v, red, sizeof v);
    out[0] = v[1];
    out[1] = v[2];
    out[2] = v[3];
    return CSC_OK;
}

int csc_get_trace(csc_handle_t h, int64_t cap, int64_t *updates, double *decrease,
                  int64_t *t_ns, int64_t *n, double *E_start)
{
    if (!h || cap < 0 || (cap > 0 && (!updates || !decrease || !t_ns)))
        return fail(CSC_EINVAL, "csc_get_trace: bad arguments");
    CSC_ON_DEVICE(h->device);
    const int64_t g = h->g_used < kPhaseRing ? h->g_used : kPhaseRing;
    const int64_t m = cap < g ? cap : g;
    if (n)
        *n = h->g_used;
    if (E_start)
        *E_start = h->E_start;
    if (m == 0)
        return CSC_OK;
    unsigned long long t0 = 0;
    CSC_CUDA(cudaMemcpyAsync(updates, h->sc->upd, sizeof(long long) * m, cudaMemcpyDeviceToHost,
                             h->stream));
    CSC_CUDA(cudaMemcpyAsync(decrease, h->sc->dec, sizeof(double) * m, cudaMemcpyDeviceToHost,
                             h->stream));
    CSC_CUDA(cudaMemcpyAsync(t_ns, h->sc->tend, sizeof(int64_t) * m, cudaMemcpyDeviceToHost,
                             h->stream));
    CSC_CUDA(cudaMemcpyAsync(&t0, &h->sc->tstart, sizeof t0, cudaMemcpyDeviceToHost, h->stream));
    CSC_CUDA(cudaStreamSynchronize(h->stream));
    for (int64_t i = 0; i < m; i++)
        t_ns[i] = t_ns[i] ? (int64_t)((unsigned long long)t_ns[i] - t0) : -1;
    return CSC_OK;
}

}  // extern "C"
