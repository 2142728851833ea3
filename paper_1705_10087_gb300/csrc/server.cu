// Serving engine (include/csc_server.h): resident dictionaries, a device
// memory pool that bounds admission, and continuous batching of requests.
//
// Every dictionary is a group with its own stream and moves through these
// stages on its own: csc_server_step advances each group whose previous stage
// has completed (an event query, no waiting), so the groups' kernels overlap
// on the device and a slow dictionary never holds back a fast one:
//   1. admission: queued requests (per group, in submission order) get a pool
//      block while the pool has room; X is copied in, beta0 = D~ * X (the
//      same dtx kernel as csc_init) with lambda_max, r = beta0, Z = 0;
//   2. the group's plan is rebuilt when its active set changed: every request
//      cut into segments of the group's width, two phases;
//   3. S sweeps of phase launches over all active requests of the group, then
//      a per-request count of segments still needing a visit;
//   4. requests with no such segment ended a CD round: an exact resync of
//      their r (per-request reductions), accepted when max |Delta Z| < tol;
//   5. accepted (or out of resyncs) requests get their FP64 objective and are
//      retired from the active set; their pool block is released on fetch.
// A request only ever reads and writes its own pool block, and its schedule
// (segments, phases, S sweeps per round, resync points) does not depend on
// the others, so its result is the same bitwise alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "csc_internal.cuh"
#include "csc_server.h"
#include "host_util.cuh"
#include "pool.h"

int csc_record_error(int code, const char *fmt, ...);

using namespace csc;

namespace {

#define SRV_CUDA(expr)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return csc_record_error(e_ == cudaErrorMemoryAllocation ? CSC_ENOMEM : CSC_ECUDA,   \
                                    "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),     \
                                    __FILE__, __LINE__);                                        \
    } while (0)

#define SRV_TRY(expr)              \
    do {                           \
        int rc_ = (expr);          \
        if (rc_ != CSC_OK)         \
            return rc_;            \
    } while (0)

constexpr int kRed = 8;  // resync reduction slots per request
// threads per segment of the phase launches: a block (the faster form, see
// kAutoThreadsPerSegment in capi.cu)
constexpr int kServerThreadsPerSegment = 128;

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First bytes of a request's pool block.
struct ReqHeader {
    unsigned int lmax_bits;
    int tc_err;  // the tensor-core beta0 kernel gave up waiting
    double x2;
};

struct Request {
    int64_t id = 0;
    int dict = 0;
    int64_t T = 0, Tz = 0;
    double lam_spec = 0.0, tol = 0.0;
    int state = CSC_REQ_QUEUED;
    std::vector<float> Xh;  // until admitted
    size_t off = 0, bytes = 0;
    ReqHeader *hdr = nullptr;
    float *X = nullptr, *beta0 = nullptr, *r = nullptr, *Z = nullptr;
    double lam = 0.0, lmax = 0.0, E = 0.0, mdz = 0.0;
    int resyncs = 0, converged = 0;
    int64_t rounds = 0;
    int64_t sweeps = 0, sweeps_at_resync = 0;  // CD sweeps so far / at the last resync
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
};

// A request still not converged after this many CD sweeps is finished with
// converged = 0 (as csc_solve's max_sweeps).
constexpr int64_t kMaxRequestSweeps = 100000;

// Per-launch scratch of the phase kernel (one step's launches at most).
constexpr int kMaxLaunches = 4096;
struct PhaseScratch {
    long long upd[kMaxLaunches];
    double dec[kMaxLaunches];
    unsigned long long tend[kMaxLaunches];
    long long total;
    long long visits;
    int done;
    int qhead[2];  // drain launches: next queue entry, queue length
};

// Number of segments of problem i that still need a visit.
__global__ void count_dirty_kernel(const unsigned char *__restrict__ dirty,
                                   const SigDesc *__restrict__ sigs, int *__restrict__ cnt)
{
    const SigDesc sd = sigs[blockIdx.x];
    int c = 0;
    for (int j = threadIdx.x; j < sd.nseg; j += blockDim.x)
        c += dirty[sd.seg0 + j] != 0;
    for (int o = 16; o > 0; o >>= 1)
        c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ int ws[32];
    if ((threadIdx.x & 31) == 0)
        ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++)
            t += ws[w];
        cnt[blockIdx.x] = t;
    }
}

// What a group's stream is working on; the group moves to the next stage
// when the event recorded after that work has completed.
enum Stage { kIdle, kAdmitting, kSweeping, kResyncing, kFinishing };

struct Group {
    int K = 0, P = 0, L = 0, w = 0, u = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    Stage stage = kIdle;
    float *D = nullptr, *C = nullptr, *Ct = nullptr, *norms = nullptr;
    std::deque<int64_t> queue;    // submission order
    std::vector<int64_t> active;  // admission order; index = problem index of the plan
    bool stale = true;
    // plan of the active set
    std::vector<SigDesc> sigs;
    std::vector<int64_t> seg_s, seg_e;
    std::vector<int> seg_sig, list;
    int c = 2;                    // phases of the group's schedule
    std::vector<int> phase_off;   // [c+1] into the phase list
    int M = 0, w_max = 1;
    size_t held = 0;  // pool bytes of its admitted, not yet fetched requests
    SigDesc *d_sig = nullptr, *d_sub = nullptr;
    int64_t *d_seg_s = nullptr, *d_seg_e = nullptr;
    int *d_seg_sig = nullptr, *d_list = nullptr, *d_queue = nullptr;
    unsigned char *dirty = nullptr, *touched = nullptr;
    int *d_cnt = nullptr;
    unsigned long long *d_red = nullptr;
    double *d_E = nullptr, *d_partials = nullptr;
    int *d_tsig = nullptr;
    int64_t *d_tstart = nullptr, *d_toff = nullptr;
    int *d_nzc = nullptr;  // nonzero lists per resync tile (kernels_fp64.cu)
    uint2 *d_nze = nullptr;
    size_t cap_nzc = 0, cap_nze = 0;
    size_t cap_sig = 0, cap_sub = 0, cap_seg_s = 0, cap_seg_e = 0, cap_seg_sig = 0, cap_list = 0,
           cap_dirty = 0, cap_touched = 0, cap_cnt = 0, cap_red = 0, cap_E = 0, cap_partials = 0,
           cap_tsig = 0, cap_tstart = 0, cap_toff = 0, cap_queue = 0;
    PhaseScratch *ps = nullptr;
    // pinned host mirrors
    int *h_cnt = nullptr;
    unsigned long long *h_red = nullptr;
    double *h_E = nullptr;
    unsigned int *h_lmax = nullptr;
    size_t cap_h = 0;
    // host tile lists kept alive until their asynchronous upload completes
    std::vector<int> t_sig;
    std::vector<int64_t> t_start, t_off;
    std::vector<SigDesc> sub;
    // requests of the current round
    std::vector<int64_t> admitted, finished;
    std::vector<int> ended;    // problem indices resynced in this round
    std::vector<char> forced;  // per ended entry: the CD round had not settled
};

}  // namespace

struct csc_server_s {
    int device = 0;
    csc_server_opts opts{};
    Pool pool;
    std::vector<Group> groups;
    std::unordered_map<int64_t, Request> reqs;
    int64_t next_id = 1;
    std::deque<int64_t> completed;  // finished requests not yet reported by csc_server_completed
    int64_t launches = 0;
    double t0 = 0.0;
    cudaStream_t copy_st = nullptr;  // result copies
};

namespace {

int host_buffers(Group &g, size_t n)
{
    if (g.cap_h >= n && g.h_cnt)
        return CSC_OK;
    cudaFreeHost(g.h_cnt);
    cudaFreeHost(g.h_red);
    cudaFreeHost(g.h_E);
    cudaFreeHost(g.h_lmax);
    g.h_cnt = nullptr;
    g.h_red = nullptr;
    g.h_E = nullptr;
    g.h_lmax = nullptr;
    g.cap_h = 0;
    const size_t m = std::max<size_t>(n, 64);
    SRV_CUDA(cudaHostAlloc(&g.h_cnt, sizeof(int) * m, cudaHostAllocDefault));
    SRV_CUDA(cudaHostAlloc(&g.h_red, sizeof(unsigned long long) * kRed * m, cudaHostAllocDefault));
    SRV_CUDA(cudaHostAlloc(&g.h_E, sizeof(double) * m, cudaHostAllocDefault));
    SRV_CUDA(cudaHostAlloc(&g.h_lmax, 2 * sizeof(unsigned int) * m, cudaHostAllocDefault));
    g.cap_h = m;
    return CSC_OK;
}

size_t request_bytes(const Group &g, int64_t T)
{
    const int64_t Tz = T - g.L + 1;
    return align_up(sizeof(ReqHeader)) + align_up(sizeof(float) * g.P * T) +
           3 * align_up(sizeof(float) * g.K * Tz);
}

// Stage 1 for one group: admit queued requests while the pool has room.
// Fair share: while another dictionary has requests waiting, a group may hold
// at most pool / (number of groups), so a dictionary whose requests are slow
// to converge cannot take the whole pool from the others.
int admit(csc_server_t s, Group &g, double t)
{
    g.admitted.clear();
    bool others_waiting = false;
    for (const Group &o : s->groups)
        if (&o != &g && !o.queue.empty())
            others_waiting = true;
    const size_t share = s->pool.size / std::max<size_t>(1, s->groups.size());
    while (!g.queue.empty()) {
        if (s->opts.max_active > 0 && (int)g.active.size() >= s->opts.max_active)
            break;
        Request &q = s->reqs[g.queue.front()];
        if (others_waiting && g.held > 0 && g.held + align_up(q.bytes) > share)
            break;
        size_t off;
        if (!s->pool.alloc(q.bytes, &off))
            break;  // first come, first served: later requests wait behind it
        q.off = off;
        g.held += align_up(q.bytes);
        char *b = s->pool.base + off;
        q.hdr = reinterpret_cast<ReqHeader *>(b);
        b += align_up(sizeof(ReqHeader));
        q.X = reinterpret_cast<float *>(b);
        b += align_up(sizeof(float) * g.P * q.T);
        q.beta0 = reinterpret_cast<float *>(b);
        b += align_up(sizeof(float) * g.K * q.Tz);
        q.r = reinterpret_cast<float *>(b);
        b += align_up(sizeof(float) * g.K * q.Tz);
        q.Z = reinterpret_cast<float *>(b);
        const size_t nz = sizeof(float) * g.K * q.Tz;
        SRV_CUDA(cudaMemcpyAsync(q.X, q.Xh.data(), sizeof(float) * g.P * q.T,
                                 cudaMemcpyHostToDevice, g.st));
        SRV_CUDA(cudaMemsetAsync(q.hdr, 0, sizeof(ReqHeader), g.st));
        // Z = 0: r = beta0, written by the same kernel
        SRV_CUDA(launch_dtx_any(g.D, q.X, g.K, g.P, g.L, q.T, 0, q.beta0, q.r,
                                &q.hdr->lmax_bits, &q.hdr->x2, &q.hdr->tc_err, g.st));
        s->launches += 1;
        SRV_CUDA(cudaMemsetAsync(q.Z, 0, nz, g.st));
        q.state = CSC_REQ_ACTIVE;
        q.t_admit = t;
        g.queue.pop_front();
        g.active.push_back(q.id);
        g.admitted.push_back(q.id);
        g.stale = true;
    }
    if (g.admitted.empty())
        return CSC_OK;
    SRV_TRY(host_buffers(g, g.admitted.size()));
    for (size_t j = 0; j < g.admitted.size(); j++) {
        Request &q = s->reqs[g.admitted[j]];
        SRV_CUDA(cudaMemcpyAsync(&g.h_lmax[2 * j], &q.hdr->lmax_bits, 2 * sizeof(unsigned int),
                                 cudaMemcpyDeviceToHost, g.st));
    }
    return CSC_OK;
}

int finish_admit(csc_server_t s, Group &g)
{
    if (g.admitted.empty())
        return CSC_OK;
    for (size_t j = 0; j < g.admitted.size(); j++) {
        Request &q = s->reqs[g.admitted[j]];
        std::vector<float>().swap(q.Xh);  // the copy has completed
        if (g.h_lmax[2 * j + 1])
            return csc_record_error(CSC_ETIMEOUT,
                                    "csc_server_step: the tensor-core beta0 kernel gave up waiting");
        float v;
        std::memcpy(&v, &g.h_lmax[2 * j], sizeof v);
        q.lmax = v;
        q.lam = q.lam_spec > 0.0 ? q.lam_spec : -q.lam_spec * q.lmax;
        if (!(q.lam > 0.0))
            q.lam = 1.0;  // X gives D~ * X = 0: Z* = 0 for every positive lambda
    }
    return CSC_OK;
}

// Stage 2: segments of every active request and the phase lists: c phases,
// c = 1 + ceil((2L-2) / w) for segments of at least w columns (two for the
// default width 2L-2).
int rebuild(csc_server_t s, Group &g)
{
    if (!g.stale)
        return CSC_OK;
    g.stale = false;
    const int n = (int)g.active.size();
    g.sigs.assign(n, SigDesc{});
    g.seg_s.clear();
    g.seg_e.clear();
    g.seg_sig.clear();
    std::vector<int> local;
    const int max_resyncs = s->opts.max_resyncs < 0 ? 3 : s->opts.max_resyncs;
    for (int i = 0; i < n; i++) {
        const Request &q = s->reqs[g.active[i]];
        SigDesc &d = g.sigs[i];
        d.r = q.r;
        d.Z = q.Z;
        d.beta0 = q.beta0;
        d.X = q.X;
        d.ld = q.Tz;
        d.ldx = q.T;
        d.Tz = q.Tz;
        d.lam = (float)q.lam;
        d.lam_d = q.lam;
        d.tol = (float)(max_resyncs > 0 ? 0.5 * q.tol : q.tol);
        const int Mi = (int)std::max<int64_t>(1, q.Tz / g.w);
        d.seg0 = (int)g.seg_s.size();
        d.nseg = Mi;
        for (int m = 0; m < Mi; m++) {
            g.seg_s.push_back(seg_start(q.Tz, Mi, m));
            g.seg_e.push_back(seg_start(q.Tz, Mi, m + 1));
            g.seg_sig.push_back(i);
            local.push_back(m);
        }
    }
    g.M = (int)g.seg_s.size();
    g.w_max = 1;
    for (int m = 0; m < g.M; m++)
        g.w_max = std::max<int>(g.w_max, (int)(g.seg_e[m] - g.seg_s[m]));
    g.c = 1 + (int)((2 * (int64_t)g.L - 2 + g.w - 1) / g.w);
    g.list.clear();
    g.phase_off.assign(g.c + 1, 0);
    int most = 0;
    for (int p = 0; p < g.c; p++) {
        g.phase_off[p] = (int)g.list.size();
        for (int m = 0; m < g.M; m++)
            if (local[m] % g.c == p)
                g.list.push_back(m);
        most = std::max(most, (int)g.list.size() - g.phase_off[p]);
    }
    g.phase_off[g.c] = (int)g.list.size();
    if (n == 0)
        return CSC_OK;
    SRV_CUDA(upload(&g.d_sig, &g.cap_sig, g.sigs, g.st));
    SRV_CUDA(upload(&g.d_seg_s, &g.cap_seg_s, g.seg_s, g.st));
    SRV_CUDA(upload(&g.d_seg_e, &g.cap_seg_e, g.seg_e, g.st));
    SRV_CUDA(upload(&g.d_seg_sig, &g.cap_seg_sig, g.seg_sig, g.st));
    SRV_CUDA(upload(&g.d_list, &g.cap_list, g.list, g.st));
    SRV_CUDA(grow(&g.dirty, &g.cap_dirty, (size_t)g.M));
    SRV_CUDA(grow(&g.touched, &g.cap_touched, (size_t)g.M));
    SRV_CUDA(grow(&g.d_queue, &g.cap_queue, (size_t)std::max(most, 1)));
    SRV_CUDA(grow(&g.d_cnt, &g.cap_cnt, (size_t)n));
    SRV_CUDA(grow(&g.d_red, &g.cap_red, (size_t)n * kRed));
    SRV_CUDA(grow(&g.d_E, &g.cap_E, (size_t)n));
    // every segment gets a visit: clean ones find nothing and change nothing
    SRV_CUDA(cudaMemsetAsync(g.dirty, 1, (size_t)g.M, g.st));
    SRV_TRY(host_buffers(g, n));
    return CSC_OK;
}

// Stage 3: S sweeps of the c phases over the group's active requests.
int run_sweeps(csc_server_t s, Group &g)
{
    const int n = (int)g.active.size();
    if (n == 0)
        return CSC_OK;
    const int S = s->opts.sweeps_per_step > 0 ? s->opts.sweeps_per_step : 4;
    const int c = g.c;
    const PhaseConfig cfg = phase_config(g.K, g.L, g.w_max, kServerThreadsPerSegment);
    SRV_CUDA(cudaMemsetAsync(g.ps, 0, sizeof(PhaseScratch), g.st));
    PhaseParams pp{};
    pp.sig = g.d_sig;
    pp.seg_sig = g.d_seg_sig;
    pp.C = g.C;
    pp.Ct = g.Ct;
    pp.norms = g.norms;
    pp.dirty = g.dirty;
    pp.touched = g.touched;
    pp.seg_s = g.d_seg_s;
    pp.seg_e = g.d_seg_e;
    pp.upd = g.ps->upd;
    pp.dec = g.ps->dec;
    pp.tend = g.ps->tend;
    pp.total = &g.ps->total;
    pp.visits = &g.ps->visits;
    pp.done = &g.ps->done;
    pp.max_updates = (long long)1 << 62;
    pp.M = g.M;
    pp.c = c;
    pp.K = g.K;
    pp.Kp = coef_pad(g.K);
    pp.L = g.L;
    pp.u = g.u;
    pp.w_max = g.w_max;
    pp.g_round = 0;
    pp.qhead = g.ps->qhead;
    pp.qlen = g.ps->qhead + 1;
    pp.queue = g.d_queue;
    const int resident = phase_resident_blocks(cfg, g.K);
    int gi = 0;
    for (int i = 0; i < S; i++)
        for (int p = 0; p < c; p++) {
            pp.p = p;
            pp.g = gi++;
            pp.phase_list = g.d_list + g.phase_off[p];
            const int cnt = g.phase_off[p + 1] - g.phase_off[p];
            if (cnt > 4 * resident) {
                SRV_CUDA(launch_phase_drain(pp, cfg, cnt, resident, g.st));
                s->launches += 2;
            } else {
                SRV_CUDA(launch_phase(pp, cfg, cnt, g.st));
                s->launches += 1;
            }
        }
    count_dirty_kernel<<<n, 256, 0, g.st>>>(g.dirty, g.d_sig, g.d_cnt);
    SRV_CUDA(cudaGetLastError());
    s->launches += 1;
    SRV_CUDA(cudaMemcpyAsync(g.h_cnt, g.d_cnt, sizeof(int) * n, cudaMemcpyDeviceToHost, g.st));
    return CSC_OK;
}

// Stage 4: requests whose CD round ended get an exact resync.
int resync_ended(csc_server_t s, Group &g)
{
    g.ended.clear();
    g.forced.clear();
    const int n = (int)g.active.size();
    if (n == 0)
        return CSC_OK;
    g.t_sig.clear();
    g.t_start.clear();
    const int S = s->opts.sweeps_per_step > 0 ? s->opts.sweeps_per_step : 4;
    const int max_resyncs = s->opts.max_resyncs < 0 ? 3 : s->opts.max_resyncs;
    for (int i = 0; i < n; i++) {
        Request &q = s->reqs[g.active[i]];
        q.rounds++;
        q.sweeps += S;
        // a round still running after kDriftSweeps sweeps, or at the sweep cap,
        // is interrupted by a resync as in csc_solve
        const bool settled = g.h_cnt[i] == 0;
        const bool drift = max_resyncs > 0 && q.sweeps - q.sweeps_at_resync >= kDriftSweeps;
        const bool capped = q.sweeps >= kMaxRequestSweeps;
        if (!settled && !drift && !capped)
            continue;
        q.sweeps_at_resync = q.sweeps;
        g.ended.push_back(i);
        g.forced.push_back(settled ? 0 : 1);
        for (int64_t t = 0; t < q.Tz; t += kResyncCols) {
            g.t_sig.push_back(i);
            g.t_start.push_back(t);
        }
    }
    if (g.ended.empty())
        return CSC_OK;
    SRV_CUDA(upload(&g.d_tsig, &g.cap_tsig, g.t_sig, g.st));
    SRV_CUDA(upload(&g.d_tstart, &g.cap_tstart, g.t_start, g.st));
    SRV_CUDA(cudaMemsetAsync(g.d_red, 0, sizeof(unsigned long long) * kRed * n, g.st));
    const Tiles tiles{g.d_tsig, g.d_tstart, (int64_t)g.t_sig.size()};
    SRV_CUDA(grow(&g.d_nzc, &g.cap_nzc, g.t_sig.size()));
    SRV_CUDA(grow(&g.d_nze, &g.cap_nze, g.t_sig.size() * kNzCap));
    SRV_CUDA(launch_resync(g.d_sig, tiles, g.Ct, g.norms, g.K, g.L, 1, g.d_red, kRed, g.dirty,
                           -1.f, nullptr, nullptr, NzLists{g.d_nzc, g.d_nze}, g.st));
    count_dirty_kernel<<<n, 256, 0, g.st>>>(g.dirty, g.d_sig, g.d_cnt);
    SRV_CUDA(cudaGetLastError());
    s->launches += 3;  // bucket lists, resync, dirty count
    SRV_CUDA(cudaMemcpyAsync(g.h_red, g.d_red, sizeof(unsigned long long) * kRed * n,
                             cudaMemcpyDeviceToHost, g.st));
    return CSC_OK;
}

// Stage 5: decide, and compute the objective of the finished requests.
int objective_finished(csc_server_t s, Group &g)
{
    g.finished.clear();
    if (g.ended.empty())
        return CSC_OK;
    const int max_resyncs = s->opts.max_resyncs < 0 ? 3 : s->opts.max_resyncs;
    for (size_t e = 0; e < g.ended.size(); e++) {
        const int i = g.ended[e];
        Request &q = s->reqs[g.active[i]];
        double v[kRed];
        std::memcpy(v, &g.h_red[(size_t)i * kRed], sizeof v);
        const bool settled = !g.forced[e];
        const bool last = (settled && q.resyncs >= max_resyncs) || q.sweeps >= kMaxRequestSweeps;
        if (settled && q.resyncs < max_resyncs)
            q.resyncs++;
        q.mdz = v[3];
        if (v[4] < q.tol || last) {
            q.converged = v[4] < q.tol ? 1 : 0;
            g.finished.push_back(i);
        }
    }
    if (g.finished.empty())
        return CSC_OK;
    g.sub.clear();
    g.t_sig.clear();
    g.t_start.clear();
    g.t_off.clear();
    for (size_t j = 0; j < g.finished.size(); j++) {
        const int i = g.finished[j];
        g.sub.push_back(g.sigs[i]);
        g.t_off.push_back((int64_t)g.t_sig.size());
        const int64_t T = g.sigs[i].Tz + g.L - 1;
        for (int64_t t = 0; t < T; t += kTile) {
            g.t_sig.push_back((int)j);
            g.t_start.push_back(t);
        }
    }
    g.t_off.push_back((int64_t)g.t_sig.size());
    const int nf = (int)g.finished.size();
    SRV_CUDA(upload(&g.d_sub, &g.cap_sub, g.sub, g.st));
    SRV_CUDA(upload(&g.d_tsig, &g.cap_tsig, g.t_sig, g.st));
    SRV_CUDA(upload(&g.d_tstart, &g.cap_tstart, g.t_start, g.st));
    SRV_CUDA(upload(&g.d_toff, &g.cap_toff, g.t_off, g.st));
    SRV_CUDA(grow(&g.d_partials, &g.cap_partials, 2 * g.t_sig.size()));
    const Tiles tiles{g.d_tsig, g.d_tstart, (int64_t)g.t_sig.size()};
    SRV_CUDA(launch_objective(g.D, g.d_sub, nf, tiles, g.d_toff, g.K, g.P, g.L, nullptr, nullptr,
                              g.d_partials, g.d_E, g.st));
    s->launches += 2;
    SRV_CUDA(cudaMemcpyAsync(g.h_E, g.d_E, sizeof(double) * nf, cudaMemcpyDeviceToHost, g.st));
    return CSC_OK;
}

int retire(csc_server_t s, Group &g, double t, int *n_done)
{
    if (g.finished.empty())
        return CSC_OK;
    std::vector<char> gone(g.active.size(), 0);
    for (size_t j = 0; j < g.finished.size(); j++) {
        const int i = g.finished[j];
        Request &q = s->reqs[g.active[i]];
        q.E = g.h_E[j];
        q.state = CSC_REQ_DONE;
        q.t_done = t;
        s->completed.push_back(q.id);
        gone[i] = 1;
        (*n_done)++;
    }
    std::vector<int64_t> keep;
    for (size_t i = 0; i < g.active.size(); i++)
        if (!gone[i])
            keep.push_back(g.active[i]);
    g.active.swap(keep);
    g.stale = true;
    return CSC_OK;
}

void release_group(Group &g)
{
    void *bufs[] = {g.D,       g.C,       g.Ct,       g.norms,   g.d_sig,    g.d_sub,
                    g.d_seg_s, g.d_seg_e, g.d_seg_sig, g.d_list, g.dirty,    g.touched,
                    g.d_cnt,   g.d_red,   g.d_E,      g.d_partials, g.d_tsig, g.d_tstart,
                    g.d_toff,  g.ps,      g.d_queue,  g.d_nzc,   g.d_nze};
    for (void *p : bufs)
        cudaFree(p);
    cudaFreeHost(g.h_cnt);
    cudaFreeHost(g.h_red);
    cudaFreeHost(g.h_E);
    cudaFreeHost(g.h_lmax);
    if (g.ev)
        cudaEventDestroy(g.ev);
    if (g.st)
        cudaStreamDestroy(g.st);
}

// Advances one group through as many stages as have completed, issuing the
// next stage's work without waiting for it.  Returns CSC_OK; *moved is set
// when the group changed stage.
int advance(csc_server_t s, Group &g, int *n_done, bool *moved)
{
    for (;;) {
        if (g.stage != kIdle) {
            const cudaError_t q = cudaEventQuery(g.ev);
            if (q == cudaErrorNotReady)
                return CSC_OK;
            SRV_CUDA(q);
            *moved = true;
        }
        switch (g.stage) {
        case kIdle:
            SRV_TRY(admit(s, g, now_s() - s->t0));
            if (!g.admitted.empty()) {
                SRV_CUDA(cudaEventRecord(g.ev, g.st));
                g.stage = kAdmitting;
                *moved = true;
                continue;
            }
            if (g.active.empty())
                return CSC_OK;  // nothing to do
            *moved = true;
            SRV_TRY(rebuild(s, g));
            SRV_TRY(run_sweeps(s, g));
            SRV_CUDA(cudaEventRecord(g.ev, g.st));
            g.stage = kSweeping;
            return CSC_OK;
        case kAdmitting:
            SRV_TRY(finish_admit(s, g));
            SRV_TRY(rebuild(s, g));
            SRV_TRY(run_sweeps(s, g));
            SRV_CUDA(cudaEventRecord(g.ev, g.st));
            g.stage = kSweeping;
            return CSC_OK;
        case kSweeping:
            SRV_TRY(resync_ended(s, g));
            if (g.ended.empty()) {
                g.stage = kIdle;
                continue;
            }
            SRV_CUDA(cudaEventRecord(g.ev, g.st));
            g.stage = kResyncing;
            continue;
        case kResyncing:
            SRV_TRY(objective_finished(s, g));
            if (g.finished.empty()) {
                g.stage = kIdle;
                continue;
            }
            SRV_CUDA(cudaEventRecord(g.ev, g.st));
            g.stage = kFinishing;
            continue;
        case kFinishing:
            SRV_TRY(retire(s, g, now_s() - s->t0, n_done));
            g.stage = kIdle;
            continue;
        }
    }
}

}  // namespace

extern "C" {

int csc_server_create(csc_server_t *sp, const csc_server_opts *opts)
{
    if (!sp)
        return csc_record_error(CSC_EINVAL, "csc_server_create: null pointer");
    csc_server_opts o{};
    o.max_resyncs = -1;
    if (opts) {
        o = *opts;
        if (o.hbm_budget_bytes < 0 || o.sweeps_per_step < 0 || o.max_resyncs < -1 ||
            o.max_active < 0 || o.reserved[0] || o.reserved[1] || o.reserved[2])
            return csc_record_error(CSC_EINVAL, "csc_server_create: invalid options");
    }
    if (o.hbm_budget_bytes == 0)
        o.hbm_budget_bytes = (int64_t)40 << 30;
    if (o.sweeps_per_step * 2 > kMaxLaunches)
        return csc_record_error(CSC_EINVAL, "csc_server_create: sweeps_per_step above %d",
                                kMaxLaunches / 2);
    csc_server_t s = new (std::nothrow) csc_server_s();
    if (!s)
        return csc_record_error(CSC_ENOMEM, "csc_server_create: host allocation failed");
    s->opts = o;
    cudaGetDevice(&s->device);
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, (size_t)o.hbm_budget_bytes);
    if (e != cudaSuccess) {
        delete s;
        return csc_record_error(CSC_ENOMEM, "csc_server_create: pool of %lld bytes: %s",
                                (long long)o.hbm_budget_bytes, cudaGetErrorString(e));
    }
    s->pool.init(static_cast<char *>(base), (size_t)o.hbm_budget_bytes);
    e = cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(base);
        delete s;
        return csc_record_error(CSC_ECUDA, "csc_server_create: %s", cudaGetErrorString(e));
    }
    s->t0 = now_s();
    *sp = s;
    return CSC_OK;
}

int csc_server_add_dictionary(csc_server_t s, const float *D, int K, int P, int L,
                              int32_t segment_width, int32_t updates_per_visit, int *dict)
{
    csc::TraceRange trace_("csc_server_add_dictionary");
    if (!s || !D || !dict)
        return csc_record_error(CSC_EINVAL, "csc_server_add_dictionary: null argument");
    if (K < 1 || K > 256 || P < 1 || L < 1 || L > kMaxL)
        return csc_record_error(CSC_EINVAL, "csc_server_add_dictionary: bad sizes %d,%d,%d", K,
                                P, L);
    const int wmin = std::max(1, 2 * L - 2);
    if (segment_width < 0)
        return csc_record_error(CSC_EINVAL, "csc_server_add_dictionary: segment_width < 0");
    {
        // launches of one scheduling step (S sweeps of c phases) index the
        // group's per-launch counters
        const int w = segment_width ? segment_width : wmin;
        const int S = s->opts.sweeps_per_step > 0 ? s->opts.sweeps_per_step : 4;
        const int64_t c = 1 + (2 * (int64_t)L - 2 + w - 1) / w;
        if (S * c > kMaxLaunches)
            return csc_record_error(CSC_EINVAL,
                                    "csc_server_add_dictionary: %lld phases x %d sweeps per step "
                                    "exceed %d launches",
                                    (long long)c, S, kMaxLaunches);
    }
    if (updates_per_visit < 0)
        return csc_record_error(CSC_EINVAL, "csc_server_add_dictionary: updates_per_visit < 0");
    csc::DeviceGuard dev_guard_(s->device);
    if (dev_guard_.err != cudaSuccess)
        return csc_record_error(CSC_ECUDA, "cudaSetDevice(%d) failed: %s", s->device,
                                cudaGetErrorString(dev_guard_.err));
    s->groups.emplace_back();
    Group &g = s->groups.back();
    g.K = K;
    g.P = P;
    g.L = L;
    g.w = segment_width ? segment_width : wmin;
    g.u = updates_per_visit ? updates_per_visit : 24;
    auto body = [&]() -> int {
        SRV_CUDA(cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking));
        SRV_CUDA(cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming));
        size_t cap = 0;
        SRV_CUDA(grow(&g.D, &cap, (size_t)K * P * L));
        cap = 0;
        SRV_CUDA(grow(&g.C, &cap, (size_t)K * K * (2 * L - 1)));
        cap = 0;
        SRV_CUDA(grow(&g.Ct, &cap, (size_t)K * (2 * L - 1) * coef_pad(K)));
        cap = 0;
        SRV_CUDA(grow(&g.norms, &cap, (size_t)K));
        SRV_CUDA(cudaMalloc(&g.ps, sizeof(PhaseScratch)));
        SRV_CUDA(copy_in(g.D, D, sizeof(float) * K * P * L, g.st));
        SRV_CUDA(launch_dtd(g.D, K, P, L, g.C, g.norms, g.st));
        SRV_CUDA(launch_coef_by_lag(g.C, K, L, g.Ct, g.st));
        s->launches += 2;
        SRV_CUDA(cudaStreamSynchronize(g.st));
        return CSC_OK;
    };
    int rc = body();
    if (rc != CSC_OK) {
        release_group(g);
        s->groups.pop_back();
        return rc;
    }
    *dict = (int)s->groups.size() - 1;
    return CSC_OK;
}

int csc_server_submit(csc_server_t s, int dict, const float *X, int64_t T, double lambda,
                      double tol, int64_t *request)
{
    csc::TraceRange trace_("csc_server_submit");
    if (!s || !X || !request)
        return csc_record_error(CSC_EINVAL, "csc_server_submit: null argument");
    if (dict < 0 || dict >= (int)s->groups.size())
        return csc_record_error(CSC_EINVAL, "csc_server_submit: no dictionary %d", dict);
    Group &g = s->groups[dict];
    if (T < g.L || T - g.L + 1 >= ((int64_t)1 << 31) - 1)
        return csc_record_error(CSC_EINVAL, "csc_server_submit: need L <= T < 2^31 + L - 2");
    if (!(lambda != 0.0) || !std::isfinite(lambda) || !(tol > 0.0))
        return csc_record_error(CSC_EINVAL, "csc_server_submit: need lambda != 0 and tol > 0");
    Request q;
    q.id = s->next_id++;
    q.dict = dict;
    q.T = T;
    q.Tz = T - g.L + 1;
    q.lam_spec = lambda;
    q.tol = tol;
    q.bytes = request_bytes(g, T);
    if (align_up(q.bytes) > s->pool.size)
        return csc_record_error(CSC_ENOMEM,
                                "csc_server_submit: the request needs %zu bytes, more than the "
                                "whole pool (%zu)",
                                q.bytes, s->pool.size);
    q.Xh.resize((size_t)g.P * T);
    csc::DeviceGuard dev_guard_(s->device);
    if (dev_guard_.err != cudaSuccess)
        return csc_record_error(CSC_ECUDA, "cudaSetDevice(%d) failed: %s", s->device,
                                cudaGetErrorString(dev_guard_.err));
    if (is_device_pointer(X)) {
        SRV_CUDA(cudaMemcpy(q.Xh.data(), X, sizeof(float) * g.P * T, cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(q.Xh.data(), X, sizeof(float) * g.P * T);
    }
    q.t_submit = now_s() - s->t0;
    const int64_t id = q.id;
    s->reqs.emplace(id, std::move(q));
    g.queue.push_back(id);
    *request = id;
    return CSC_OK;
}

int csc_server_step(csc_server_t s, int *n_active, int *n_queued, int *n_done)
{
    csc::TraceRange trace_("csc_server_step");
    if (!s)
        return csc_record_error(CSC_EINVAL, "csc_server_step: null server");
    csc::DeviceGuard dev_guard_(s->device);
    if (dev_guard_.err != cudaSuccess)
        return csc_record_error(CSC_ECUDA, "cudaSetDevice(%d) failed: %s", s->device,
                                cudaGetErrorString(dev_guard_.err));
    int done = 0;
    // every group advances on its own: a dictionary whose rounds are slow does
    // not hold back the others; if no group could move, wait for the first
    // busy one and try again
    for (int attempt = 0; attempt < 2; attempt++) {
        bool moved = false;
        for (Group &g : s->groups)
            SRV_TRY(advance(s, g, &done, &moved));
        if (moved)
            break;
        Group *busy = nullptr;
        for (Group &g : s->groups)
            if (g.stage != kIdle) {
                busy = &g;
                break;
            }
        if (!busy)
            break;
        SRV_CUDA(cudaEventSynchronize(busy->ev));
    }
    int na = 0, nq = 0;
    for (const Group &g : s->groups) {
        na += (int)g.active.size();
        nq += (int)g.queue.size();
    }
    if (n_active)
        *n_active = na;
    if (n_queued)
        *n_queued = nq;
    if (n_done)
        *n_done = done;
    return CSC_OK;
}

int csc_server_completed(csc_server_t s, int64_t *requests, int cap, int *n)
{
    if (!s || !n || cap < 0 || (cap > 0 && !requests))
        return csc_record_error(CSC_EINVAL, "csc_server_completed: bad arguments");
    int k = 0;
    while (k < cap && !s->completed.empty()) {
        requests[k++] = s->completed.front();
        s->completed.pop_front();
    }
    *n = k;
    return CSC_OK;
}

int csc_server_info(csc_server_t s, int64_t request, csc_request_info *info)
{
    if (!s || !info)
        return csc_record_error(CSC_EINVAL, "csc_server_info: null argument");
    auto it = s->reqs.find(request);
    if (it == s->reqs.end())
        return csc_record_error(CSC_EINVAL, "csc_server_info: no request %lld", (long long)request);
    const Request &q = it->second;
    std::memset(info, 0, sizeof *info);
    info->state = q.state;
    info->dict = q.dict;
    info->T = q.T;
    info->lambda = q.lam;
    info->lambda_max = q.lmax;
    info->objective = q.E;
    info->max_delta_z = q.mdz;
    info->resyncs = q.resyncs;
    info->converged = q.converged;
    info->rounds = q.rounds;
    info->device_bytes = q.state == CSC_REQ_QUEUED ? 0 : (int64_t)align_up(q.bytes);
    info->t_submit = q.t_submit;
    info->t_admit = q.t_admit;
    info->t_done = q.t_done;
    return CSC_OK;
}

int csc_server_fetch(csc_server_t s, int64_t request, float *Z_out, csc_request_info *info)
{
    csc::TraceRange trace_("csc_server_fetch");
    if (!s)
        return csc_record_error(CSC_EINVAL, "csc_server_fetch: null server");
    auto it = s->reqs.find(request);
    if (it == s->reqs.end())
        return csc_record_error(CSC_EINVAL, "csc_server_fetch: no request %lld",
                                (long long)request);
    Request &q = it->second;
    if (q.state != CSC_REQ_DONE)
        return csc_record_error(CSC_ESTATE, "csc_server_fetch: request %lld is not done",
                                (long long)request);
    csc::DeviceGuard dev_guard_(s->device);
    if (dev_guard_.err != cudaSuccess)
        return csc_record_error(CSC_ECUDA, "cudaSetDevice(%d) failed: %s", s->device,
                                cudaGetErrorString(dev_guard_.err));
    const Group &g = s->groups[q.dict];
    // the request left its group's active set in a completed round, so no
    // kernel in flight touches its block: copy on the server's own stream,
    // without waiting for the group's running work
    if (Z_out) {
        SRV_CUDA(copy_out(Z_out, q.Z, sizeof(float) * g.K * q.Tz, s->copy_st));
        SRV_CUDA(cudaStreamSynchronize(s->copy_st));
    }
    if (info)
        SRV_TRY(csc_server_info(s, request, info));
    if (info)
        info->device_bytes = 0;
    s->pool.release(q.off, q.bytes);
    s->groups[q.dict].held -= align_up(q.bytes);
    s->reqs.erase(it);
    return CSC_OK;
}

int csc_server_memory(csc_server_t s, int64_t *pool_bytes, int64_t *in_use, int64_t *peak)
{
    if (!s)
        return csc_record_error(CSC_EINVAL, "csc_server_memory: null server");
    if (pool_bytes)
        *pool_bytes = (int64_t)s->pool.size;
    if (in_use)
        *in_use = (int64_t)s->pool.in_use;
    if (peak)
        *peak = (int64_t)s->pool.peak;
    return CSC_OK;
}

int csc_server_kernel_launches(csc_server_t s, int64_t *out)
{
    if (!s || !out)
        return csc_record_error(CSC_EINVAL, "csc_server_kernel_launches: null argument");
    *out = s->launches;
    return CSC_OK;
}

int csc_server_destroy(csc_server_t s)
{
    if (!s)
        return CSC_OK;
    csc::DeviceGuard dev_guard_(s->device);
    if (dev_guard_.err != cudaSuccess)
        return csc_record_error(CSC_ECUDA, "cudaSetDevice(%d) failed: %s", s->device,
                                cudaGetErrorString(dev_guard_.err));
    for (Group &g : s->groups) {
        if (g.st)
            cudaStreamSynchronize(g.st);
        release_group(g);
    }
    if (s->copy_st) {
        cudaStreamSynchronize(s->copy_st);
        cudaStreamDestroy(s->copy_st);
    }
    cudaFree(s->pool.base);
    delete s;
    return CSC_OK;
}

}  // extern "C"
