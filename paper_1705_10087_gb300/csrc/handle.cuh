// The solver handle (struct csc_handle_s of include/csc.h) and its small
// device-side state, shared by the translation units that implement the C
// ABI on a handle (capi.cu: single signals and batches; shard.cu: one shard
// of a signal cut across processes).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstddef>
#include <cstring>
#include <vector>

#include "csc_internal.cuh"
#include "host_util.cuh"

namespace csc {

// Small device-side state of a handle (one allocation).
struct Scratch {
    long long upd[kPhaseRing];
    double dec[kPhaseRing];
    unsigned long long tend[kPhaseRing];
    // polled after a CD round (Poll mirrors total .. gctr[0]); zeroed at the
    // start of a solve up to red (solve_begin)
    long long total;
    int done;
    int gctr[2];   // graph replays: launch index of the next launch, first index of the round
    int pad;
    long long visits;
    unsigned long long red[8];
    double x2;  // sum X^2 of the last csc_init
    // (the end of a solve reads total .. x2 back in one copy: Fin)
    unsigned int lmax_bits;
    int tc_err;  // a bounded wait of the tensor-core beta0 kernel gave up
    unsigned long long tstart;
    double obj[2];
    int qhead[2];  // drain launches: next queue entry, queue length
    long long round_lim[4];  // stopping rules of a CD round run as a graph (launch_round_step)
};

// Host mirror of what the solve loop polls (pinned): Scratch::total .. gctr[0].
struct Poll {
    long long total;
    int done;
    int g_next;  // launch index after a CD round run as a graph (Scratch::gctr[0])
};

// What the end of a solve reads back, in one pinned block and one copy:
// Scratch::total .. x2.
struct Fin {
    long long total;
    int done;
    int gctr[2];
    int pad;
    long long visits;
    unsigned long long red[8];
    double x2;
};

#define CSC_MIRRORS(S, f)                                                               \
    static_assert(offsetof(S, f) == offsetof(Scratch, f) - offsetof(Scratch, total), \
                  #S " mirrors Scratch")
CSC_MIRRORS(Poll, total);
CSC_MIRRORS(Poll, done);
static_assert(offsetof(Poll, g_next) == offsetof(Scratch, gctr) - offsetof(Scratch, total),
              "Poll mirrors Scratch");
CSC_MIRRORS(Fin, done);
CSC_MIRRORS(Fin, gctr);
CSC_MIRRORS(Fin, visits);
CSC_MIRRORS(Fin, red);
CSC_MIRRORS(Fin, x2);
static_assert(sizeof(Fin) == offsetof(Scratch, lmax_bits) - offsetof(Scratch, total),
              "Fin mirrors Scratch");
#undef CSC_MIRRORS

// The host-side segment plan of one shard (shard.cu); empty for ordinary handles.
struct ShardState {
    bool on = false;
    int64_t Tz_global = 0, T_global = 0;
    int M_global = 0, seg_first = 0, seg_count = 0;
    int64_t col_first = 0, col_count = 0;  // owned global columns
    int64_t hl = 0, hr = 0;                // halo columns held left / right
    bool last = false;                     // owns the end of the signal (samples [Tz, T))
    int64_t g = 0;                         // phase launches so far (trace slots)
    // tiles over the owned columns (resync) and the owned samples (objective)
    int *d_rt_sig = nullptr, *d_ot_sig = nullptr;
    int64_t *d_rt_s = nullptr, *d_rt_e = nullptr, *d_ot_s = nullptr, *d_ot_e = nullptr,
            *d_ot_off = nullptr;
    size_t cap_rt_sig = 0, cap_ot_sig = 0, cap_rt_s = 0, cap_rt_e = 0, cap_ot_s = 0,
           cap_ot_e = 0, cap_ot_off = 0;
    int64_t n_rt = 0, n_ot = 0;
    float *stage = nullptr;  // device staging of host halo buffers
    size_t cap_stage = 0;
};

}  // namespace csc

using csc::NzLists;
using csc::Fin;
using csc::Poll;
using csc::Scratch;
using csc::SigDesc;
using csc::Tiles;

struct csc_handle_s {
    csc::ShardState shard;
    int device = 0;
    cudaStream_t stream = nullptr;
    csc_opts opts{};
    int K = 0, P = 0, L = 0;
    float *D = nullptr, *C = nullptr, *Ct = nullptr, *norms = nullptr;
    size_t cap_D = 0, cap_C = 0, cap_Ct = 0, cap_n = 0;

    // problem: n signals concatenated in time, T samples, Tz = T - L + 1 columns
    bool initialized = false;
    int64_t T = 0, Tz = 0;
    int n = 0;
    std::vector<int64_t> a;         // [n+1] sample starts
    std::vector<double> lam;        // [n]
    std::vector<double> lmax;       // [n]
    std::vector<double> E_sig;      // [n] objectives of the last solve / csc_objective
    std::vector<SigDesc> sigs;      // [n] descriptors of the signals
    std::vector<SigDesc> sigs_dev;  // what d_sig holds (see push_sigs)
    SigDesc *d_sig = nullptr;
    size_t cap_sig = 0;
    SigDesc *d_sig_alt = nullptr;   // [n] the same over a caller's Z (csc_kkt)
    size_t cap_sig_alt = 0;
    // objective / absmax tiles (kTile samples) and resync tiles (kResyncCols columns)
    std::vector<int64_t> tile_off;  // [n+1] first objective tile of each signal
    int64_t ntiles = 0, nrtiles = 0;
    int64_t *d_tile_s = nullptr, *d_tile_off = nullptr, *d_rtile_s = nullptr, *d_rtile_off = nullptr;
    int64_t *d_sig_a = nullptr;  // [n+1] first sample of each problem (a)
    size_t cap_sig_a = 0;
    int *d_tile_sig = nullptr, *d_rtile_sig = nullptr;
    size_t cap_rtile_s = 0, cap_rtile_sig = 0, cap_rtile_off = 0;
    double *d_E = nullptr;
    unsigned int *d_lmax = nullptr;
    size_t cap_tile_s = 0, cap_tile_off = 0, cap_tile_sig = 0, cap_E = 0, cap_lmax = 0;

    // r = beta - ||D_k||^2 Z, the form of beta the kernels keep (csc_internal.cuh)
    float *X = nullptr, *r = nullptr, *beta0 = nullptr, *Z = nullptr;
    size_t cap_X = 0, cap_r = 0, cap_beta0 = 0, cap_Z = 0;
    double *partials = nullptr;
    size_t cap_partials = 0;

    // segment plan (rebuilt when the signals, lambdas or segment options change)
    bool plan_ok = false;
    // what the current plan and tile tables were built for (re-used when a
    // csc_setup / csc_init repeats the same signal lengths and options)
    std::vector<int64_t> plan_a, tiles_a;
    int plan_L = -1, plan_segments = -1, plan_width = -1, tiles_L = -1;
    std::vector<int> plan_seg0, plan_nseg;
    int M = 0, c = 0, w_max = 0;
    std::vector<int> phase_off;  // [c+1] into the phase list
    int64_t *d_seg_s = nullptr, *d_seg_e = nullptr;
    int *d_seg_sig = nullptr;
    int *d_phase_list = nullptr;
    size_t cap_seg_s = 0, cap_seg_e = 0, cap_seg_sig = 0, cap_phase = 0;
    unsigned char *dirty = nullptr, *touched = nullptr;
    size_t cap_dirty = 0, cap_touched = 0;
    int *d_queue = nullptr;  // drain launches: the phase's segments to visit
    size_t cap_queue = 0;
    // the poll batch (S sweeps of c phases) captured as a CUDA graph, and what
    // it was captured for
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> gkey, gkey_seen;
    cudaStream_t cap_stream = nullptr;  // captures happen here (not on a legacy stream)
    float *tile_rep = nullptr;  // stored resync report per resync tile
    size_t cap_tile_rep = 0;
    int *nz_count = nullptr;  // nonzeros of Z per resync tile (bucket lists)
    uint2 *nz_ent = nullptr;
    size_t cap_nz_count = 0, cap_nz_ent = 0;

    float *tmpZ = nullptr, *tmpB = nullptr;
    size_t cap_tmpZ = 0, cap_tmpB = 0;
    Scratch *sc = nullptr;
    Poll *poll = nullptr;  // pinned
    Fin *fin = nullptr;    // pinned
    double *E_pin = nullptr;  // pinned, [n] objectives of the last solve
    size_t cap_E_pin = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t ev_i0 = nullptr, ev_i1 = nullptr;  // around the beta0 kernel (time_kernels)
    cudaEvent_t ev_r0 = nullptr, ev_r1 = nullptr;  // around a resync / the objective
    double init_ms = -1.0;
    // csc_init's results, copied back without waiting: init_pin[0] = the
    // tensor-core kernel's give-up flag, init_pin[1 + i] = max |beta0| bits of
    // signal i (pinned; complete once ev_init has completed)
    unsigned *init_pin = nullptr;
    size_t cap_init_pin = 0;
    cudaEvent_t ev_init = nullptr;
    cudaEvent_t ev_copy = nullptr;  // after csc_init's copies of the caller's arrays
    bool init_pending = false;
    cudaEvent_t *kev = nullptr;  // per-launch timing events (2 per launch of a poll batch)
    int n_kev = 0;
    int64_t launches = 0;        // kernels launched through this handle
    bool z_is_zero = false;      // Z == 0 since csc_init: E(Z) = sum X^2 / 2 is known
    // last solve
    int64_t g_used = 0;
    double E_start = 0.0;

    Tiles obj_tiles() const { return Tiles{d_tile_sig, d_tile_s, ntiles}; }
    NzLists nz_lists() const { return NzLists{nz_count, nz_ent}; }
    Tiles resync_tiles() const { return Tiles{d_rtile_sig, d_rtile_s, nrtiles}; }
};

// Completes csc_init's asynchronous read-back (capi.cu): lambda_max per
// signal, the beta0 kernel's time and its give-up flag; CSC_ETIMEOUT if the
// tensor-core kernel gave up.  Every call that reads them calls it first.
int finish_init(csc_handle_s *h);

// d_sig <- h->sigs, skipped when the device copy already holds exactly these
// descriptors: a copy from pageable memory waits for the stream, and repeated
// solves of the same signals would otherwise stall the queue at every call.
static_assert(sizeof(csc::SigDesc) == 80, "SigDesc has no padding (compared bytewise)");
inline cudaError_t push_sigs(csc_handle_s *h, cudaStream_t s)
{
    if (h->d_sig && h->sigs_dev.size() == h->sigs.size() &&
        std::memcmp(h->sigs_dev.data(), h->sigs.data(), sizeof(csc::SigDesc) * h->sigs.size()) == 0)
        return cudaSuccess;
    const cudaError_t e = csc::upload(&h->d_sig, &h->cap_sig, h->sigs, s);
    if (e == cudaSuccess)
        h->sigs_dev = h->sigs;
    else
        h->sigs_dev.clear();
    return e;
}
