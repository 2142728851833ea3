/*
 * A plain C99 caller of the library's C ABI (include/csc.h and
 * include/csc_server.h): it must compile as C with every warning an error,
 * link against libcsc.so and, without a GPU, get the documented results of
 * the host-only entry points and of argument validation.  Exit status 0 on
 * success; the first failed check is printed.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "csc.h"
#include "csc2d.h"
#include "csc_server.h"
#include "csc_shard.h"

#define CHECK(c)                                                  \
    do {                                                          \
        if (!(c)) {                                               \
            printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #c);   \
            return 1;                                             \
        }                                                         \
    } while (0)

/* "layout": one line per struct, its size then the offset of every field in
 * declaration order, for the binding's ctypes mirrors to be compared with */
#define OFF(T, f) (unsigned)offsetof(T, f)
static void print_layouts(void)
{
    printf("csc_opts %u %u %u %u %u %u %u %u %u %u %u\n", (unsigned)sizeof(csc_opts),
           OFF(csc_opts, segments), OFF(csc_opts, updates_per_visit),
           OFF(csc_opts, max_resyncs), OFF(csc_opts, sweeps_per_poll),
           OFF(csc_opts, max_sweeps), OFF(csc_opts, time_kernels),
           OFF(csc_opts, segment_width), OFF(csc_opts, init_mode), OFF(csc_opts, launch_mode),
           OFF(csc_opts, threads_per_segment));
    printf("csc_stats %u %u %u %u %u %u %u %u %u %u %u %u %u %u %u %u %u %u %u %u\n",
           (unsigned)sizeof(csc_stats), OFF(csc_stats, updates), OFF(csc_stats, sweeps),
           OFF(csc_stats, segments), OFF(csc_stats, phases), OFF(csc_stats, resyncs),
           OFF(csc_stats, converged), OFF(csc_stats, objective), OFF(csc_stats, max_drift),
           OFF(csc_stats, kkt_zero_excess), OFF(csc_stats, kkt_nonzero_gap),
           OFF(csc_stats, max_delta_z), OFF(csc_stats, solve_ms), OFF(csc_stats, phase_ms),
           OFF(csc_stats, phase_launches), OFF(csc_stats, visits),
           OFF(csc_stats, kernel_launches), OFF(csc_stats, drift_resyncs),
           OFF(csc_stats, resync_ms), OFF(csc_stats, objective_ms));
    printf("csc_shard_plan %u %u %u %u %u %u %u %u %u %u %u %u %u %u %u %u\n",
           (unsigned)sizeof(csc_shard_plan), OFF(csc_shard_plan, T), OFF(csc_shard_plan, Tz),
           OFF(csc_shard_plan, L), OFF(csc_shard_plan, M), OFF(csc_shard_plan, phases),
           OFF(csc_shard_plan, world), OFF(csc_shard_plan, rank), OFF(csc_shard_plan, seg_first),
           OFF(csc_shard_plan, seg_count), OFF(csc_shard_plan, col_first),
           OFF(csc_shard_plan, col_count), OFF(csc_shard_plan, halo_left),
           OFF(csc_shard_plan, halo_right), OFF(csc_shard_plan, x_first),
           OFF(csc_shard_plan, x_count));
    printf("csc2d_stats %u %u %u %u %u %u %u %u %u %u %u %u %u\n", (unsigned)sizeof(csc2d_stats),
           OFF(csc2d_stats, updates), OFF(csc2d_stats, sweeps), OFF(csc2d_stats, bands),
           OFF(csc2d_stats, col_blocks), OFF(csc2d_stats, phases), OFF(csc2d_stats, resyncs),
           OFF(csc2d_stats, converged), OFF(csc2d_stats, reserved), OFF(csc2d_stats, objective),
           OFF(csc2d_stats, max_delta_z), OFF(csc2d_stats, solve_ms),
           OFF(csc2d_stats, kernel_launches));
    printf("csc_tune_result %u %u %u %u %u %u %u %u\n", (unsigned)sizeof(csc_tune_result),
           OFF(csc_tune_result, segment_width), OFF(csc_tune_result, updates_per_visit),
           OFF(csc_tune_result, phases), OFF(csc_tune_result, candidates),
           OFF(csc_tune_result, best_ms), OFF(csc_tune_result, default_ms),
           OFF(csc_tune_result, threads_per_segment));
    printf("csc_server_opts %u %u %u %u %u %u\n", (unsigned)sizeof(csc_server_opts),
           OFF(csc_server_opts, hbm_budget_bytes), OFF(csc_server_opts, sweeps_per_step),
           OFF(csc_server_opts, max_resyncs), OFF(csc_server_opts, max_active),
           OFF(csc_server_opts, reserved));
    printf("csc_request_info %u %u %u %u %u %u %u %u %u %u %u %u %u %u %u\n",
           (unsigned)sizeof(csc_request_info), OFF(csc_request_info, state),
           OFF(csc_request_info, dict), OFF(csc_request_info, T), OFF(csc_request_info, lambda),
           OFF(csc_request_info, lambda_max), OFF(csc_request_info, objective),
           OFF(csc_request_info, max_delta_z), OFF(csc_request_info, resyncs),
           OFF(csc_request_info, converged), OFF(csc_request_info, rounds),
           OFF(csc_request_info, device_bytes), OFF(csc_request_info, t_submit),
           OFF(csc_request_info, t_admit), OFF(csc_request_info, t_done));
}

int main(int argc, char **argv)
{
    csc_opts o;
    csc_handle_t h = NULL;
    csc_server_t srv = NULL;
    int M = 0, c = 0, k;
    int64_t starts[11];
    float D[2 * 1 * 4];
    double out[3];

    if (argc > 1 && strcmp(argv[1], "layout") == 0) {
        print_layouts();
        return 0;
    }
    memset(&o, 0x7f, sizeof o);
    csc_default_opts(&o);
    CHECK(o.segments == 0 && o.updates_per_visit == 0 && o.max_resyncs == -1);
    CHECK(o.threads_per_segment == 0);

    /* Sec. 2.2 segments: [floor(m*Tz/M), floor((m+1)*Tz/M)) */
    CHECK(csc_plan(1985, 16, 10, &M, &c, starts) == CSC_OK);
    CHECK(M == 10 && c == 2);
    for (k = 0; k <= 10; k++)
        CHECK(starts[k] == (int64_t)k * 1985 / 10);
    CHECK(csc_plan(10, 3, 11, &M, &c, NULL) == CSC_EINVAL);
    CHECK(strstr(csc_last_error_string(), "csc_plan") != NULL);

    /* argument validation happens before any device work */
    memset(D, 0, sizeof D);
    CHECK(csc_setup(&h, D, 0, 1, 4, NULL, NULL) == CSC_EINVAL);
    CHECK(csc_setup(&h, NULL, 2, 1, 4, NULL, NULL) == CSC_EINVAL);
    CHECK(csc_init(NULL, D, 10, 1.0, NULL) == CSC_EINVAL);
    CHECK(csc_solve(NULL, 1e-6, 10, NULL, NULL, NULL) == CSC_EINVAL);
    CHECK(csc_kkt(NULL, D, out) == CSC_EINVAL);
    CHECK(csc_check_wait_timeout(0) == CSC_EINVAL);
    CHECK(csc_destroy(NULL) == CSC_OK);
    CHECK(csc_server_step(srv, NULL, NULL, NULL) == CSC_EINVAL);
    CHECK(csc_server_destroy(NULL) == CSC_OK);

    /* host-only plans of the sharded and the 2-D solves */
    {
        csc_shard_plan sp;
        CHECK(csc_shard_plan_make(2000, 16, 10, 2, 1, &sp) == CSC_OK);
        CHECK(sp.seg_first == 5 && sp.col_first == 5 * 1985 / 10 && sp.halo_left == 15);
        CHECK(csc_shard_plan_make(2000, 16, 10, 11, 0, &sp) == CSC_EINVAL);
        CHECK(csc_shard_phase(NULL, 0, 1e-6) == CSC_EINVAL);
        CHECK(csc2d_plan(121, 8, 8, &M, &c, starts) == CSC_OK);
        CHECK(M == 8 && c == 2 && starts[1] == 15);
        CHECK(csc2d_solve(NULL, 1, 1, 2, 2, NULL, 4, 4, 0.1, 1e-6, 1, 0, 0, 0, NULL, NULL, NULL,
                          NULL) == CSC_EINVAL);
    }
    printf("ok\n");
    return 0;
}
