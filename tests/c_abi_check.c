/*
 * A plain C99 caller of the library's C ABI (include/csc.h and
 * include/csc_server.h): it must compile as C with every warning an error,
 * link against libcsc.so and, without a GPU, get the documented results of
 * the host-only entry points and of argument validation.  Exit status 0 on
 * success; the first failed check is printed.
 */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "csc.h"
#include "csc_server.h"

#define CHECK(c)                                                  \
    do {                                                          \
        if (!(c)) {                                               \
            printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #c);   \
            return 1;                                             \
        }                                                         \
    } while (0)

int main(void)
{
    csc_opts o;
    csc_handle_t h = NULL;
    csc_server_t srv = NULL;
    int M = 0, c = 0, k;
    int64_t starts[11];
    float D[2 * 1 * 4];
    double out[3];

    memset(&o, 0x7f, sizeof o);
    csc_default_opts(&o);
    CHECK(o.segments == 0 && o.updates_per_visit == 0 && o.max_resyncs == -1);
    CHECK(o.reserved[0] == 0);

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
    printf("ok\n");
    return 0;
}
