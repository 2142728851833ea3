/*
 * Multi-core CPU baseline (benchmark only, not a test reference): the FP64
 * locally greedy coordinate descent of csc_oracle.c's segment phase schedule
 * (Sec. 2.3, Alg. 3 visited in the phases of Sec. 2.2), with the segments of
 * one phase run in parallel by OpenMP threads.  Co-active segments never
 * touch the same beta entries (their update windows are disjoint), so every
 * thread count gives the same arithmetic, in the same order per segment, as
 * the single-threaded oracle: the tests check that the result is identical.
 * This is the CPU analogue of DICOD (one worker per segment of a phase).
 *
 * Plain C, FP64, built with -fopenmp -ffp-contract=off.  Shares no code with
 * the CUDA path.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef long long i64;

static double sh(double u, double lam)
{
    double a = fabs(u) - lam;
    return a > 0.0 ? copysign(a, u) : 0.0;
}

static i64 seg_start(i64 Tz, int M, int m)
{
    return (i64)m * Tz / M;
}

static int phase_count(i64 Tz, int M, int L)
{
    if (M <= 1)
        return 1;
    i64 wmin = Tz / M;
    i64 need = 2 * (i64)L - 2;
    i64 c = 1 + (need + wmin - 1) / wmin;
    return (int)(c > M ? M : c);
}

int omp_threads_used(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Returns the applied updates; Z [K][Tz] and beta [K][Tz] are caller-owned;
 * *converged = 1 after a sweep without update; threads <= 0: the default. */
i64 omp_phase_cd(const float *D, const float *X, int K, int P, int L, i64 T, double lam,
                 double eps, int M, int updates_per_visit, int threads, double *Z, double *beta,
                 int *converged, i64 *sweeps)
{
    const i64 Tz = T - L + 1;
    const int W2 = 2 * L - 1;
    *converged = 0;
    *sweeps = 0;
    if (M < 1 || M > Tz)
        return -1;
#ifdef _OPENMP
    if (threads > 0)
        omp_set_num_threads(threads);
#endif
    double *S = (double *)malloc(sizeof(double) * (size_t)K * K * W2);
    double *n = (double *)malloc(sizeof(double) * (size_t)K);
    if (!S || !n) {
        free(S);
        free(n);
        return -1;
    }
    /* S_{k,l}[s-(L-1)] and the norms, in the oracle's summation order */
    for (int k = 0; k < K; k++)
        for (int l = 0; l < K; l++)
            for (int s = 0; s < W2; s++) {
                int d = s - (L - 1);
                double acc = 0.0;
                for (int p = 0; p < P; p++)
                    for (int tau = 0; tau < L; tau++) {
                        int u = tau + d;
                        if (u < 0 || u >= L)
                            continue;
                        acc += (double)D[((i64)k * P + p) * L + tau] *
                               (double)D[((i64)l * P + p) * L + u];
                    }
                S[((i64)k * K + l) * W2 + s] = acc;
            }
    for (int k = 0; k < K; k++) {
        double acc = 0.0;
        for (int p = 0; p < P; p++)
            for (int tau = 0; tau < L; tau++) {
                double v = D[((i64)k * P + p) * L + tau];
                acc += v * v;
            }
        n[k] = acc;
    }
    /* Z = 0, beta = D~ * X */
#pragma omp parallel for schedule(static)
    for (i64 kt = 0; kt < (i64)K * Tz; kt++) {
        const int k = (int)(kt / Tz);
        const i64 t = kt % Tz;
        double acc = 0.0;
        for (int p = 0; p < P; p++)
            for (int tau = 0; tau < L; tau++)
                acc += (double)D[((i64)k * P + p) * L + tau] * (double)X[(i64)p * T + t + tau];
        beta[kt] = acc;
        Z[kt] = 0.0;
    }
    const int c = phase_count(Tz, M, L);
    i64 q = 0;
    for (;;) {
        i64 in_sweep = 0;
        for (int p = 0; p < c; p++) {
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : in_sweep)
            for (int m = p; m < M; m += c) {
                const i64 a = seg_start(Tz, M, m), b = seg_start(Tz, M, m + 1);
                for (int it = 0; updates_per_visit <= 0 || it < updates_per_visit; it++) {
                    /* local argmax of |Z - Z'|, ties to the lowest k*Tz+t */
                    double best = -1.0, znew = 0.0;
                    int k0 = 0;
                    i64 t0 = 0;
                    for (int k = 0; k < K; k++)
                        for (i64 t = a; t < b; t++) {
                            double zp = sh(beta[(i64)k * Tz + t], lam) / n[k];
                            double d = fabs(Z[(i64)k * Tz + t] - zp);
                            if (d > best) {
                                best = d;
                                k0 = k;
                                t0 = t;
                                znew = zp;
                            }
                        }
                    if (best < eps)
                        break;
                    /* Eq. beta_up on the window, own coordinate excluded */
                    const double delta = znew - Z[(i64)k0 * Tz + t0];
                    i64 lo = t0 - (L - 1), hi = t0 + (L - 1);
                    if (lo < 0)
                        lo = 0;
                    if (hi > Tz - 1)
                        hi = Tz - 1;
                    for (int k = 0; k < K; k++) {
                        const double *Sk = S + ((i64)k * K + k0) * W2;
                        for (i64 t = lo; t <= hi; t++) {
                            if (k == k0 && t == t0)
                                continue;
                            beta[(i64)k * Tz + t] -= Sk[t - t0 + (L - 1)] * delta;
                        }
                    }
                    Z[(i64)k0 * Tz + t0] = znew;
                    in_sweep++;
                }
            }
        }
        q += in_sweep;
        (*sweeps)++;
        if (in_sweep == 0) {
            *converged = 1;
            break;
        }
    }
    free(S);
    free(n);
    return q;
}
