/*
 * FP64 CPU oracle for 1-D multichannel convolutional sparse coding solved by
 * greedy and locally greedy coordinate descent, after Moreau, Oudre & Vayatis,
 * "DICOD: Distributed Convolutional Coordinate Descent for Convolutional
 * Sparse Coding" (ICML 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA solver is checked against.  Only the tests, the package smoke check and
 * the benchmark's CPU-baseline / reference leg may load it.  It shares no code,
 * header, table or helper with the CUDA path.  Build:
 *     gcc -O2 -ffp-contract=off -std=c11 -fPIC -shared -o liboracle.so csc_oracle.c
 * (-ffp-contract=off: every product and sum is rounded separately, as written.)
 *
 * Notation (Sec. 2, "Notations" and "Convolutional Sparse Coding").  The paper
 * calls the atom length W and the activation length L; here the atom length is
 * L and the activation length is Tz = T - L + 1.
 *   D[k][p][tau]  atom k, channel p, tau in [0,L)        (float input)
 *   X[p][t]       signal, t in [0,T), zero outside        (float input)
 *   Z[k][t]       activations, t in [0,Tz)                (double)
 *   beta[k][t]    auxiliary variable of Sec. 2.1           (double)
 *   S[k][l][s]    cross-correlation of atoms (Eq. beta_up), lag s-(L-1):
 *                 S[k][l][s] = sum_p sum_tau D[k][p][tau] * D[l][p][tau+s-(L-1)]
 *
 * Readings of the paper used here (each is also listed in the design notes):
 *  - beta update sign.  From the definition of beta (Sec. 2.1), raising
 *    Z_k0[t0] by delta = Z'-Z lowers beta_k[t] by S_{k,k0}[t-t0]*delta, so the
 *    update applied is beta -= S*(Z' - Z_old) for all (k,t) != (k0,t0).
 *  - Lag direction.  S_{k,l}[t] = sum_u D_k[u] D_l[u+t] (reversal taken about
 *    0, so S vanishes outside [-(L-1), L-1] as Sec. 2.1 states).
 *  - Segments (Sec. 2.2) are 0-based [floor(m*Tz/M), floor((m+1)*Tz/M)).
 *  - Argmax ties (Alg. 1 / Alg. 3) go to the lowest flat index k*Tz + t.
 *  - Sh(u, lambda) with |u| == lambda is 0.
 *  - Alg. 3's dZ_m is the magnitude |Z'-Z| of the update just made in m.
 *  - Alg. 3's random segment choice uses SplitMix64 (Steele, Lea & Flood
 *    2014) on (seed, step), reduced modulo M.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef long long i64;

/* ---------------------------------------------------------------- basics */

/* Soft thresholding, Sec. 2.1: Sh(u, lam) = sign(u) max(|u| - lam, 0). */
double orc_soft_threshold(double u, double lam)
{
    double a = fabs(u) - lam;
    if (a <= 0.0)
        return 0.0;
    return u > 0.0 ? a : -a;
}

/* ||D_k||_2^2 for every atom (the denominator of Eq. pb_coord). */
void orc_norms(const float *D, int K, int P, int L, double *n)
{
    for (int k = 0; k < K; k++) {
        double s = 0.0;
        for (int p = 0; p < P; p++)
            for (int tau = 0; tau < L; tau++) {
                double d = (double)D[((i64)k * P + p) * L + tau];
                s += d * d;
            }
        n[k] = s;
    }
}

/* S_{k,l}[s-(L-1)] for s in [0, 2L-1) (Sec. 2.1, below Eq. beta_up). */
void orc_crosscorr(const float *D, int K, int P, int L, double *S)
{
    int W2 = 2 * L - 1;
    for (int k = 0; k < K; k++)
        for (int l = 0; l < K; l++)
            for (int s = 0; s < W2; s++) {
                int lag = s - (L - 1);
                double acc = 0.0;
                for (int p = 0; p < P; p++)
                    for (int tau = 0; tau < L; tau++) {
                        int u = tau + lag;
                        if (u < 0 || u >= L)
                            continue;
                        acc += (double)D[((i64)k * P + p) * L + tau] *
                               (double)D[((i64)l * P + p) * L + u];
                    }
                S[((i64)k * K + l) * W2 + s] = acc;
            }
}

/* (D~_k * X)[t] = sum_p sum_tau D[k][p][tau] X[p][t+tau], t in [0,Tz):
 * the initial beta of Alg. 1 (Z = 0). */
void orc_dtx(const float *D, const float *X, int K, int P, int L, i64 T, double *beta)
{
    i64 Tz = T - L + 1;
    for (int k = 0; k < K; k++)
        for (i64 t = 0; t < Tz; t++) {
            double acc = 0.0;
            for (int p = 0; p < P; p++)
                for (int tau = 0; tau < L; tau++)
                    acc += (double)D[((i64)k * P + p) * L + tau] * (double)X[(i64)p * T + t + tau];
            beta[(i64)k * Tz + t] = acc;
        }
}

/* Residual R = X - sum_k Z_k * D_k (Eq. model without noise term), where
 * (Z*D)[t] = sum_tau Z[t-tau] D[tau] (Sec. 2, "Notations").  Zero entries of
 * Z contribute nothing and are skipped. */
void orc_residual(const float *D, const float *X, const double *Z, int K, int P, int L, i64 T,
                  double *R)
{
    i64 Tz = T - L + 1;
    for (i64 i = 0; i < (i64)P * T; i++)
        R[i] = (double)X[i];
    for (int k = 0; k < K; k++)
        for (i64 t0 = 0; t0 < Tz; t0++) {
            double z = Z[(i64)k * Tz + t0];
            if (z == 0.0)
                continue;
            for (int p = 0; p < P; p++)
                for (int tau = 0; tau < L; tau++)
                    R[(i64)p * T + t0 + tau] -= z * (double)D[((i64)k * P + p) * L + tau];
        }
}

/* E(Z) = 1/2 ||X - sum_k Z_k*D_k||_2^2 + lambda sum_k ||Z_k||_1 (Eq. sparse_code). */
double orc_objective(const float *D, const float *X, const double *Z, int K, int P, int L, i64 T,
                     double lam)
{
    i64 Tz = T - L + 1;
    double *R = (double *)malloc(sizeof(double) * (size_t)(P * T));
    if (!R)
        return NAN;
    orc_residual(D, X, Z, K, P, L, T, R);
    double sq = 0.0, l1 = 0.0;
    for (i64 i = 0; i < (i64)P * T; i++)
        sq += R[i] * R[i];
    for (i64 i = 0; i < (i64)K * Tz; i++)
        l1 += fabs(Z[i]);
    free(R);
    return 0.5 * sq + lam * l1;
}

/* beta from its definition (Sec. 2.1): the correlation of D_k with the
 * residual in which Z_k[t] itself is set to zero, i.e.
 *   beta_k[t] = (D~_k * R)[t] + ||D_k||^2 Z_k[t],  R = X - sum Z*D. */
void orc_beta_fresh(const float *D, const float *X, const double *Z, int K, int P, int L, i64 T,
                    double *beta)
{
    i64 Tz = T - L + 1;
    double *R = (double *)malloc(sizeof(double) * (size_t)(P * T));
    double *n = (double *)malloc(sizeof(double) * (size_t)K);
    if (!R || !n) {
        free(R);
        free(n);
        return;
    }
    orc_residual(D, X, Z, K, P, L, T, R);
    orc_norms(D, K, P, L, n);
    for (int k = 0; k < K; k++)
        for (i64 t = 0; t < Tz; t++) {
            double acc = 0.0;
            for (int p = 0; p < P; p++)
                for (int tau = 0; tau < L; tau++)
                    acc += (double)D[((i64)k * P + p) * L + tau] * R[(i64)p * T + t + tau];
            beta[(i64)k * Tz + t] = acc + n[k] * Z[(i64)k * Tz + t];
        }
    free(R);
    free(n);
}

/* Optimality report.  By coordinate-wise optimality (Theorem A.1, after
 * Osher & Li 2009) Z is optimal iff every coordinate solves Eq. pb_coord:
 *   Z_k[t] == 0  =>  |beta_k[t]| <= lambda            (out[0] = max excess)
 *   Z_k[t] != 0  =>  Z_k[t] == Sh(beta_k[t],lam)/n_k  (out[1] = max |gap|)
 * out[2] = max over all coordinates of |Z - Sh(beta,lam)/n| (max |Delta Z|). */
void orc_kkt(const double *beta, const double *Z, const double *n, int K, i64 Tz, double lam,
             double *out)
{
    double v0 = 0.0, v1 = 0.0, vall = 0.0;
    for (int k = 0; k < K; k++)
        for (i64 t = 0; t < Tz; t++) {
            double b = beta[(i64)k * Tz + t], z = Z[(i64)k * Tz + t];
            double d = fabs(z - orc_soft_threshold(b, lam) / n[k]);
            if (z == 0.0) {
                double e = fabs(b) - lam;
                if (e > v0)
                    v0 = e;
            } else if (d > v1) {
                v1 = d;
            }
            if (d > vall)
                vall = d;
        }
    out[0] = v0;
    out[1] = v1;
    out[2] = vall;
}

/* Segment m of M over [0,Tz): [floor(m*Tz/M), floor((m+1)*Tz/M)). */
i64 orc_segment_start(i64 Tz, int M, int m)
{
    return (i64)m * Tz / M;
}

/* Number of phases of the segment schedule: segments m and m' are processed
 * together only when m == m' (mod c).  Each update touches beta on
 * [t0-L+1, t0+L-1] (Eq. beta_up), so the segments strictly between two
 * co-active ones must span at least 2L-2 samples: (c-1)*w_min >= 2L-2. */
int orc_phase_count(i64 Tz, int M, int L)
{
    if (M <= 1)
        return 1;
    i64 wmin = Tz / M;
    if (wmin < 1)
        return -1;
    i64 need = 2 * (i64)L - 2;
    i64 c = 1 + (need + wmin - 1) / wmin;
    if (c > M)
        c = M;
    return (int)c;
}

/* ------------------------------------------------------------ CD state */

typedef struct {
    int K, P, L;
    i64 T, Tz;
    double lam;
    double *S;    /* K*K*(2L-1) */
    double *n;    /* K */
    double *Z;    /* K*Tz, caller-owned */
    double *beta; /* K*Tz, caller-owned */
    /* optional update trace (all applied updates, in order) */
    int *tr_k;
    i64 *tr_t;
    double *tr_old, *tr_new;
    i64 tr_cap, tr_len;
} cd_state;

static int state_init(cd_state *s, const float *D, const float *X, int K, int P, int L, i64 T,
                      double lam, double *Z, double *beta)
{
    memset(s, 0, sizeof(*s));
    s->K = K;
    s->P = P;
    s->L = L;
    s->T = T;
    s->Tz = T - L + 1;
    s->lam = lam;
    s->Z = Z;
    s->beta = beta;
    s->S = (double *)malloc(sizeof(double) * (size_t)K * K * (2 * L - 1));
    s->n = (double *)malloc(sizeof(double) * (size_t)K);
    if (!s->S || !s->n)
        return -1;
    orc_crosscorr(D, K, P, L, s->S);
    orc_norms(D, K, P, L, s->n);
    /* Alg. 1 / Alg. 3 initialisation: Z = 0, beta = D~ * X. */
    for (i64 i = 0; i < (i64)K * s->Tz; i++)
        Z[i] = 0.0;
    orc_dtx(D, X, K, P, L, T, beta);
    return 0;
}

static void state_free(cd_state *s)
{
    free(s->S);
    free(s->n);
}

/* Coordinate optimum, Eq. pb_coord: Z'_k[t] = Sh(beta_k[t], lam) / ||D_k||^2. */
static double zprime(const cd_state *s, int k, i64 t)
{
    return orc_soft_threshold(s->beta[(i64)k * s->Tz + t], s->lam) / s->n[k];
}

/* argmax over k in [0,K), t in [a,b) of |Z - Z'|, ties to the lowest k*Tz+t.
 * Returns the max |Delta Z|; (k0,t0,z0new) receive the chosen coordinate. */
static double local_argmax(const cd_state *s, i64 a, i64 b, int *k0, i64 *t0, double *znew)
{
    double best = -1.0;
    for (int k = 0; k < s->K; k++)
        for (i64 t = a; t < b; t++) {
            double zp = zprime(s, k, t);
            double d = fabs(s->Z[(i64)k * s->Tz + t] - zp);
            if (d > best) {
                best = d;
                *k0 = k;
                *t0 = t;
                *znew = zp;
            }
        }
    return best;
}

/* Set Z_k0[t0] <- znew and keep beta consistent with Eq. beta_up (sign as
 * derived from the beta definition): for all (k,t) != (k0,t0) with
 * |t - t0| < L, beta_k[t] -= S_{k,k0}[t - t0] * (znew - Z_old). */
static void apply_update(cd_state *s, int k0, i64 t0, double znew)
{
    int L = s->L, W2 = 2 * L - 1;
    double zold = s->Z[(i64)k0 * s->Tz + t0];
    double delta = znew - zold;
    i64 lo = t0 - (L - 1), hi = t0 + (L - 1);
    if (lo < 0)
        lo = 0;
    if (hi > s->Tz - 1)
        hi = s->Tz - 1;
    for (int k = 0; k < s->K; k++) {
        const double *Sk = s->S + ((i64)k * s->K + k0) * W2;
        for (i64 t = lo; t <= hi; t++) {
            if (k == k0 && t == t0)
                continue;
            s->beta[(i64)k * s->Tz + t] -= Sk[t - t0 + (L - 1)] * delta;
        }
    }
    s->Z[(i64)k0 * s->Tz + t0] = znew;
    if (s->tr_len < s->tr_cap) {
        s->tr_k[s->tr_len] = k0;
        s->tr_t[s->tr_len] = t0;
        s->tr_old[s->tr_len] = zold;
        s->tr_new[s->tr_len] = znew;
    }
    s->tr_len++;
}

/* ------------------------------------------------------------- Alg. 1 */

/* Greedy coordinate descent (Alg. 1), literal order: choose the global
 * argmax of |Delta Z|, apply it, stop once the applied |Delta Z| < eps.
 * Returns the number of applied updates; *converged = 1 if stopped by eps,
 * 0 if max_updates was reached first.  Z, beta: K*Tz outputs. */
i64 orc_greedy_cd(const float *D, const float *X, int K, int P, int L, i64 T, double lam,
                  double eps, i64 max_updates, double *Z, double *beta, int *tr_k, i64 *tr_t,
                  double *tr_old, double *tr_new, i64 tr_cap, int *converged)
{
    cd_state s;
    *converged = 0;
    if (state_init(&s, D, X, K, P, L, T, lam, Z, beta)) {
        state_free(&s);
        return -1;
    }
    s.tr_k = tr_k;
    s.tr_t = tr_t;
    s.tr_old = tr_old;
    s.tr_new = tr_new;
    s.tr_cap = tr_cap;
    i64 q = 0;
    while (q < max_updates) {
        int k0 = 0;
        i64 t0 = 0;
        double znew = 0.0;
        double d = local_argmax(&s, 0, s.Tz, &k0, &t0, &znew);
        apply_update(&s, k0, t0, znew);
        q++;
        if (d < eps) {
            *converged = 1;
            break;
        }
    }
    state_free(&s);
    return q;
}

/* ------------------------------------------------------------- Alg. 3 */

static uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

/* Locally greedy coordinate descent on M segments (Sec. 2.3).
 *
 * mode 0 (Alg. 3, SeqDICOD_M, literal): each step picks a segment uniformly
 *   at random, applies its local argmax update, records dZ_m = |Delta Z|, and
 *   stops when ||dZ||_inf < eps and the global ||Delta Z||_inf < eps.
 *   max_updates bounds the number of steps.
 * mode 1 (the segment phase schedule, a DICOD_M interleaving meeting H2):
 *   sweeps visit phases p = 0..c-1 (c = orc_phase_count); in phase p the
 *   segments m == p (mod c) are visited in ascending order; a visit applies
 *   local argmax updates while |Delta Z| >= eps, at most updates_per_visit
 *   of them (0 = no cap).  Stops after a sweep with no update.  Segments of
 *   one phase never touch the same beta entries, so visiting them one after
 *   the other gives the same result as visiting them at the same time.
 * Returns applied updates; *converged, *sweeps as described. */
i64 orc_locally_greedy_cd(const float *D, const float *X, int K, int P, int L, i64 T, double lam,
                          double eps, i64 max_updates, int M, int mode, unsigned long long seed,
                          int updates_per_visit, double *Z, double *beta, int *tr_k, i64 *tr_t,
                          double *tr_old, double *tr_new, i64 tr_cap, int *converged,
                          i64 *sweeps)
{
    cd_state s;
    *converged = 0;
    *sweeps = 0;
    i64 Tz = T - L + 1;
    if (M < 1 || M > Tz)
        return -1;
    if (state_init(&s, D, X, K, P, L, T, lam, Z, beta)) {
        state_free(&s);
        return -1;
    }
    s.tr_k = tr_k;
    s.tr_t = tr_t;
    s.tr_old = tr_old;
    s.tr_new = tr_new;
    s.tr_cap = tr_cap;
    i64 q = 0;
    if (mode == 0) {
        double *dZ = (double *)malloc(sizeof(double) * (size_t)M);
        for (int m = 0; m < M; m++)
            dZ[m] = INFINITY;
        while (q < max_updates) {
            int m = (int)(splitmix64(seed ^ splitmix64((uint64_t)q)) % (uint64_t)M);
            int k0 = 0;
            i64 t0 = 0;
            double znew = 0.0;
            double d = local_argmax(&s, orc_segment_start(Tz, M, m),
                                    orc_segment_start(Tz, M, m + 1), &k0, &t0, &znew);
            apply_update(&s, k0, t0, znew);
            q++;
            dZ[m] = d;
            double dmax = 0.0;
            for (int j = 0; j < M; j++)
                if (dZ[j] > dmax)
                    dmax = dZ[j];
            if (dmax < eps) {
                int kk;
                i64 tt;
                double zz;
                if (local_argmax(&s, 0, Tz, &kk, &tt, &zz) < eps) {
                    *converged = 1;
                    break;
                }
            }
        }
        free(dZ);
    } else {
        int c = orc_phase_count(Tz, M, L);
        int stop = 0;
        while (!stop) {
            i64 in_sweep = 0;
            for (int p = 0; p < c && !stop; p++)
                for (int m = p; m < M && !stop; m += c) {
                    i64 a = orc_segment_start(Tz, M, m), b = orc_segment_start(Tz, M, m + 1);
                    for (int it = 0; updates_per_visit <= 0 || it < updates_per_visit; it++) {
                        int k0 = 0;
                        i64 t0 = 0;
                        double znew = 0.0;
                        double d = local_argmax(&s, a, b, &k0, &t0, &znew);
                        if (d < eps)
                            break;
                        if (q >= max_updates) {
                            stop = 1;
                            break;
                        }
                        apply_update(&s, k0, t0, znew);
                        q++;
                        in_sweep++;
                    }
                }
            (*sweeps)++;
            if (!stop && in_sweep == 0) {
                *converged = 1;
                stop = 1;
            }
        }
    }
    state_free(&s);
    return q;
}
