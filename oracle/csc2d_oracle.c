/*
 * FP64 CPU oracle for the 2-D variant of convolutional sparse coding solved by
 * greedy and locally greedy coordinate descent with the image cut into bands
 * along one axis only (Moreau, Oudre & Vayatis, "DICOD", ICML 2018: the
 * paper's conclusion names splitting images along a single direction as the
 * way to keep its 1-D analysis, where a worker has only two neighbours).
 *
 * TEST INFRASTRUCTURE ONLY.  Like csc_oracle.c this is the slow, plain
 * reference a GPU implementation is checked against; only the tests may load
 * it.  It shares no code with any CUDA path.  Build:
 *     gcc -O2 -ffp-contract=off -std=c11 -fPIC -shared -o liboracle2d.so csc2d_oracle.c
 *
 * The problem is Eq. sparse_code with 2-D convolutions:
 *   D[k][p][u][v]  atom k, channel p, u in [0,h), v in [0,w)       (float input)
 *   X[p][y][x]     image, y in [0,H), x in [0,W), zero outside     (float input)
 *   Z[k][i][j]     activations, i in [0,Hz), j in [0,Wz),
 *                  Hz = H - h + 1, Wz = W - w + 1 ("valid" placement) (double)
 *   E(Z) = 1/2 sum_p || X_p - sum_k Z_k * D_kp ||^2 + lambda sum |Z|
 * with (Z_k * D_kp)[y][x] = sum_{u,v} Z_k[y-u][x-v] D[k][p][u][v].
 * Everything of Sec. 2.1 carries over with 2-D lags:
 *   beta_k[i][j] = sum_p sum_{u,v} D[k][p][u][v] R[p][i+u][j+v] + ||D_k||^2 Z_k[i][j],
 *       R = X - sum_l Z_l * D_l (the residual);
 *   S[k][l][a][b] = sum_p sum_{u,v} D[k][p][u][v] D[l][p][u+a-(h-1)][v+b-(w-1)],
 *       the cross-correlation at lag (a-(h-1), b-(w-1));
 *   the coordinate optimum is Sh(beta, lambda) / ||D_k||^2 (Eq. pb_coord), and
 *   changing Z_k0[i0][j0] by delta lowers beta_k[i][j] by
 *   S[k][k0][i-i0+h-1][j-j0+w-1] * delta on the (2h-1) x (2w-1) window, own
 *   coordinate excluded (Eq. beta_up, sign as derived in csc_oracle.c).
 * Bands (the segments of Sec. 2.2 along rows): band m of M holds the rows
 * [floor(m*Hz/M), floor((m+1)*Hz/M)) and every column.  An update in a band
 * touches rows [start-h+1, end+h-1), so bands m, m' run together only when
 * m == m' (mod c) with (c-1) * min band height >= 2h-2.
 * Argmax ties go to the lowest flat index (k*Hz + i)*Wz + j.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef long long i64;

static double sh(double u, double lam)
{
    double a = fabs(u) - lam;
    if (a <= 0.0)
        return 0.0;
    return u > 0.0 ? a : -a;
}

/* ||D_k||^2 over channels and both lags. */
void o2_norms(const float *D, int K, int P, int h, int w, double *n)
{
    const i64 A = (i64)P * h * w;
    for (int k = 0; k < K; k++) {
        double s = 0.0;
        for (i64 e = 0; e < A; e++) {
            double d = (double)D[(i64)k * A + e];
            s += d * d;
        }
        n[k] = s;
    }
}

/* S[k][l][a][b] as defined above, shape K*K*(2h-1)*(2w-1). */
void o2_crosscorr(const float *D, int K, int P, int h, int w, double *S)
{
    const int H2 = 2 * h - 1, W2 = 2 * w - 1;
    for (int k = 0; k < K; k++)
        for (int l = 0; l < K; l++)
            for (int a = 0; a < H2; a++)
                for (int b = 0; b < W2; b++) {
                    const int da = a - (h - 1), db = b - (w - 1);
                    double acc = 0.0;
                    for (int p = 0; p < P; p++)
                        for (int u = 0; u < h; u++) {
                            const int u2 = u + da;
                            if (u2 < 0 || u2 >= h)
                                continue;
                            for (int v = 0; v < w; v++) {
                                const int v2 = v + db;
                                if (v2 < 0 || v2 >= w)
                                    continue;
                                acc += (double)D[(((i64)k * P + p) * h + u) * w + v] *
                                       (double)D[(((i64)l * P + p) * h + u2) * w + v2];
                            }
                        }
                    S[(((i64)k * K + l) * H2 + a) * W2 + b] = acc;
                }
}

/* beta with the residual replaced by a given image R (double), plus nothing:
 * out[k][i][j] = sum_p sum_{u,v} D[k][p][u][v] R[p][i+u][j+v]. */
static void corr_valid(const float *D, const double *R, int K, int P, int h, int w, i64 H, i64 W,
                       double *out)
{
    const i64 Hz = H - h + 1, Wz = W - w + 1;
    for (int k = 0; k < K; k++)
        for (i64 i = 0; i < Hz; i++)
            for (i64 j = 0; j < Wz; j++) {
                double acc = 0.0;
                for (int p = 0; p < P; p++)
                    for (int u = 0; u < h; u++)
                        for (int v = 0; v < w; v++)
                            acc += (double)D[(((i64)k * P + p) * h + u) * w + v] *
                                   R[((i64)p * H + i + u) * W + j + v];
                out[((i64)k * Hz + i) * Wz + j] = acc;
            }
}

static double *to_double(const float *X, i64 n)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    if (r)
        for (i64 e = 0; e < n; e++)
            r[e] = (double)X[e];
    return r;
}

/* beta0 = D~ * X (Alg. 1 initialisation), [K][Hz][Wz]. */
void o2_dtx(const float *D, const float *X, int K, int P, int h, int w, i64 H, i64 W, double *beta)
{
    double *R = to_double(X, (i64)P * H * W);
    if (!R)
        return;
    corr_valid(D, R, K, P, h, w, H, W, beta);
    free(R);
}

/* R = X - sum_k Z_k * D_k, [P][H][W]. */
void o2_residual(const float *D, const float *X, const double *Z, int K, int P, int h, int w,
                 i64 H, i64 W, double *R)
{
    const i64 Hz = H - h + 1, Wz = W - w + 1;
    for (i64 e = 0; e < (i64)P * H * W; e++)
        R[e] = (double)X[e];
    for (int k = 0; k < K; k++)
        for (i64 i = 0; i < Hz; i++)
            for (i64 j = 0; j < Wz; j++) {
                const double z = Z[((i64)k * Hz + i) * Wz + j];
                if (z == 0.0)
                    continue;
                for (int p = 0; p < P; p++)
                    for (int u = 0; u < h; u++)
                        for (int v = 0; v < w; v++)
                            R[((i64)p * H + i + u) * W + j + v] -=
                                z * (double)D[(((i64)k * P + p) * h + u) * w + v];
            }
}

/* E(Z) of the 2-D Eq. sparse_code. */
double o2_objective(const float *D, const float *X, const double *Z, int K, int P, int h, int w,
                    i64 H, i64 W, double lam)
{
    const i64 nR = (i64)P * H * W, nZ = (i64)K * (H - h + 1) * (W - w + 1);
    double *R = (double *)malloc(sizeof(double) * (size_t)nR);
    if (!R)
        return NAN;
    o2_residual(D, X, Z, K, P, h, w, H, W, R);
    double sq = 0.0, l1 = 0.0;
    for (i64 e = 0; e < nR; e++)
        sq += R[e] * R[e];
    for (i64 e = 0; e < nZ; e++)
        l1 += fabs(Z[e]);
    free(R);
    return 0.5 * sq + lam * l1;
}

/* beta from its definition at Z (Sec. 2.1 in 2-D). */
void o2_beta_fresh(const float *D, const float *X, const double *Z, int K, int P, int h, int w,
                   i64 H, i64 W, double *beta)
{
    const i64 Hz = H - h + 1, Wz = W - w + 1;
    double *R = (double *)malloc(sizeof(double) * (size_t)((i64)P * H * W));
    double *n = (double *)malloc(sizeof(double) * (size_t)K);
    if (!R || !n) {
        free(R);
        free(n);
        return;
    }
    o2_residual(D, X, Z, K, P, h, w, H, W, R);
    corr_valid(D, R, K, P, h, w, H, W, beta);
    o2_norms(D, K, P, h, w, n);
    for (int k = 0; k < K; k++)
        for (i64 e = 0; e < Hz * Wz; e++)
            beta[(i64)k * Hz * Wz + e] += n[k] * Z[(i64)k * Hz * Wz + e];
    free(R);
    free(n);
}

/* Band m of M over the Hz rows: [floor(m*Hz/M), floor((m+1)*Hz/M)). */
i64 o2_band_start(i64 Hz, int M, int m)
{
    return (i64)m * Hz / M;
}

/* Phases of the band schedule: c with (c-1) * min band height >= 2h-2. */
int o2_phase_count(i64 Hz, int M, int h)
{
    if (M <= 1)
        return 1;
    const i64 hmin = Hz / M;
    if (hmin < 1)
        return -1;
    const i64 need = 2 * (i64)h - 2;
    i64 c = 1 + (need + hmin - 1) / hmin;
    if (c > M)
        c = M;
    return (int)c;
}

/* ------------------------------------------------------------ CD state */

typedef struct {
    int K, P, h, w;
    i64 H, W, Hz, Wz;
    double lam;
    double *S, *n, *Z, *beta;
    int *tr_k;
    i64 *tr_t;
    double *tr_old, *tr_new;
    i64 tr_cap, tr_len;
} st2;

static int st_init(st2 *s, const float *D, const float *X, int K, int P, int h, int w, i64 H, i64 W,
                   double lam, double *Z, double *beta)
{
    memset(s, 0, sizeof(*s));
    s->K = K;
    s->P = P;
    s->h = h;
    s->w = w;
    s->H = H;
    s->W = W;
    s->Hz = H - h + 1;
    s->Wz = W - w + 1;
    s->lam = lam;
    s->Z = Z;
    s->beta = beta;
    s->S = (double *)malloc(sizeof(double) * (size_t)K * K * (2 * h - 1) * (2 * w - 1));
    s->n = (double *)malloc(sizeof(double) * (size_t)K);
    if (!s->S || !s->n)
        return -1;
    o2_crosscorr(D, K, P, h, w, s->S);
    o2_norms(D, K, P, h, w, s->n);
    for (i64 e = 0; e < (i64)K * s->Hz * s->Wz; e++)
        Z[e] = 0.0;
    o2_dtx(D, X, K, P, h, w, H, W, beta);
    return 0;
}

static void st_free(st2 *s)
{
    free(s->S);
    free(s->n);
}

/* argmax of |Z - Sh(beta,lam)/n| over k and rows [r0, r1), all columns;
 * ties to the lowest flat index.  Returns the max |Delta Z|. */
static double band_argmax(const st2 *s, i64 r0, i64 r1, int *k0, i64 *i0, i64 *j0, double *znew)
{
    double best = -1.0;
    for (int k = 0; k < s->K; k++)
        for (i64 i = r0; i < r1; i++)
            for (i64 j = 0; j < s->Wz; j++) {
                const i64 e = ((i64)k * s->Hz + i) * s->Wz + j;
                const double zp = sh(s->beta[e], s->lam) / s->n[k];
                const double d = fabs(s->Z[e] - zp);
                if (d > best) {
                    best = d;
                    *k0 = k;
                    *i0 = i;
                    *j0 = j;
                    *znew = zp;
                }
            }
    return best;
}

/* Z_k0[i0][j0] <- znew and the 2-D Eq. beta_up on the window. */
static void apply2(st2 *s, int k0, i64 i0, i64 j0, double znew)
{
    const int h = s->h, w = s->w, H2 = 2 * h - 1, W2 = 2 * w - 1;
    const i64 e0 = ((i64)k0 * s->Hz + i0) * s->Wz + j0;
    const double zold = s->Z[e0], delta = znew - zold;
    i64 ilo = i0 - (h - 1), ihi = i0 + (h - 1), jlo = j0 - (w - 1), jhi = j0 + (w - 1);
    if (ilo < 0)
        ilo = 0;
    if (ihi > s->Hz - 1)
        ihi = s->Hz - 1;
    if (jlo < 0)
        jlo = 0;
    if (jhi > s->Wz - 1)
        jhi = s->Wz - 1;
    for (int k = 0; k < s->K; k++) {
        const double *Sk = s->S + ((i64)k * s->K + k0) * H2 * W2;
        for (i64 i = ilo; i <= ihi; i++)
            for (i64 j = jlo; j <= jhi; j++) {
                if (k == k0 && i == i0 && j == j0)
                    continue;
                s->beta[((i64)k * s->Hz + i) * s->Wz + j] -=
                    Sk[(i - i0 + (h - 1)) * W2 + (j - j0 + (w - 1))] * delta;
            }
    }
    s->Z[e0] = znew;
    if (s->tr_len < s->tr_cap) {
        s->tr_k[s->tr_len] = k0;
        s->tr_t[s->tr_len] = i0 * s->Wz + j0;
        s->tr_old[s->tr_len] = zold;
        s->tr_new[s->tr_len] = znew;
    }
    s->tr_len++;
}

/* Greedy CD (Alg. 1) on the image, literal order: apply the global argmax,
 * stop once the applied |Delta Z| < eps.  Trace positions are i*Wz + j. */
i64 o2_greedy_cd(const float *D, const float *X, int K, int P, int h, int w, i64 H, i64 W,
                 double lam, double eps, i64 max_updates, double *Z, double *beta, int *tr_k,
                 i64 *tr_t, double *tr_old, double *tr_new, i64 tr_cap, int *converged)
{
    st2 s;
    *converged = 0;
    if (st_init(&s, D, X, K, P, h, w, H, W, lam, Z, beta)) {
        st_free(&s);
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
        i64 i0 = 0, j0 = 0;
        double znew = 0.0;
        const double d = band_argmax(&s, 0, s.Hz, &k0, &i0, &j0, &znew);
        apply2(&s, k0, i0, j0, znew);
        q++;
        if (d < eps) {
            *converged = 1;
            break;
        }
    }
    st_free(&s);
    return q;
}

/* SplitMix64 output function (Steele, Lea & Flood 2014) for the random band
 * choice of Alg. 3. */
static uint64_t mix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

/* Locally greedy CD on M row bands (Alg. 3 along one axis).
 * mode 0: a band drawn uniformly per step (SplitMix64 on (seed, step)); its
 *   argmax is applied and dZ_m recorded; stop when every recorded dZ_m < eps
 *   and the global max |Delta Z| < eps.
 * mode 1: the band phase schedule: sweeps over phases p = 0..c-1, in phase p
 *   the bands m == p (mod c) in ascending order, each visit applying up to
 *   updates_per_visit (0 = no limit) updates while its max |Delta Z| >= eps;
 *   converged after a sweep that applied nothing.
 * Returns the applied updates; *sweeps receives the sweeps (mode 1). */
i64 o2_locally_greedy_cd(const float *D, const float *X, int K, int P, int h, int w, i64 H, i64 W,
                         double lam, double eps, i64 max_updates, int M, int mode, uint64_t seed,
                         int updates_per_visit, double *Z, double *beta, int *tr_k, i64 *tr_t,
                         double *tr_old, double *tr_new, i64 tr_cap, int *converged, i64 *sweeps)
{
    st2 s;
    *converged = 0;
    *sweeps = 0;
    const i64 Hz = H - h + 1;
    if (M < 1 || M > Hz)
        return -1;
    if (st_init(&s, D, X, K, P, h, w, H, W, lam, Z, beta)) {
        st_free(&s);
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
            const int m = (int)(mix64(seed ^ mix64((uint64_t)q)) % (uint64_t)M);
            int k0 = 0;
            i64 i0 = 0, j0 = 0;
            double znew = 0.0;
            const double d = band_argmax(&s, o2_band_start(Hz, M, m), o2_band_start(Hz, M, m + 1),
                                         &k0, &i0, &j0, &znew);
            apply2(&s, k0, i0, j0, znew);
            q++;
            dZ[m] = d;
            double dmax = 0.0;
            for (int b = 0; b < M; b++)
                if (dZ[b] > dmax)
                    dmax = dZ[b];
            if (dmax < eps) {
                int kk;
                i64 ii, jj;
                double zz;
                if (band_argmax(&s, 0, Hz, &kk, &ii, &jj, &zz) < eps) {
                    *converged = 1;
                    break;
                }
            }
        }
        free(dZ);
    } else {
        const int c = o2_phase_count(Hz, M, h);
        int stop = 0;
        while (!stop) {
            i64 in_sweep = 0;
            for (int p = 0; p < c && !stop; p++)
                for (int m = p; m < M && !stop; m += c) {
                    const i64 r0 = o2_band_start(Hz, M, m), r1 = o2_band_start(Hz, M, m + 1);
                    for (int it = 0; updates_per_visit <= 0 || it < updates_per_visit; it++) {
                        int k0 = 0;
                        i64 i0 = 0, j0 = 0;
                        double znew = 0.0;
                        const double d = band_argmax(&s, r0, r1, &k0, &i0, &j0, &znew);
                        if (d < eps)
                            break;
                        if (q >= max_updates) {
                            stop = 1;
                            break;
                        }
                        apply2(&s, k0, i0, j0, znew);
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
    st_free(&s);
    return q;
}
