/*
 * ksg_oracle.c -- plain, slow, brute-force CPU oracle for the KSG conditional
 * mutual information estimator used by greedy multivariate transfer-entropy
 * network inference (Novelli et al., "Large-scale directed network inference
 * with multivariate transfer entropy and hierarchical statistical testing").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * What it computes (Methods, "Coupled logistic maps process": Kraskov's
 * estimator I^(1) with k nearest neighbours and its extension to conditional
 * mutual information; the paper prints no formula, the reading used here is
 * the Frenzel-Pompe form):
 *
 *   points i = 0..N-1 at time t_i = t0 + i; a variable (p, lag) has the value
 *   series[p][t_i - lag] at point i.  The X variables of a surrogate are read
 *   through a permutation pi: x at point i is series[p][t0 + pi(i) - lag]
 *   (Methods, "Maximum statistic test": the embedded source samples are
 *   shuffled, the target never is).
 *
 *   for each valid pair (j != i and |i - j| > theiler):
 *     dX = max_d fabsf(x_i,d - x_j,d)   (float32; the subtraction is the only
 *     dY, dZ likewise                    rounding; dZ = -inf when Z is empty)
 *   eps_i = k-th smallest max(dX, dY, dZ) over valid j (with multiplicity)
 *   n_xz = #{max(dX,dZ) < eps_i}, n_yz = #{max(dY,dZ) < eps_i},
 *   n_z  = #{dZ < eps_i}                                  (strict <)
 *   I = psi(k) + (1/N) sum_i [psi(n_z+1) - psi(n_xz+1) - psi(n_yz+1)]
 *
 * Two forms of the sum are reported:
 *   (a) I_plain: the FP64 sum in point order with an independent long-double
 *       digamma (asymptotic series + recurrence);
 *   (b) the exact key K = sum_i (Q[n_z+1] - Q[n_xz+1] - Q[n_yz+1]) in 128-bit
 *       integers, Q[n] = round_half_even(2^52 psi(n)), psi(n) = -gamma +
 *       H_{n-1}, and I_key = Q[k] 2^-52 + (double)K / (2^52 N).
 *
 * Surrogate permutations: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) keyed
 * by (seed, target, stage, iteration, surrogate), driving a Fisher-Yates
 * shuffle with Lemire's multiply-high range reduction.
 *
 * Parity pins for every function here live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2

/* ------------------------------------------------------------------------ */
/* Digamma at integers, exact fixed point.                                   */
/* psi(n) = -gamma + sum_{m=1}^{n-1} 1/m, accumulated with 100 fractional    */
/* bits in a signed 128-bit integer, then rounded half-to-even to 52 bits.   */
/* Euler-Mascheroni constant, 50 decimals (OEIS A001620).                    */
/* ------------------------------------------------------------------------ */
static const char *kGammaDigits = "57721566490153286060651209008240243104215933593992";

#define FRAC_BITS 100

static i128 gamma_fixed(void)
{
    /* gamma = 0.d1 d2 ... dn: Horner from the last digit, x <- (d + x) / 10 */
    const int n = (int)strlen(kGammaDigits);
    i128 one = (i128)1 << FRAC_BITS;
    i128 x = 0;
    for (int p = n - 1; p >= 0; --p) {
        i128 d = (i128)(kGammaDigits[p] - '0');
        x = (d * one + x) / 10;
    }
    return x;
}

/* Fill q[0..n_max]; q[0] is unused (psi has a pole at 0) and set to 0.
 * Returns the smallest distance (in units of 2^-100) from a rounding tie seen,
 * so a caller can confirm no entry sits near a tie. */
int oracle_digamma_q(int32_t n_max, int64_t *q, double *min_tie_margin)
{
    if (n_max < 1 || !q) return OR_EINVAL;
    const i128 one = (i128)1 << FRAC_BITS;
    const i128 g = gamma_fixed();
    const int shift = FRAC_BITS - 52;
    const i128 half = (i128)1 << (shift - 1);
    const i128 mod = (i128)1 << shift;
    i128 h = 0; /* H_{n-1} */
    double margin = 1e300;
    q[0] = 0;
    for (int32_t n = 1; n <= n_max; ++n) {
        if (n >= 2) h += one / (i128)(n - 1);
        i128 p = h - g; /* psi(n) * 2^100 */
        /* floor division by 2^shift for a signed value */
        i128 fl = p >= 0 ? p / mod : -((-p + mod - 1) / mod);
        i128 r = p - fl * mod; /* in [0, mod) */
        i128 qn;
        if (r > half) qn = fl + 1;
        else if (r < half) qn = fl;
        else qn = (fl & 1) ? fl + 1 : fl;
        i128 dist = r > half ? r - half : half - r;
        double dd = (double)dist;
        if (dd < margin) margin = dd;
        q[n] = (int64_t)qn;
    }
    if (min_tie_margin) *min_tie_margin = margin;
    return OR_OK;
}

/* Independent long-double digamma for the plain FP64 form: recurrence up to
 * x >= 16, then the asymptotic series ln x - 1/(2x) - sum B_2k/(2k x^2k). */
static long double digamma_ld(long double x)
{
    long double acc = 0.0L;
    while (x < 16.0L) {
        acc -= 1.0L / x;
        x += 1.0L;
    }
    long double inv = 1.0L / x;
    long double inv2 = inv * inv;
    /* Bernoulli numbers B2..B16 divided by 2k */
    long double series = inv2 * (1.0L / 12.0L -
                         inv2 * (1.0L / 120.0L -
                         inv2 * (1.0L / 252.0L -
                         inv2 * (1.0L / 240.0L -
                         inv2 * (1.0L / 132.0L -
                         inv2 * (691.0L / 32760.0L -
                         inv2 * (1.0L / 12.0L)))))));
    return acc + logl(x) - 0.5L * inv - series;
}

double oracle_digamma_plain(int32_t n) { return (double)digamma_ld((long double)n); }

/* ------------------------------------------------------------------------ */
/* SplitMix64 and Fisher-Yates                                               */
/* ------------------------------------------------------------------------ */
static uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* one SplitMix64 output from state x (state advanced once) */
static uint64_t splitmix64_from(uint64_t x) { return splitmix64_next(&x); }

/* n successive outputs of a SplitMix64 generator whose state starts at `state` */
void oracle_splitmix64_stream(uint64_t state, int32_t n, uint64_t *out)
{
    for (int32_t i = 0; i < n; ++i) out[i] = splitmix64_next(&state);
}

uint64_t oracle_perm_key(uint64_t seed, uint64_t target, uint64_t stage, uint64_t iter,
                         uint64_t surr)
{
    uint64_t h = splitmix64_from(seed ^ target);
    h = splitmix64_from(h ^ stage);
    h = splitmix64_from(h ^ iter);
    h = splitmix64_from(h ^ surr);
    return h;
}

int oracle_permutation(uint64_t seed, uint64_t target, uint64_t stage, uint64_t iter,
                       uint64_t surr, int32_t n, int32_t *perm)
{
    if (n < 1 || !perm) return OR_EINVAL;
    uint64_t state = oracle_perm_key(seed, target, stage, iter, surr);
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = n - 1; i >= 1; --i) {
        uint64_t r = splitmix64_next(&state);
        int32_t j = (int32_t)(((u128)r * (u128)(uint64_t)(i + 1)) >> 64);
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
    return OR_OK;
}

/* Surrogates of data with R replications (trials) of n points each, points
 * pooled trial by trial (point r*n + t).  Methods, Statistical tests,
 * surrogate paragraph: with enough replications the candidate's trial order
 * is shuffled (mode 0: perm[r*n + t] = sigma[r]*n + t, sigma a Fisher-Yates
 * shuffle of the R trials); otherwise its samples are shuffled inside each
 * trial (mode 1: one Fisher-Yates shuffle per trial, trial 0 first, all drawn
 * from one generator, so R = 1 gives oracle_permutation).  The generator
 * state starts at the same key as oracle_permutation. */
int oracle_permutation_trials(uint64_t seed, uint64_t target, uint64_t stage, uint64_t iter,
                              uint64_t surr, int32_t R, int32_t n, int32_t mode, int32_t *perm)
{
    if (R < 1 || n < 1 || !perm || (mode != 0 && mode != 1)) return OR_EINVAL;
    uint64_t state = oracle_perm_key(seed, target, stage, iter, surr);
    if (mode == 0) {
        int32_t *sigma = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
        if (!sigma) return OR_EINVAL;
        for (int32_t r = 0; r < R; ++r) sigma[r] = r;
        for (int32_t i = R - 1; i >= 1; --i) {
            uint64_t x = splitmix64_next(&state);
            int32_t j = (int32_t)(((u128)x * (u128)(uint64_t)(i + 1)) >> 64);
            int32_t t = sigma[i];
            sigma[i] = sigma[j];
            sigma[j] = t;
        }
        for (int32_t r = 0; r < R; ++r)
            for (int32_t t = 0; t < n; ++t) perm[(size_t)r * n + t] = sigma[r] * n + t;
        free(sigma);
        return OR_OK;
    }
    for (int32_t r = 0; r < R; ++r) {
        int32_t *b = perm + (size_t)r * n;
        for (int32_t t = 0; t < n; ++t) b[t] = r * n + t;
        for (int32_t i = n - 1; i >= 1; --i) {
            uint64_t x = splitmix64_next(&state);
            int32_t j = (int32_t)(((u128)x * (u128)(uint64_t)(i + 1)) >> 64);
            int32_t t = b[i];
            b[i] = b[j];
            b[j] = t;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Brute-force KSG CMI for one member                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    const float *series;
    int32_t n_proc, T, t0, N;
    const int32_t *xv; int32_t dx; /* (proc, lag) pairs */
    const int32_t *yv; int32_t dy;
    const int32_t *zv; int32_t dz;
    const int32_t *perm; /* nullable: x read at pi(i) */
    int32_t k, theiler;
} member_t;

static float coord(const member_t *m, const int32_t *vars, int32_t d, int32_t point)
{
    int32_t p = vars[2 * d], lag = vars[2 * d + 1];
    return m->series[(int64_t)p * m->T + (m->t0 + point - lag)];
}

static float sub_dist(const member_t *m, const int32_t *vars, int32_t nd, int32_t pi, int32_t pj)
{
    float r = -INFINITY;
    for (int32_t d = 0; d < nd; ++d) {
        float a = coord(m, vars, d, pi);
        float b = coord(m, vars, d, pj);
        float v = fabsf(a - b);
        if (v > r) r = v;
    }
    return r;
}

static int validate(const member_t *m)
{
    if (!m->series || m->n_proc < 1 || m->T < 1 || m->N < 1 || m->k < 1 || m->theiler < 0)
        return OR_EINVAL;
    if (m->dx < 1 || m->dy < 1 || m->dz < 0) return OR_EINVAL;
    if (m->t0 + m->N > m->T) return OR_EINVAL;
    const int32_t *vs[3] = {m->xv, m->yv, m->zv};
    const int32_t ds[3] = {m->dx, m->dy, m->dz};
    for (int s = 0; s < 3; ++s)
        for (int32_t d = 0; d < ds[s]; ++d) {
            int32_t p = vs[s][2 * d], lag = vs[s][2 * d + 1];
            if (p < 0 || p >= m->n_proc || lag < 0 || lag > m->t0) return OR_EINVAL;
        }
    /* every point needs at least k valid neighbours; the worst point is in
     * the middle of the series */
    int64_t worst = (int64_t)m->N - 1 - 2 * (int64_t)m->theiler;
    if (worst < m->k) return OR_EINVAL;
    if (m->perm)
        for (int32_t i = 0; i < m->N; ++i)
            if (m->perm[i] < 0 || m->perm[i] >= m->N) return OR_EINVAL;
    return OR_OK;
}

static int ksg_member(const member_t *m, const int64_t *q, int64_t *key_hi, uint64_t *key_lo,
                      double *i_key, double *i_plain, float *eps_out, int32_t *nxz_out,
                      int32_t *nyz_out, int32_t *nz_out)
{
    const int32_t N = m->N, k = m->k, w = m->theiler;
    float *best = (float *)malloc(sizeof(float) * (size_t)k);
    if (!best) return OR_ENOMEM;
    i128 K = 0;
    double plain_sum = 0.0;
    for (int32_t i = 0; i < N; ++i) {
        const int32_t xi = m->perm ? m->perm[i] : i;
        /* pass 1: k smallest joint distances, kept sorted ascending */
        for (int32_t a = 0; a < k; ++a) best[a] = INFINITY;
        for (int32_t j = 0; j < N; ++j) {
            int32_t gap = i > j ? i - j : j - i;
            if (j == i || gap <= w) continue;
            const int32_t xj = m->perm ? m->perm[j] : j;
            float dxv = sub_dist(m, m->xv, m->dx, xi, xj);
            float dyv = sub_dist(m, m->yv, m->dy, i, j);
            float dzv = sub_dist(m, m->zv, m->dz, i, j);
            float D = dxv;
            if (dyv > D) D = dyv;
            if (dzv > D) D = dzv;
            if (D < best[k - 1]) {
                int32_t a = k - 1;
                while (a > 0 && best[a - 1] > D) {
                    best[a] = best[a - 1];
                    --a;
                }
                best[a] = D;
            }
        }
        const float eps = best[k - 1];
        /* pass 2: strict range counts in the three marginal spaces */
        int32_t nxz = 0, nyz = 0, nz = 0;
        for (int32_t j = 0; j < N; ++j) {
            int32_t gap = i > j ? i - j : j - i;
            if (j == i || gap <= w) continue;
            const int32_t xj = m->perm ? m->perm[j] : j;
            float dxv = sub_dist(m, m->xv, m->dx, xi, xj);
            float dyv = sub_dist(m, m->yv, m->dy, i, j);
            float dzv = sub_dist(m, m->zv, m->dz, i, j);
            float dxz = dxv > dzv ? dxv : dzv;
            float dyz = dyv > dzv ? dyv : dzv;
            if (dxz < eps) ++nxz;
            if (dyz < eps) ++nyz;
            if (dzv < eps) ++nz;
        }
        if (eps_out) eps_out[i] = eps;
        if (nxz_out) nxz_out[i] = nxz;
        if (nyz_out) nyz_out[i] = nyz;
        if (nz_out) nz_out[i] = nz;
        K += (i128)q[nz + 1] - (i128)q[nxz + 1] - (i128)q[nyz + 1];
        plain_sum += oracle_digamma_plain(nz + 1) - oracle_digamma_plain(nxz + 1) -
                     oracle_digamma_plain(nyz + 1);
    }
    free(best);
    u128 uk = (u128)K;
    *key_hi = (int64_t)(uk >> 64);
    *key_lo = (uint64_t)uk;
    const double scale = 4503599627370496.0; /* 2^52 */
    const double psi_k = ldexp((double)q[k], -52);
    const double t = (double)K;
    const double d = scale * (double)N;
    *i_key = psi_k + t / d;
    *i_plain = oracle_digamma_plain(k) + plain_sum / (double)N;
    return OR_OK;
}

/* One estimate.  key2 = {hi, lo} of the 128-bit key (two's complement). */
int oracle_ksg_cmi(const float *series, int32_t n_proc, int32_t T, int32_t t0, int32_t N,
                   const int32_t *xv, int32_t dx, const int32_t *yv, int32_t dy,
                   const int32_t *zv, int32_t dz, const int32_t *perm, int32_t k,
                   int32_t theiler, int64_t *key2, double *i_key, double *i_plain,
                   float *eps, int32_t *n_xz, int32_t *n_yz, int32_t *n_z)
{
    member_t m = {series, n_proc, T, t0, N, xv, dx, yv, dy, zv, dz, perm, k, theiler};
    int st = validate(&m);
    if (st) return st;
    int64_t *q = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 2));
    if (!q) return OR_ENOMEM;
    oracle_digamma_q(N + 1, q, NULL);
    int64_t hi;
    uint64_t lo;
    st = ksg_member(&m, q, &hi, &lo, i_key, i_plain, eps, n_xz, n_yz, n_z);
    free(q);
    if (st) return st;
    key2[0] = hi;
    key2[1] = (int64_t)lo;
    return OR_OK;
}

/* Many members sharing Y and Z: member b uses X vars xv[b*dx*2 ...] and the
 * permutation perms[perm_idx[b]] (perm_idx < 0: identity).  Members are
 * independent, so they are spread over n_threads OpenMP threads; each member
 * is still the single-threaded brute force above. */
int oracle_ksg_batch(const float *series, int32_t n_proc, int32_t T, int32_t t0, int32_t N,
                     int32_t n_members, const int32_t *xv, int32_t dx, const int32_t *yv,
                     int32_t dy, const int32_t *zv, int32_t dz, const int32_t *perms,
                     int32_t n_perms, const int32_t *perm_idx, int32_t k, int32_t theiler,
                     int32_t n_threads, int64_t *key2, double *i_key, double *i_plain)
{
    if (n_members < 0) return OR_EINVAL;
    for (int32_t b = 0; b < n_members; ++b) {
        int32_t pidx = perm_idx ? perm_idx[b] : -1;
        if (pidx >= n_perms) return OR_EINVAL;
        member_t m = {series, n_proc, T, t0, N, xv + (size_t)b * dx * 2, dx, yv, dy, zv, dz,
                      pidx >= 0 ? perms + (size_t)pidx * N : NULL, k, theiler};
        int st = validate(&m);
        if (st) return st;
    }
    int64_t *q = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 2));
    if (!q) return OR_ENOMEM;
    oracle_digamma_q(N + 1, q, NULL);
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
    for (int32_t b = 0; b < n_members; ++b) {
        int32_t pidx = perm_idx ? perm_idx[b] : -1;
        member_t m = {series, n_proc, T, t0, N, xv + (size_t)b * dx * 2, dx, yv, dy, zv, dz,
                      pidx >= 0 ? perms + (size_t)pidx * N : NULL, k, theiler};
        int64_t hi;
        uint64_t lo;
        if (ksg_member(&m, q, &hi, &lo, &i_key[b], &i_plain[b], NULL, NULL, NULL, NULL)) {
#pragma omp atomic write
            failed = 1;
            continue;
        }
        key2[2 * b] = hi;
        key2[2 * b + 1] = (int64_t)lo;
    }
    free(q);
    return failed ? OR_ENOMEM : OR_OK;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
