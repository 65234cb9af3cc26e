/*
 * Plain CPU Monte Carlo oracle for the discretized amplitude A_N^(p)(a,b;T).
 *
 * TEST INFRASTRUCTURE ONLY: called from tests/, __graft_entry__.smoke() and
 * bench.py's CPU baseline through oracle/mc.py; the product library never
 * links it.  It shares no code with the CUDA path.
 *
 * What it computes, one sample at a time, in double precision:
 *
 *  - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 *    easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies by
 *    M0 = 0xD2511F53 and M1 = 0xCD9E8D57 with the Weyl key bumps
 *    W0 = 0x9E3779B9, W1 = 0xBB67AE85 between rounds.
 *    Key = (seed lo32, seed hi32); counter = (call t, instance, sample lo32,
 *    sample hi32).
 *  - Box-Muller (Sec. 4.1): r = sqrt(-2 ln u1), theta = 2 pi u2,
 *    z_{2t} = r cos theta, z_{2t+1} = r sin theta, both branches used.
 *    53-bit uniforms u = ((w0 * 2^21 + (w1 >> 11)) + 0.5) * 2^-53 from
 *    (w0,w1) and (w2,w3): normal j is branch j & 1 of call j >> 1.
 *    24-bit uniforms u = ((w >> 8) + 0.5) * 2^-24, rounded in float exactly
 *    as a float kernel forms them, four normals per call: with j' = j + 1,
 *    normal j is branch j' & 1 of the pair (u1, u2) = (w0, w1) for
 *    (j' & 3) < 2 and (w2, w3) otherwise, of call j' >> 2.
 *  - Bisection (Sec. 4.1): for level n = 1..s and i = 0..2^(n-1)-1 the normal
 *    with heap index j = 2^(n-1) - 1 + i places
 *      q[(2i+1) 2^(s-n)] = (q[i 2^(s-n+1)] + q[(i+1) 2^(s-n+1)]) / 2
 *                          + wf * sigma_n * z_j,
 *    sigma_n^2 = T / 2^(n+1), the exact Brownian-bridge variance at the
 *    midpoint; q[0] = a, q[N] = b.  wf = 1 samples the exact bridge; wf != 1
 *    (wf = sqrt 2 is the paper's literal width sqrt(T/2^n)) adds the Gaussian
 *    density ratio log wf + z^2 (1 - wf^2) / 2 of every midpoint at levels
 *    <= n to the level-n log-weight, which keeps the estimator unbiased.
 *  - The level-n log-weight (Eq. SNp with the kinetic term and the
 *    normalisation (2 pi eps)^(-N/2) cancelled against the bridge density):
 *      w_n = - eps_n sum_{k=0}^{2^n - 1} W_p(x_k, xb_k; eps_n),
 *    eps_n = T / 2^n, on the level-n subpath q[i 2^(s-n)] (Sec. 4.1),
 *    x_k = (q_k + q_{k+1})/2, xb_k = (q_{k+1} - q_k)/2, and W_p evaluated
 *    directly from its coefficients (Eq. ansatz truncated at m <= p-1):
 *      W_p = sum_{m<p} sum_{k<=m} c_{m,k}(z) eps^(m-k) xb^(2k),
 *    z = x or z = tanh(alpha x).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int p;              /* level of the effective action */
    int ring;           /* 0: z = x, 1: z = tanh(alpha x) */
    double alpha;
    const double *coef; /* concatenated polynomial coefficients, lowest first */
    const int *off;     /* c_{m,k} starts at coef[off[m*p+k]] */
    const int *len;     /* and has len[m*p+k] coefficients */
} oracle_wp;

/* ---------------------------------------------------------------- Philox */

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k);
        k[0] += 0x9E3779B9u;
        k[1] += 0xBB67AE85u;
    }
    memcpy(out, c, sizeof c);
}

void oracle_philox_words(uint64_t seed, uint32_t instance, uint64_t sample,
                         uint32_t call, uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {call, instance, (uint32_t)sample, (uint32_t)(sample >> 32)};
    oracle_philox(ctr, key, out);
}

/* ----------------------------------------------------------- Box-Muller */

static double u24(uint32_t w)
{
    volatile float f = (float)(w >> 8) + 0.5f;  /* rounded in float */
    return (double)f * 0x1p-24;
}

static const double TWO_PI = 6.283185307179586476925286766559;

/* normal number j of the sample's stream (both Box-Muller branches) */
static double normal_j(uint64_t seed, uint32_t instance, uint64_t sample, int64_t j, int bits)
{
    uint32_t w[4];
    double u1, u2;
    int branch;
    if (bits == 53) {
        oracle_philox_words(seed, instance, sample, (uint32_t)(j >> 1), w);
        uint64_t a = ((uint64_t)w[0] << 21) | (w[1] >> 11);
        uint64_t b = ((uint64_t)w[2] << 21) | (w[3] >> 11);
        u1 = ((double)a + 0.5) * 0x1p-53;
        u2 = ((double)b + 0.5) * 0x1p-53;
        branch = (int)(j & 1);
    } else {
        int64_t jp = j + 1;
        oracle_philox_words(seed, instance, sample, (uint32_t)(jp >> 2), w);
        int pr = (int)((jp >> 1) & 1);
        u1 = u24(w[2 * pr]);
        u2 = u24(w[2 * pr + 1]);
        branch = (int)(jp & 1);
    }
    double r = sqrt(-2.0 * log(u1));
    double th = TWO_PI * u2;
    return branch ? r * sin(th) : r * cos(th);
}

void oracle_normals(uint64_t seed, uint32_t instance, uint64_t sample, int64_t n,
                    int bits, double *z)
{
    for (int64_t j = 0; j < n; ++j) z[j] = normal_j(seed, instance, sample, j, bits);
}

/* ------------------------------------------------------------------ W_p */

static double poly_at(const double *c, int n, double z)
{
    double acc = 0.0;
    for (int i = n - 1; i >= 0; --i) acc = acc * z + c[i];
    return acc;
}

double oracle_Wp(const oracle_wp *W, double x, double xb, double eps)
{
    double z = (W->ring == 0) ? x : tanh(W->alpha * x);
    double tot = 0.0;
    for (int m = 0; m < W->p; ++m)
        for (int k = 0; k <= m; ++k) {
            int id = m * W->p + k;
            if (W->len[id] == 0) continue;
            double c = poly_at(W->coef + W->off[id], W->len[id], z);
            tot += c * pow(eps, (double)(m - k)) * pow(xb, (double)(2 * k));
        }
    return tot;
}

/* ------------------------------------------------------------- sampling */

/* path points of one sample, q[0..2^s] */
void oracle_path(uint64_t seed, uint32_t instance, uint64_t sample, int s,
                 double a, double b, double T, int bits, double wf, double *q,
                 double *corr /* s entries, may be NULL */)
{
    int64_t N = (int64_t)1 << s;
    q[0] = a;
    q[N] = b;
    double c = 0.0;
    for (int n = 1; n <= s; ++n) {
        double sig = sqrt(T / (double)((int64_t)1 << (n + 1)));
        int64_t h = (int64_t)1 << (s - n);
        for (int64_t i = 0; i < ((int64_t)1 << (n - 1)); ++i) {
            int64_t j = ((int64_t)1 << (n - 1)) - 1 + i;
            double z = normal_j(seed, instance, sample, j, bits);
            int64_t idx = (2 * i + 1) * h;
            q[idx] = 0.5 * (q[idx - h] + q[idx + h]) + wf * sig * z;
            if (wf != 1.0) c += log(wf) + 0.5 * z * z * (1.0 - wf * wf);
        }
        if (corr) corr[n - 1] = c;
    }
}

/* sum over the (m,k) terms of |c_{m,k}(z) eps^(m-k) xb^(2k)|: the size of the
   numbers W_p is summed from, which bounds the rounding error of any order of
   evaluating it (a condition measure, not part of the estimate) */
double oracle_Wp_abs(const oracle_wp *W, double x, double xb, double eps)
{
    double z = (W->ring == 0) ? x : tanh(W->alpha * x);
    double tot = 0.0;
    for (int m = 0; m < W->p; ++m)
        for (int k = 0; k <= m; ++k) {
            int id = m * W->p + k;
            const double *c = W->coef + W->off[id];
            double zp = 1.0;
            for (int i = 0; i < W->len[id]; ++i) {
                tot += fabs(c[i] * zp) * pow(eps, (double)(m - k)) * pow(xb, (double)(2 * k));
                zp *= z;
            }
        }
    return tot;
}

/* log-weight of level n (1..s) for a given path */
static double level_logweight(const oracle_wp *W, const double *q, int s, int n, double T)
{
    double eps = T / (double)((int64_t)1 << n);
    int64_t st = (int64_t)1 << (s - n);
    double sum = 0.0;
    for (int64_t k = 0; k < ((int64_t)1 << n); ++k) {
        double ql = q[k * st], qr = q[(k + 1) * st];
        sum += oracle_Wp(W, 0.5 * (ql + qr), 0.5 * (qr - ql), eps);
    }
    return -eps * sum;
}

/* the level-0 log-weight, -T W_p((a+b)/2, (b-a)/2; T), the same for every sample */
double oracle_level0(const oracle_wp *W, double a, double b, double T)
{
    return -T * oracle_Wp(W, 0.5 * (a + b), 0.5 * (b - a), T);
}

/* eps_n sum_k |W_p terms| on the level-n subpath: the condition scale of w_n */
static double level_abs(const oracle_wp *W, const double *q, int s, int n, double T)
{
    double eps = T / (double)((int64_t)1 << n);
    int64_t st = (int64_t)1 << (s - n);
    double sum = 0.0;
    for (int64_t k = 0; k < ((int64_t)1 << n); ++k) {
        double ql = q[k * st], qr = q[(k + 1) * st];
        sum += oracle_Wp_abs(W, 0.5 * (ql + qr), 0.5 * (qr - ql), eps);
    }
    return eps * sum;
}

/* condition scales a[(i - sample0) * s + (n - 1)] of the same samples as
   oracle_logweights (plain loop, one thread) */
void oracle_logweights_abs(const oracle_wp *W, double a, double b, double T, int s,
                           uint64_t seed, uint32_t instance, int64_t sample0, int64_t nsamples,
                           int bits, double wf, double *out)
{
    if (s < 1 || nsamples <= 0) return;
    int64_t N = (int64_t)1 << s;
    double *q = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    for (int64_t i = 0; i < nsamples; ++i) {
        oracle_path(seed, instance, (uint64_t)(sample0 + i), s, a, b, T, bits, wf, q, NULL);
        for (int n = 1; n <= s; ++n) out[i * s + (n - 1)] = level_abs(W, q, s, n, T);
    }
    free(q);
}

/*
 * Per-sample log-weights w[(i - sample0) * s + (n - 1)] for samples
 * sample0 .. sample0 + nsamples - 1 and levels n = 1..s.
 * Returns the number of threads used.
 */
int oracle_logweights(const oracle_wp *W, double a, double b, double T, int s,
                      uint64_t seed, uint32_t instance, int64_t sample0, int64_t nsamples,
                      int bits, double wf, int nthreads, double *w)
{
    int used = 1;
    if (s < 1 || nsamples <= 0) return used;
    int64_t N = (int64_t)1 << s;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
#pragma omp single
        used = omp_get_num_threads();
#else
    (void)nthreads;
    {
#endif
        double *q = (double *)malloc(sizeof(double) * (size_t)(N + 1));
        double *corr = (double *)malloc(sizeof(double) * (size_t)s);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t i = 0; i < nsamples; ++i) {
            oracle_path(seed, instance, (uint64_t)(sample0 + i), s, a, b, T, bits, wf, q, corr);
            for (int n = 1; n <= s; ++n)
                w[i * s + (n - 1)] = level_logweight(W, q, s, n, T) + corr[n - 1];
        }
        free(q);
        free(corr);
    }
    return used;
}
