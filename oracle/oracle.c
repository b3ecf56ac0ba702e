/*
 * oracle.c -- plain FP64 CPU oracle for the normalized Lomb-Scargle
 * periodogram (Townsend, "Fast Calculation of the Lomb-Scargle Periodogram
 * Using Graphics Processing Units").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is slow on purpose and shares nothing
 * with the CUDA library: no headers, no helpers, no tables.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * The product path never calls it.
 *
 * Every routine follows the textbook definition it cites, in FP64, with
 * Neumaier-compensated sums and OpenMP parallelism over frequencies only.
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC oracle.c -lm
 * (-ffp-contract=off keeps every a*b+c as two rounded operations, so the
 * FP32-phase model below is reproducible on x86-64 and aarch64 alike).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_BAD_ARG 1
#define OR_DEGENERATE 2
#define OR_NONFINITE 3
#define OR_NOMEM 4

static const double TWO_PI = 6.283185307179586476925286766559;

/* Neumaier's improvement of Kahan summation: running sum s, correction c. */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_value(const nsum *a) { return a->s + a->c; }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Pre-normalization of the data (Sec. 3, first paragraph; Sec. 4.2): the
 * series is shifted to zero mean and scaled to unit variance.  The paper does
 * not say which variance; the population form (divide by N_t) is used, so
 * that the largest attainable P_n is exactly N_t/2 and 2P_n/N_t is the
 * beta-distributed variable behind Eq. 3.  Two passes.
 */
int oracle_normalize(const double *X, int64_t n, double *x_out,
                     double *mean_out, double *var_out)
{
    if (n < 1 || !X || !x_out) return OR_BAD_ARG;
    nsum m = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
        if (!isfinite(X[j])) return OR_NONFINITE;
        nsum_add(&m, X[j]);
    }
    double mean = nsum_value(&m) / (double)n;
    nsum v = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
        double d = X[j] - mean;
        nsum_add(&v, d * d);
    }
    double var = nsum_value(&v) / (double)n;
    if (mean_out) *mean_out = mean;
    if (var_out) *var_out = var;
    if (!(var > 0.0)) return OR_DEGENERATE;
    double sd = sqrt(var);
    for (int64_t j = 0; j < n; ++j) x_out[j] = (X[j] - mean) / sd;
    return OR_OK;
}

static double min_time(const double *t, int64_t n)
{
    double m = t[0];
    for (int64_t j = 1; j < n; ++j)
        if (t[j] < m) m = t[j];
    return m;
}

/* f*t in turns, reduced to [-1/2, 1/2] by subtracting the nearest integer
 * (the range reduction of Sec. 4.3, here in FP64). */
static double reduced_turns(double f, double t)
{
    double p = f * t;
    return p - nearbyint(p);
}

/*
 * One frequency of the direct definition, Eq. 1 with tau from Eq. 2.
 * tt: times already shifted by the earliest sample (a shift of the time
 * origin leaves P_n unchanged, Eq. 1-2); x: normalized data.
 * Pass 1 gives omega*tau = (1/2) atan2(sum sin 2wt, sum cos 2wt); pass 2 the
 * four sums over w(t - tau).  A term whose denominator is <= N_t * 2^-40
 * (e.g. every sin w(t_j - tau) = 0 at the Nyquist frequency of an even grid)
 * is taken as zero: its numerator vanishes with it.
 */
static double direct_one(const double *tt, const double *x, int64_t n, double f)
{
    nsum s2 = {0, 0}, c2 = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
        double r = reduced_turns(f, tt[j]);
        nsum_add(&s2, sin(2.0 * TWO_PI * r));
        nsum_add(&c2, cos(2.0 * TWO_PI * r));
    }
    double wtau = 0.5 * atan2(nsum_value(&s2), nsum_value(&c2));
    nsum a = {0, 0}, b = {0, 0}, dc = {0, 0}, ds = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
        double r = reduced_turns(f, tt[j]);
        double arg = TWO_PI * r - wtau;
        double c = cos(arg), s = sin(arg);
        nsum_add(&a, x[j] * c);
        nsum_add(&b, x[j] * s);
        nsum_add(&dc, c * c);
        nsum_add(&ds, s * s);
    }
    double eps = (double)n * ldexp(1.0, -40);
    double A = nsum_value(&a), B = nsum_value(&b);
    double Dc = nsum_value(&dc), Ds = nsum_value(&ds);
    double P = 0.0;
    if (Dc > eps) P += A * A / Dc;
    if (Ds > eps) P += B * B / Ds;
    return 0.5 * P;
}

/* Shared loop: normalize, shift times, evaluate one routine per frequency. */
typedef double (*one_freq_fn)(const double *tt, const double *x, int64_t n, double f);

static int run_at(one_freq_fn fn, const double *t, const double *X, int64_t n,
                  const double *freqs, int64_t nf, double *P)
{
    if (n < 2 || nf < 0 || !t || !X || (nf > 0 && (!freqs || !P))) return OR_BAD_ARG;
    for (int64_t j = 0; j < n; ++j)
        if (!isfinite(t[j])) return OR_NONFINITE;
    for (int64_t k = 0; k < nf; ++k)
        if (!isfinite(freqs[k])) return OR_NONFINITE;
    double *x = (double *)malloc((size_t)n * sizeof(double));
    double *tt = (double *)malloc((size_t)n * sizeof(double));
    if (!x || !tt) { free(x); free(tt); return OR_NOMEM; }
    int st = oracle_normalize(X, n, x, NULL, NULL);
    if (st != OR_OK) { free(x); free(tt); return st; }
    double t0 = min_time(t, n);
    for (int64_t j = 0; j < n; ++j) tt[j] = t[j] - t0;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nf; ++k) P[k] = fn(tt, x, n, freqs[k]);
    free(x);
    free(tt);
    return OR_OK;
}

/* Eq. 1-2 at an arbitrary list of frequencies (cycles per time unit). */
int oracle_periodogram_at(const double *t, const double *X, int64_t n,
                          const double *freqs, int64_t nf, double *P)
{
    return run_at(direct_one, t, X, n, freqs, nf, P);
}

/* Eq. 1-2 on the uniform grid f_k = f0 + k*df, k = 0..nf-1 (Eq. 9 with the
 * grid origin made explicit: the paper's grid is f0 = df). */
int oracle_periodogram(const double *t, const double *X, int64_t n,
                       double f0, double df, int64_t nf, double *P)
{
    if (nf < 0) return OR_BAD_ARG;
    double *fr = (double *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(double));
    if (!fr) return OR_NOMEM;
    for (int64_t k = 0; k < nf; ++k) fr[k] = f0 + (double)k * df;
    int st = oracle_periodogram_at(t, X, n, fr, nf, P);
    free(fr);
    return st;
}

/*
 * The refactored single-pass form, Eq. 5-8: the five sums XC, XS, CC, SS, CS
 * over w*t_j (SS accumulated on its own here, not rebuilt from CC), then
 * tan 2wtau = 2CS/(CC - SS) (Eq. 6) and P_n from Eq. 5.  Algebraically equal
 * to Eq. 1-2; used to pin the oracle's two forms against each other.
 */
static double refac_one(const double *tt, const double *x, int64_t n, double f)
{
    nsum xc = {0, 0}, xs = {0, 0}, cc = {0, 0}, ss = {0, 0}, cs = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
        double arg = TWO_PI * reduced_turns(f, tt[j]);
        double c = cos(arg), s = sin(arg);
        nsum_add(&xc, x[j] * c);
        nsum_add(&xs, x[j] * s);
        nsum_add(&cc, c * c);
        nsum_add(&ss, s * s);
        nsum_add(&cs, c * s);
    }
    double XC = nsum_value(&xc), XS = nsum_value(&xs);
    double CC = nsum_value(&cc), SS = nsum_value(&ss), CS = nsum_value(&cs);
    double wtau = 0.5 * atan2(2.0 * CS, CC - SS);
    double ct = cos(wtau), st = sin(wtau);
    double num1 = ct * XC + st * XS, num2 = ct * XS - st * XC;
    double den1 = ct * ct * CC + 2.0 * ct * st * CS + st * st * SS;
    double den2 = ct * ct * SS - 2.0 * ct * st * CS + st * st * CC;
    double eps = (double)n * ldexp(1.0, -40);
    double P = 0.0;
    if (den1 > eps) P += num1 * num1 / den1;
    if (den2 > eps) P += num2 * num2 / den2;
    return 0.5 * P;
}

int oracle_periodogram_refac_at(const double *t, const double *X, int64_t n,
                                const double *freqs, int64_t nf, double *P)
{
    return run_at(refac_one, t, X, n, freqs, nf, P);
}

/*
 * Brute-force least-squares reading of the periodogram: half the drop in the
 * sum of squared residuals when the normalized data are fitted by
 * a cos(wt) + b sin(wt) (Lomb 1976; the chi^2 reduction that Eq. 1 equals).
 * The 2x2 normal equations are solved in long double and the residual is
 * formed explicitly.  Meant for tiny n.
 */
int oracle_lsq_power(const double *t, const double *X, int64_t n, double f, double *P)
{
    if (n < 2 || !t || !X || !P) return OR_BAD_ARG;
    double *x = (double *)malloc((size_t)n * sizeof(double));
    if (!x) return OR_NOMEM;
    int st = oracle_normalize(X, n, x, NULL, NULL);
    if (st != OR_OK) { free(x); return st; }
    const long double tp = 6.283185307179586476925286766559L;
    long double t0 = (long double)min_time(t, n);
    long double Scc = 0, Sss = 0, Scs = 0, Sxc = 0, Sxs = 0, Sxx = 0;
    for (int64_t j = 0; j < n; ++j) {
        long double p = (long double)f * ((long double)t[j] - t0);
        p -= nearbyintl(p);
        long double c = cosl(tp * p), s = sinl(tp * p);
        Scc += c * c; Sss += s * s; Scs += c * s;
        Sxc += x[j] * c; Sxs += x[j] * s; Sxx += (long double)x[j] * x[j];
    }
    long double a = 0, b = 0;
    long double det = Scc * Sss - Scs * Scs;
    long double tiny = (long double)n * 1e-24L;
    if (det > tiny * (Scc + Sss)) {
        a = (Sxc * Sss - Sxs * Scs) / det;
        b = (Sxs * Scc - Sxc * Scs) / det;
    } else if (Scc >= Sss && Scc > tiny) {
        a = Sxc / Scc; /* rank one: only the cosine column survives */
    } else if (Sss > tiny) {
        b = Sxs / Sss;
    }
    long double chi2 = 0;
    for (int64_t j = 0; j < n; ++j) {
        long double p = (long double)f * ((long double)t[j] - t0);
        p -= nearbyintl(p);
        long double r = x[j] - a * cosl(tp * p) - b * sinl(tp * p);
        chi2 += r * r;
    }
    *P = (double)(0.5L * (Sxx - chi2));
    free(x);
    return OR_OK;
}

/*
 * False-alarm probability, Eq. 3: Q = 1 - [1 - (1 - 2P/N_t)^((N_t-3)/2)]^N_f,
 * evaluated with log1p/expm1 so that Q near 0 and near 1 keep their digits.
 */
double oracle_fap(double P, int64_t n, double nf)
{
    double z = 2.0 * P / (double)n;
    if (z <= 0.0) return 1.0;
    double base = (z >= 1.0) ? 0.0 : exp(0.5 * (double)(n - 3) * log1p(-z));
    if (base >= 1.0) return 1.0;
    return -expm1(nf * log1p(-base));
}

/* Uniform grid of Eq. 9-11: df = 1/(F_over (t_N - t_1)), N_f = F_high F_over N_t / 2
 * (rounded down), f_0 = df.  Returns OR_BAD_ARG for a zero time span. */
int oracle_grid(double t_min, double t_max, int64_t n, double f_over, double f_high,
                double *f0, double *df, int64_t *nf)
{
    double span = t_max - t_min;
    if (!(span > 0.0) || !(f_over > 0.0) || !(f_high > 0.0) || n < 1) return OR_BAD_ARG;
    *df = 1.0 / (f_over * span);
    *f0 = *df;
    *nf = (int64_t)floor(f_high * f_over * (double)n / 2.0);
    return OR_OK;
}

/*
 * The paper's own FP32 phase (Sec. 4.3 and the kernel of Fig. 1): the
 * frequency and the time are single-precision numbers, their product is
 * rounded to single precision and the nearest integer is subtracted.  Here
 * f_k = (float)(f0 + k*df) and t = (float)(t_j - t_min); the reduced float
 * phase is then fed to FP64 trig and to Eq. 1-2, so that what remains of the
 * error is the phase rounding alone.  Evaluated at grid indices ks[].
 */
static double fp32phase_one(const double *tt, const double *x, int64_t n, float f32)
{
    nsum s2 = {0, 0}, c2 = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
        volatile float ft = f32 * (float)tt[j];
        float r = ft - rintf(ft);
        nsum_add(&s2, sin(2.0 * TWO_PI * (double)r));
        nsum_add(&c2, cos(2.0 * TWO_PI * (double)r));
    }
    double wtau = 0.5 * atan2(nsum_value(&s2), nsum_value(&c2));
    nsum a = {0, 0}, b = {0, 0}, dc = {0, 0}, ds = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
        volatile float ft = f32 * (float)tt[j];
        float r = ft - rintf(ft);
        double arg = TWO_PI * (double)r - wtau;
        double c = cos(arg), s = sin(arg);
        nsum_add(&a, x[j] * c);
        nsum_add(&b, x[j] * s);
        nsum_add(&dc, c * c);
        nsum_add(&ds, s * s);
    }
    double eps = (double)n * ldexp(1.0, -40);
    double A = nsum_value(&a), B = nsum_value(&b);
    double Dc = nsum_value(&dc), Ds = nsum_value(&ds);
    double P = 0.0;
    if (Dc > eps) P += A * A / Dc;
    if (Ds > eps) P += B * B / Ds;
    return 0.5 * P;
}

int oracle_periodogram_fp32phase_at(const double *t, const double *X, int64_t n,
                                    double f0, double df, const int64_t *ks,
                                    int64_t nk, double *P)
{
    if (n < 2 || nk < 0 || !t || !X || (nk > 0 && (!ks || !P))) return OR_BAD_ARG;
    double *x = (double *)malloc((size_t)n * sizeof(double));
    double *tt = (double *)malloc((size_t)n * sizeof(double));
    if (!x || !tt) { free(x); free(tt); return OR_NOMEM; }
    int st = oracle_normalize(X, n, x, NULL, NULL);
    if (st != OR_OK) { free(x); free(tt); return st; }
    double t0 = min_time(t, n);
    for (int64_t j = 0; j < n; ++j) tt[j] = t[j] - t0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nk; ++i) {
        double fk = f0 + (double)ks[i] * df;
        P[i] = fp32phase_one(tt, x, n, (float)fk);
    }
    free(x);
    free(tt);
    return OR_OK;
}

/*
 * Spectral window |sum_j exp(2 pi i f t_j)|^2 / N_t^2 at the given
 * frequencies: the periodogram machinery with X = 1 and no tau, used for the
 * sampling-pattern features.
 */
int oracle_window_at(const double *t, int64_t n, const double *freqs, int64_t nf, double *W)
{
    if (n < 1 || nf < 0 || !t || (nf > 0 && (!freqs || !W))) return OR_BAD_ARG;
    double t0 = min_time(t, n);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nf; ++k) {
        nsum re = {0, 0}, im = {0, 0};
        for (int64_t j = 0; j < n; ++j) {
            double arg = TWO_PI * reduced_turns(freqs[k], t[j] - t0);
            nsum_add(&re, cos(arg));
            nsum_add(&im, sin(arg));
        }
        double R = nsum_value(&re), I = nsum_value(&im);
        W[k] = (R * R + I * I) / ((double)n * (double)n);
    }
    return OR_OK;
}

/*
 * Philox-4x32-10 (Salmon, Moraes, Dror & Shaw 2011, "Parallel random
 * numbers: as easy as 1, 2, 3"): ten rounds of two 32x32->64 multiplies and
 * a Feistel-like swap, with a Weyl-sequence key schedule between rounds.
 * Pinned word for word against the authors' published known-answer vectors
 * (tests/golden/philox4x32_10_kat.txt); the GPU generator is compared with
 * this one bit for bit.
 */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Gaussian noise for Monte-Carlo periodograms (Sec. 6.2): sample j of
 * realization `real` of curve `curve` takes Philox block j/4 with counter
 * (j/4, curve, real, 0) and key (seed low word, seed high word).  Each 32-bit
 * word w maps to the uniform u = (2*(w >> 9) + 1) * 2^-24 in (0, 1), and the
 * Box-Muller transform (Box & Muller 1958) turns the pairs (u0, u1) and
 * (u2, u3) into four standard normals: sqrt(-2 ln u_a) * (cos, sin)(2 pi u_b).
 */
void oracle_noise(uint64_t seed, uint32_t curve, uint32_t real, int64_t n, double *x)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t b = 0; b * 4 < n; ++b) {
        uint32_t ctr[4] = {(uint32_t)b, curve, real, 0u}, w[4];
        oracle_philox4x32_10(ctr, key, w);
        double u[4];
        for (int i = 0; i < 4; ++i) u[i] = (double)(2u * (w[i] >> 9) + 1u) * ldexp(1.0, -24);
        double z[4];
        double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
        z[0] = r0 * cos(TWO_PI * u[1]);
        z[1] = r0 * sin(TWO_PI * u[1]);
        z[2] = r1 * cos(TWO_PI * u[3]);
        z[3] = r1 * sin(TWO_PI * u[3]);
        for (int i = 0; i < 4 && b * 4 + i < n; ++i) x[b * 4 + i] = z[i];
    }
}

/*
 * Floating-mean ("generalized") periodogram, the extension Sec. 6.3 points at
 * (Zechmeister & Kuerster 2009; Shrager 2001): the sinusoid is fitted together
 * with an offset, with weights w_j = (1/dy_j^2) / sum(1/dy^2) (w_j = 1/N_t
 * without errors).  With Y = sum w y, C = sum w cos wt, S = sum w sin wt and
 * YC = sum w y cos - Y C, YS = sum w y sin - Y S, CC = sum w cos^2 - C^2,
 * SS = sum w sin^2 - S^2, CS = sum w cos sin - C S, YY = sum w y^2 - Y^2 and
 * D = CC SS - CS^2, the fraction of the weighted variance that the fit removes
 * is p = (SS YC^2 + CC YS^2 - 2 CS YC YS) / (YY D), in [0, 1].  It is reported
 * as P = (N_t / 2) p, the scale of Eq. 1's P_n: at frequencies where C = S = 0
 * with equal weights the two periodograms coincide.
 *
 * Rank-deficient frequencies (reading): when cos and sin, once centred, are
 * linearly dependent on the samples (D <= 2^-40, e.g. the Nyquist frequency
 * of an even grid, where every sin vanishes), the fit is the projection on the
 * one remaining direction, p = (YC^2 + YS^2) / (YY (CC + SS)); when both vanish
 * (CC + SS <= 2^-40, e.g. f = 0) p = 0.  This is what the least-squares fit
 * itself gives (the data vector (YC, YS) always lies in the range of the 2x2
 * matrix [[CC, CS], [CS, SS]]), and it parallels the classic periodogram's
 * treatment of a vanishing denominator.
 */
static int gls_weights(const double *dy, int64_t n, double *w)
{
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (dy) {
            if (!isfinite(dy[j]) || !(dy[j] > 0.0)) return OR_BAD_ARG;
            w[j] = 1.0 / (dy[j] * dy[j]);
        } else {
            w[j] = 1.0;
        }
        s += w[j];
    }
    for (int64_t j = 0; j < n; ++j) w[j] /= s;
    return OR_OK;
}

int oracle_gls_at(const double *t, const double *X, const double *dy, int64_t n,
                  const double *freqs, int64_t nf, double *P)
{
    if (n < 3 || nf < 0 || !t || !X || (nf > 0 && (!freqs || !P))) return OR_BAD_ARG;
    for (int64_t j = 0; j < n; ++j)
        if (!isfinite(t[j]) || !isfinite(X[j])) return OR_NONFINITE;
    for (int64_t k = 0; k < nf; ++k)
        if (!isfinite(freqs[k])) return OR_NONFINITE;
    double *w = (double *)malloc((size_t)n * sizeof(double));
    double *tt = (double *)malloc((size_t)n * sizeof(double));
    if (!w || !tt) { free(w); free(tt); return OR_NOMEM; }
    int st = gls_weights(dy, n, w);
    if (st != OR_OK) { free(w); free(tt); return st; }
    double t0 = min_time(t, n);
    for (int64_t j = 0; j < n; ++j) tt[j] = t[j] - t0;
    nsum ys = {0, 0}, yys = {0, 0};
    for (int64_t j = 0; j < n; ++j) { nsum_add(&ys, w[j] * X[j]); nsum_add(&yys, w[j] * X[j] * X[j]); }
    const double Y = nsum_value(&ys);
    /* YY in two passes: sum w (y - Y)^2 */
    nsum yv = {0, 0};
    for (int64_t j = 0; j < n; ++j) { double d = X[j] - Y; nsum_add(&yv, w[j] * d * d); }
    const double YY = nsum_value(&yv);
    if (!(YY > 0.0)) { free(w); free(tt); return OR_DEGENERATE; }
    const double thr = ldexp(1.0, -40);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nf; ++k) {
        nsum c = {0, 0}, s = {0, 0}, yc = {0, 0}, ysn = {0, 0}, cc = {0, 0}, ss = {0, 0}, cs = {0, 0};
        for (int64_t j = 0; j < n; ++j) {
            double arg = TWO_PI * reduced_turns(freqs[k], tt[j]);
            double co = cos(arg), si = sin(arg);
            nsum_add(&c, w[j] * co);
            nsum_add(&s, w[j] * si);
            nsum_add(&yc, w[j] * X[j] * co);
            nsum_add(&ysn, w[j] * X[j] * si);
            nsum_add(&cc, w[j] * co * co);
            nsum_add(&ss, w[j] * si * si);
            nsum_add(&cs, w[j] * co * si);
        }
        double C = nsum_value(&c), S = nsum_value(&s);
        double YC = nsum_value(&yc) - Y * C, YS = nsum_value(&ysn) - Y * S;
        double CC = nsum_value(&cc) - C * C, SS = nsum_value(&ss) - S * S, CS = nsum_value(&cs) - C * S;
        double D = CC * SS - CS * CS;
        double p = 0.0;
        if (D > thr)
            p = (SS * YC * YC + CC * YS * YS - 2.0 * CS * YC * YS) / (YY * D);
        else if (CC + SS > thr)
            p = (YC * YC + YS * YS) / (YY * (CC + SS));
        P[k] = 0.5 * (double)n * p;
    }
    free(w);
    free(tt);
    return OR_OK;
}

/*
 * Brute-force reading of the floating-mean periodogram, independent of the
 * closed form above: the weighted least-squares fit of the data by the span of
 * {1, cos wt, sin wt}, found by modified Gram-Schmidt (two sweeps) in the
 * weighted inner product, in long double; a basis vector whose remainder has
 * squared weighted length at most 2^-60 (length at most 2^-30) adds nothing
 * (rank-deficient frequencies).
 * P = (N_t/2) (1 - chi2_fit / chi2_offset).  Tiny n only.
 */
int oracle_gls_lsq(const double *t, const double *X, const double *dy, int64_t n, double f, double *P)
{
    if (n < 3 || !t || !X || !P) return OR_BAD_ARG;
    double *w = (double *)malloc((size_t)n * sizeof(double));
    long double *Q = (long double *)malloc((size_t)(4 * n) * sizeof(long double));
    if (!w || !Q) { free(w); free(Q); return OR_NOMEM; }
    int st = gls_weights(dy, n, w);
    if (st != OR_OK) { free(w); free(Q); return st; }
    const long double tp = 6.283185307179586476925286766559L;
    long double t0 = (long double)min_time(t, n);
    long double *r = Q + 3 * n; /* residual of the data */
    for (int64_t j = 0; j < n; ++j) {
        long double ph = (long double)f * ((long double)t[j] - t0);
        ph -= nearbyintl(ph);
        Q[j] = 1.0L;
        Q[n + j] = cosl(tp * ph);
        Q[2 * n + j] = sinl(tp * ph);
        r[j] = X[j];
    }
    int kept[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        long double *qa = Q + a * n;
        for (int sweep = 0; sweep < 2; ++sweep)
            for (int b = 0; b < a; ++b) {
                if (!kept[b]) continue;
                long double *qb = Q + b * n, d = 0;
                for (int64_t j = 0; j < n; ++j) d += w[j] * qa[j] * qb[j];
                for (int64_t j = 0; j < n; ++j) qa[j] -= d * qb[j];
            }
        long double len = 0;
        for (int64_t j = 0; j < n; ++j) len += w[j] * qa[j] * qa[j];
        /* dependent on the earlier ones (or nothing but rounding: the basis
         * vectors have weighted length <= 1, so the test is absolute) */
        if (!(len > 0x1p-60L)) continue;
        long double inv = 1.0L / sqrtl(len);
        for (int64_t j = 0; j < n; ++j) qa[j] *= inv;
        kept[a] = 1;
    }
    /* chi2 of the offset-only fit (first basis vector) and of the full fit */
    long double chi0 = 0, chi = 0;
    for (int a = 0; a < 3; ++a) {
        if (!kept[a]) continue;
        long double *qa = Q + a * n, d = 0;
        for (int64_t j = 0; j < n; ++j) d += w[j] * r[j] * qa[j];
        for (int64_t j = 0; j < n; ++j) r[j] -= d * qa[j];
        if (a == 0) for (int64_t j = 0; j < n; ++j) chi0 += w[j] * r[j] * r[j];
    }
    for (int64_t j = 0; j < n; ++j) chi += w[j] * r[j] * r[j];
    *P = (double)(0.5L * (long double)n * (1.0L - chi / chi0));
    free(w);
    free(Q);
    return OR_OK;
}
