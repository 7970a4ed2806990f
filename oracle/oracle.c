/*
 * CPU FP64 oracle for the parity-projected (M = 2) matrix-P estimator of the
 * total-count distribution of Gaussian boson sampling, with the positive-P
 * estimator beside it (Drummond, Dellios, Reid, arXiv:2503.12749).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  It shares no code, header, table or helper
 * with the CUDA library; only tests/, the smoke check and the bench's CPU
 * baseline may load it.
 *
 * Every step is written the way the paper states it, in its order:
 *   1. counter-based normals: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw,
 *      "Parallel random numbers: as easy as 1, 2, 3", SC'11) + Box-Muller;
 *   2. squeezed-vacuum input amplitudes on the real line ("Applications to
 *      GBS": xi(alpha) = prod_j C_j exp(-alpha_j^2 coth(r_j)/2)); the +P
 *      density xi(alpha) xi(beta) exp(alpha.beta) is a bivariate Gaussian per
 *      mode, sampled through its eigen-decomposition;
 *   3. propagation alpha' = t alpha, beta' = t* beta, occupations
 *      n'_j = alpha'_j beta'_j, n_S = sum_j n'_j, input total n = alpha.beta;
 *   4. projector (Eq. c-number-variable with g_0 of the M = 2 parity case):
 *      G(m) = g_0(n_S, m) n_S^m e^{-n_S} / m!;  +P: g_0 = 1 (Eq.
 *      phase_space_projector);
 *   5. generating function sum_m z^m G(m) = cosh(n + (z-1) n_S) / cosh(n)
 *      (matrix-P) and exp((z-1) n_S) (+P), evaluated at z_k = e^{2 pi i k/K1};
 *   6. sub-ensemble means (Appendix A: N_R sub-ensembles), inverse DFT to
 *      P_r(m), mean over r and sampling error std_r / sqrt(N_R).
 * Sample e belongs to sub-ensemble e mod N_R.
 *
 * Threads: only independent per-sample or per-output work is spread across
 * OpenMP threads; every sum over samples runs in one fixed order.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* 1. Philox-4x32-10 (Salmon et al., SC'11, Sec. 3 / Random123 definition)   */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_W1 = 0xBB67AE85u; /* sqrt(3) - 1 */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) with 53 bits from two 32-bit words: 27 high bits of the
 * first, 26 high bits of the second, offset by half a unit so 0 never occurs. */
static double orc_uniform53(uint32_t a, uint32_t b)
{
    double hi = (double)(a >> 5);
    double lo = (double)(b >> 6);
    return (hi * 67108864.0 + lo + 0.5) * (1.0 / 9007199254740992.0);
}

/* Two standard normals for sample e and input mode j.  Counter (e_lo, e_hi,
 * j, 0), key (seed_lo, seed_hi); Box-Muller on the two 53-bit uniforms. */
void orc_normals(uint64_t seed, uint64_t e, uint32_t j, double *w1, double *w2)
{
    uint32_t ctr[4] = {(uint32_t)e, (uint32_t)(e >> 32), j, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u1 = orc_uniform53(x[0], x[1]);
    double u2 = orc_uniform53(x[2], x[3]);
    double rho = sqrt(-2.0 * log(u1));
    *w1 = rho * cos(2.0 * ORC_PI * u2);
    *w2 = rho * sin(2.0 * ORC_PI * u2);
}

/* ------------------------------------------------------------------------ */
/* 2. Input amplitudes ("Applications to GBS")                               */
/* ------------------------------------------------------------------------ */
/* Per mode the +P density of a squeezed vacuum, xi(a) xi(b) e^{ab} on the
 * real plane, is Gaussian with precision matrix [[coth r, -1], [-1, coth r]],
 * i.e. covariance [[sinh r cosh r, sinh^2 r], [sinh^2 r, sinh r cosh r]].
 * Its eigenvectors are (1, 1)/sqrt2 and (1, -1)/sqrt2 with eigenvalues
 * s+ = sinh r e^{r} and s- = sinh r e^{-r}.  Returns n = sum_j alpha_j beta_j. */
double orc_sample_inputs(int N, const double *r, uint64_t seed, uint64_t e,
                         double *alpha, double *beta)
{
    double n = 0.0;
    for (int j = 0; j < N; ++j) {
        double w1, w2;
        orc_normals(seed, e, (uint32_t)j, &w1, &w2);
        double sp = sinh(r[j]) * exp(r[j]);
        double sm = sinh(r[j]) * exp(-r[j]);
        alpha[j] = (sqrt(sp) * w1 + sqrt(sm) * w2) / sqrt(2.0);
        beta[j] = (sqrt(sp) * w1 - sqrt(sm) * w2) / sqrt(2.0);
        n += alpha[j] * beta[j];
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* 3. Propagation through the network (alpha' = t alpha, beta' = t* beta)     */
/* ------------------------------------------------------------------------ */
/* T is M x N complex, row-major, stored as interleaved (re, im) doubles. */
cplx orc_propagate(int N, int M, const double *T, const double *alpha, const double *beta)
{
    cplx nS = 0.0;
    for (int i = 0; i < M; ++i) {
        cplx ap = 0.0, bp = 0.0;
        for (int j = 0; j < N; ++j) {
            cplx t = T[2 * ((size_t)i * N + j)] + I * T[2 * ((size_t)i * N + j) + 1];
            ap += t * alpha[j];
            bp += conj(t) * beta[j];
        }
        nS += ap * bp; /* n'_i = alpha'_i beta'_i */
    }
    return nS;
}

/* Per-sample observables for samples e0 .. e0+E-1: n[E], nS[2E] (re, im). */
int orc_samples(int N, int M, const double *T, const double *r, uint64_t seed,
                uint64_t e0, int64_t E, double *n, double *nS, int threads)
{
    if (N <= 0 || M <= 0 || E < 0) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    int failed = 0;
#pragma omp parallel
    {
        double *alpha = (double *)malloc(sizeof(double) * (size_t)N);
        double *beta = (double *)malloc(sizeof(double) * (size_t)N);
        if (!alpha || !beta) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t i = 0; i < E; ++i) {
                n[i] = orc_sample_inputs(N, r, seed, e0 + (uint64_t)i, alpha, beta);
                cplx s = orc_propagate(N, M, T, alpha, beta);
                nS[2 * i] = creal(s);
                nS[2 * i + 1] = cimag(s);
            }
        }
        free(alpha);
        free(beta);
    }
    return failed ? -2 : 0;
}

/* Optional: the propagated amplitudes of one sample, for element checks. */
void orc_sample_amplitudes(int N, int M, const double *T, const double *r, uint64_t seed,
                           uint64_t e, double *alpha, double *beta, double *alpha_p,
                           double *beta_p)
{
    orc_sample_inputs(N, r, seed, e, alpha, beta);
    for (int i = 0; i < M; ++i) {
        cplx ap = 0.0, bp = 0.0;
        for (int j = 0; j < N; ++j) {
            cplx t = T[2 * ((size_t)i * N + j)] + I * T[2 * ((size_t)i * N + j) + 1];
            ap += t * alpha[j];
            bp += conj(t) * beta[j];
        }
        alpha_p[2 * i] = creal(ap);
        alpha_p[2 * i + 1] = cimag(ap);
        beta_p[2 * i] = creal(bp);
        beta_p[2 * i + 1] = cimag(bp);
    }
}

/* ------------------------------------------------------------------------ */
/* 4. Direct per-bin projector (Eq. c-number-variable, M = 2 parity)         */
/* ------------------------------------------------------------------------ */
/* Summed over patterns with sum_i c_i = m, prod_i n_i^{c_i} e^{-n_i}/c_i!
 * becomes n_S^m e^{-n_S}/m! (multinomial theorem), so
 *   G_mP(m) = g_0(n_S, m) n_S^m e^{-n_S}/m!,
 *   g_0(n_S, m) = (1 + pi_m e^{2(n_S - n)}) / (1 + e^{-2n}),  pi_m = (-1)^m,
 *   G_+P(m) = n_S^m e^{-n_S}/m!.
 * Evaluated in log space: with L = m Log(n_S) - lgamma(m+1) and the common
 * factor e^{n - |n|} applied to numerator and denominator,
 *   G_mP(m) = [e^{L - n_S + c} + pi_m e^{L + n_S - 2n + c}] / (1 + e^{-2|n|}),
 *   c = n - |n|.
 * Outputs (re, im) pairs for m = m0 .. m0+count-1. */
void orc_projector_direct(double n, double nS_re, double nS_im, int m0, int count,
                          double *G_mP, double *G_pP)
{
    cplx nS = nS_re + I * nS_im;
    double c = n - fabs(n);
    double den = 1.0 + exp(-2.0 * fabs(n));
    for (int q = 0; q < count; ++q) {
        int m = m0 + q;
        cplx gm, gp;
        if (nS == 0.0) {
            /* n_S^m = 0 for m > 0; 0^0 = 1 */
            if (m == 0) {
                gm = (exp(c) + exp(-2.0 * n + c)) / den;
                gp = 1.0;
            } else {
                gm = 0.0;
                gp = 0.0;
            }
        } else {
            cplx L = (double)m * clog(nS) - lgamma((double)m + 1.0);
            double pim = (m % 2 == 0) ? 1.0 : -1.0;
            gm = (cexp(L - nS + c) + pim * cexp(L + nS - 2.0 * n + c)) / den;
            gp = cexp(L - nS);
        }
        if (G_mP) { G_mP[2 * q] = creal(gm); G_mP[2 * q + 1] = cimag(gm); }
        if (G_pP) { G_pP[2 * q] = creal(gp); G_pP[2 * q + 1] = cimag(gp); }
    }
}

/* ------------------------------------------------------------------------ */
/* 5. Generating functions at the K1 roots of unity                          */
/* ------------------------------------------------------------------------ */
/* sum_m z^m G_mP(m) = [cosh(z n_S) cosh(n - n_S) + sinh(z n_S) sinh(n - n_S)]
 *                     / cosh(n) = cosh(n + (z - 1) n_S) / cosh(n),
 * sum_m z^m G_+P(m) = exp((z - 1) n_S).
 * cosh(a)/cosh(n) is written as (e^{a-|n|} + e^{-a-|n|}) / (1 + e^{-2|n|}):
 * numerator and denominator multiplied by e^{-|n|}, so nothing overflows. */
static cplx orc_gf_matrixP(double n, cplx nS, cplx z)
{
    cplx a = n + (z - 1.0) * nS;
    return (cexp(a - fabs(n)) + cexp(-a - fabs(n))) / (1.0 + exp(-2.0 * fabs(n)));
}

static cplx orc_gf_plusP(cplx nS, cplx z) { return cexp((z - 1.0) * nS); }

static cplx orc_root(int64_t k, int64_t K1)
{
    double th = 2.0 * ORC_PI * (double)(k % K1) / (double)K1;
    return cos(th) + I * sin(th);
}

void orc_gf_sample(double n, double nS_re, double nS_im, int K1, double *G_mP, double *G_pP)
{
    cplx nS = nS_re + I * nS_im;
    for (int k = 0; k < K1; ++k) {
        cplx z = orc_root(k, K1);
        cplx gm = orc_gf_matrixP(n, nS, z);
        cplx gp = orc_gf_plusP(nS, z);
        if (G_mP) { G_mP[2 * k] = creal(gm); G_mP[2 * k + 1] = cimag(gm); }
        if (G_pP) { G_pP[2 * k] = creal(gp); G_pP[2 * k + 1] = cimag(gp); }
    }
}

/* ------------------------------------------------------------------------ */
/* 6. Ensemble means, inverse DFT, sampling errors                           */
/* ------------------------------------------------------------------------ */
/* Sub-ensemble GF sums.  acc layout: [2 estimators][n_sub][K1] (re, im),
 * estimator 0 = matrix-P, 1 = +P; sample i (global index e0 + i) goes to
 * sub-ensemble (e0 + i) mod n_sub.  counts[n_sub] receives the sizes.
 * Sums over samples run in increasing sample order. */
int orc_accumulate_gf(const double *n, const double *nS, uint64_t e0, int64_t E, int n_sub,
                      int K1, double *acc, int64_t *counts, int threads)
{
    if (n_sub <= 0 || K1 <= 0) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    memset(acc, 0, sizeof(double) * 2 * 2 * (size_t)n_sub * (size_t)K1);
    for (int r = 0; r < n_sub; ++r) counts[r] = 0;
    for (int64_t i = 0; i < E; ++i) counts[(e0 + (uint64_t)i) % (uint64_t)n_sub] += 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K1; ++k) {
        cplx z = orc_root(k, K1);
        for (int64_t i = 0; i < E; ++i) {
            int r = (int)((e0 + (uint64_t)i) % (uint64_t)n_sub);
            cplx s = nS[2 * i] + I * nS[2 * i + 1];
            cplx gm = orc_gf_matrixP(n[i], s, z);
            cplx gp = orc_gf_plusP(s, z);
            size_t o0 = ((size_t)0 * n_sub + r) * K1 + k;
            size_t o1 = ((size_t)1 * n_sub + r) * K1 + k;
            acc[2 * o0] += creal(gm);
            acc[2 * o0 + 1] += cimag(gm);
            acc[2 * o1] += creal(gp);
            acc[2 * o1 + 1] += cimag(gp);
        }
    }
    return 0;
}

/* Inverse DFT of the sub-ensemble means and the statistics over sub-ensembles:
 *   P_r(m) = (1/K1) sum_k (acc_r(z_k)/count_r) z_k^{-m},  m = m_off .. m_off+K1-1,
 *   P(m) = mean_r Re P_r(m),  sigma(m) = std_r(Re P_r(m)) / sqrt(n_sub)
 * (sample standard deviation, n_sub - 1 in the denominator; sigma = 0 when
 * n_sub = 1).  Im_max[est] receives max_m |mean_r Im P_r(m)| (a diagnostic:
 * the exact P(m) is real).  Outputs: P[2][K1], sigma[2][K1]. */
int orc_invert(const double *acc, const int64_t *counts, int n_sub, int K1, int64_t m_off,
               double *P, double *sigma, double *Im_max, int threads)
{
    if (n_sub <= 0 || K1 <= 0) return -1;
    for (int r = 0; r < n_sub; ++r) if (counts[r] <= 0) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    double *Pr = (double *)malloc(sizeof(double) * 2 * 2 * (size_t)n_sub * (size_t)K1);
    if (!Pr) return -2;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int est = 0; est < 2; ++est) {
        for (int r = 0; r < n_sub; ++r) {
            const double *a = acc + 2 * (((size_t)est * n_sub + r) * K1);
            double inv_cnt = 1.0 / (double)counts[r];
            for (int q = 0; q < K1; ++q) {
                int64_t m = m_off + q;
                cplx s = 0.0;
                for (int k = 0; k < K1; ++k) {
                    /* z_k^{-m} with the exponent reduced exactly mod K1 */
                    int64_t km = ((int64_t)k * (m % K1)) % K1;
                    if (km < 0) km += K1;
                    double th = -2.0 * ORC_PI * (double)km / (double)K1;
                    cplx g = (a[2 * k] + I * a[2 * k + 1]) * inv_cnt;
                    s += g * (cos(th) + I * sin(th));
                }
                s /= (double)K1;
                size_t o = ((size_t)est * n_sub + r) * K1 + q;
                Pr[2 * o] = creal(s);
                Pr[2 * o + 1] = cimag(s);
            }
        }
    }
    for (int est = 0; est < 2; ++est) {
        double immax = 0.0;
        for (int q = 0; q < K1; ++q) {
            double mean = 0.0, mean_im = 0.0;
            for (int r = 0; r < n_sub; ++r) {
                size_t o = ((size_t)est * n_sub + r) * K1 + q;
                mean += Pr[2 * o];
                mean_im += Pr[2 * o + 1];
            }
            mean /= n_sub;
            mean_im /= n_sub;
            double var = 0.0;
            for (int r = 0; r < n_sub; ++r) {
                size_t o = ((size_t)est * n_sub + r) * K1 + q;
                double d = Pr[2 * o] - mean;
                var += d * d;
            }
            double sd = n_sub > 1 ? sqrt(var / (double)(n_sub - 1)) : 0.0;
            P[(size_t)est * K1 + q] = mean;
            sigma[(size_t)est * K1 + q] = sd / sqrt((double)n_sub);
            if (fabs(mean_im) > immax) immax = fabs(mean_im);
        }
        if (Im_max) Im_max[est] = immax;
    }
    free(Pr);
    return 0;
}

/* Direct per-bin route for bins m = m0 .. m0+count-1: sub-ensemble means of
 * the projector G(m) of step 4, then the same statistics (no DFT).
 * Outputs P[2][count], sigma[2][count]. */
int orc_direct_bins(const double *n, const double *nS, uint64_t e0, int64_t E, int n_sub,
                    int m0, int count, double *P, double *sigma, int threads)
{
    if (n_sub <= 0 || count <= 0) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    size_t per = (size_t)n_sub * (size_t)count;
    double *sum = (double *)calloc(2 * per, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)n_sub, sizeof(int64_t));
    if (!sum || !cnt) { free(sum); free(cnt); return -2; }
    for (int64_t i = 0; i < E; ++i) cnt[(e0 + (uint64_t)i) % (uint64_t)n_sub] += 1;
    for (int r = 0; r < n_sub; ++r) if (cnt[r] == 0) { free(sum); free(cnt); return -1; }
#pragma omp parallel
    {
        double *gm = (double *)malloc(sizeof(double) * 2 * (size_t)count);
        double *gp = (double *)malloc(sizeof(double) * 2 * (size_t)count);
        /* each thread owns a contiguous range of bins; samples in order */
#pragma omp for schedule(static)
        for (int q0 = 0; q0 < count; q0 += 64) {
            int cq = count - q0 < 64 ? count - q0 : 64;
            for (int64_t i = 0; i < E; ++i) {
                int r = (int)((e0 + (uint64_t)i) % (uint64_t)n_sub);
                orc_projector_direct(n[i], nS[2 * i], nS[2 * i + 1], m0 + q0, cq, gm, gp);
                for (int q = 0; q < cq; ++q) {
                    sum[(size_t)r * count + q0 + q] += gm[2 * q];
                    sum[per + (size_t)r * count + q0 + q] += gp[2 * q];
                }
            }
        }
        free(gm);
        free(gp);
    }
    for (int est = 0; est < 2; ++est) {
        for (int q = 0; q < count; ++q) {
            double mean = 0.0;
            for (int r = 0; r < n_sub; ++r)
                mean += sum[est * per + (size_t)r * count + q] / (double)cnt[r];
            mean /= n_sub;
            double var = 0.0;
            for (int r = 0; r < n_sub; ++r) {
                double d = sum[est * per + (size_t)r * count + q] / (double)cnt[r] - mean;
                var += d * d;
            }
            P[(size_t)est * count + q] = mean;
            sigma[(size_t)est * count + q] =
                n_sub > 1 ? sqrt(var / (double)(n_sub - 1)) / sqrt((double)n_sub) : 0.0;
        }
    }
    free(sum);
    free(cnt);
    return 0;
}

/* The whole estimator in one call (the CPU baseline): samples, GF sums, DFT. */
int orc_run(int N, int M, const double *T, const double *r, uint64_t seed, uint64_t e0,
            int64_t E, int n_sub, int K1, int64_t m_off, double *P, double *sigma,
            double *Im_max, int threads)
{
    double *n = (double *)malloc(sizeof(double) * (size_t)E);
    double *nS = (double *)malloc(sizeof(double) * 2 * (size_t)E);
    double *acc = (double *)malloc(sizeof(double) * 4 * (size_t)n_sub * (size_t)K1);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_sub);
    int rc = -2;
    if (n && nS && acc && cnt) {
        rc = orc_samples(N, M, T, r, seed, e0, E, n, nS, threads);
        if (rc == 0) rc = orc_accumulate_gf(n, nS, e0, E, n_sub, K1, acc, cnt, threads);
        if (rc == 0) rc = orc_invert(acc, cnt, n_sub, K1, m_off, P, sigma, Im_max, threads);
    }
    free(n);
    free(nS);
    free(acc);
    free(cnt);
    return rc;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
