/*
 * gbs.h -- C ABI of the GB300 matrix-P total-count estimator for Gaussian
 * boson sampling (Drummond, Dellios, Reid, arXiv:2503.12749).
 *
 * The library computes, for N squeezed-vacuum inputs (squeezing r_j >= 0)
 * sent through an M x N linear network T, the binned total-count
 * distribution P(m) of Eq. total_counts with two phase-space estimators on
 * the same trajectories:
 *   - the parity-projected (M = 2) matrix-P estimator, projector g_0 of
 *     Eq. c-number-variable;
 *   - the positive-P estimator, same equation with g_0 = 1
 *     (Eq. phase_space_projector).
 * Each trajectory draws real input amplitudes alpha, beta from the +P
 * density of the squeezed vacua ("Applications to GBS"), propagates them as
 * alpha' = T alpha, beta' = T* beta, and contributes its generating function
 *   G_mP(z) = cosh(n + (z-1) n_S) / cosh(n),   G_+P(z) = exp((z-1) n_S),
 *   n = sum_j alpha_j beta_j,  n_S = sum_i alpha'_i beta'_i,
 * at the K1 roots of unity z_k = exp(2 pi i k / K1).  Sub-ensemble means
 * (Appendix A: N_R sub-ensembles) are inverted by DFT to P(m) with the
 * sampling error std_r / sqrt(N_R).
 *
 * Conventions
 *   - Every function returns a status (GBS_OK = 0 or a negative code) and
 *     never aborts; gbs_last_error() returns a thread-local message for the
 *     last failure on the calling thread.
 *   - Host pointers are owned by the caller and only read/written during
 *     the call.  The library copies T and r at gbs_make_network and owns all
 *     device memory of a network until gbs_free_network.
 *   - Work is issued on the CUDA stream given at gbs_make_network (a
 *     cudaStream_t passed as void*, NULL = legacy default stream).
 *   - A network object must not be used from two host threads at once.
 *   - Trajectory e of a run with key `seed` draws its normals from
 *     Philox-4x32-10 (Salmon et al., SC'11) at counter (e, j); the result of
 *     a run is therefore fixed by (T, r, seed, sample range) and
 *     independent of how the range is split into calls.
 */
#ifndef GBS_H
#define GBS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define GBS_OK 0
#define GBS_EINVAL (-1)     /* invalid argument (sizes, r_j < 0, K1 not a power of two, ...) */
#define GBS_ENOMEM (-2)     /* device or host allocation failed */
#define GBS_ECUDA (-3)      /* a CUDA runtime/driver call failed */
#define GBS_ETIMEOUT (-4)   /* a bounded device-side wait gave up (error flag set by a kernel) */
#define GBS_ENONFINITE (-5) /* non-finite generating-function sums; the message holds the count */
#define GBS_ENOTSUP (-6)    /* feature not supported on this device / build */

/* Arithmetic of the propagation GEMM alpha' = T alpha, beta' = T* beta. */
#define GBS_FP64 0   /* FP64 sampler, FP64 SIMT GEMM, FP64 generating functions */
#define GBS_FP32 1   /* as GBS_FP64 with the SIMT GEMM in FP32: T and the samples
                        rounded to FP32, FP32 products accumulated in FP32 along
                        the N input modes; occupations and everything after
                        them in FP64 */
#define GBS_BF16X3 2 /* FP32 sampler, tcgen05 BF16 split GEMM with 3 products
                        (T0 B0 + T0 B1 + T1 B0), FP32 accumulation;
                        generating functions in double-float on the FP32
                        pipes (FP32 for terms below 2^-27), summed in FP64 */
#define GBS_BF16X6 3 /* as GBS_BF16X3 with 6 products (adds T1 B1, T0 B2, T2 B0) */

typedef struct gbs_net *gbs_net_t;

/*
 * gbs_make_network -- upload one network ("Applications to GBS": the
 * transmission matrix t acting as alpha' = t alpha, beta' = t* beta; loss as
 * a non-unitary t, "Computational results and losses").
 *   N, M       input and output mode counts, 1 <= N, M <= 65536.
 *   T          host, M*N complex numbers row-major, each as (re, im) doubles:
 *              T[2*(i*N + j)] = Re T_ij, T[2*(i*N + j) + 1] = Im T_ij.
 *              Read during the call only.  Page-locked memory that the
 *              device can address (cudaHostAlloc, cudaHostRegister) is read
 *              by the conversion kernel in place; other memory is first
 *              copied to a device buffer.
 *   r          host, N squeezing parameters, each finite and >= 0.
 *   precision  GBS_FP64, GBS_FP32, GBS_BF16X3 or GBS_BF16X6.  The BF16 paths
 *              split T (rounded to FP32) into BF16 planes T = T0 + T1 + T2;
 *              GBS_FP32 keeps T in FP64 and rounds it as the GEMM stages it.
 *   stream     cudaStream_t (as void*) used for every launch of this network.
 *   out        receives the handle.
 * Errors: EINVAL on bad sizes/values/null pointers; ENOMEM; ECUDA;
 * ENOTSUP when a BF16 precision is requested on a device without tcgen05.
 */
int gbs_make_network(int N, int M, const double *T, const double *r, int precision,
                     void *stream, gbs_net_t *out);

/*
 * gbs_make_network_device -- as gbs_make_network, with T in DEVICE memory
 * (same layout: M*N complex row-major, (re, im) doubles; read during the
 * call only, the library keeps its own converted copy).  The conversion
 * (FP64 reordering or BF16 splitting) runs on the GPU on `stream`, ordered
 * after the work already queued there only: T must be complete with respect
 * to `stream` (produced on it, or the stream made to wait for its producer).
 * Non-finite entries are counted there and rejected with EINVAL.  r stays a
 * host array.  Synchronises the stream.  Errors as gbs_make_network.
 */
int gbs_make_network_device(int N, int M, const double *T_dev, const double *r, int precision,
                            void *stream, gbs_net_t *out);

/*
 * gbs_sample -- draw trajectories first_sample .. first_sample+E-1 and add
 * their generating functions to the network's sub-ensemble sums
 * (the ensemble loop: sampling "Applications to GBS", observables
 * Eq. c-number-variable summed over m as a generating function, sub-ensembles
 * Appendix A).  Trajectory e belongs to sub-ensemble e mod n_sub.
 *   seed        Philox key (64 bits).
 *   E           number of trajectories, >= 0.
 *   n_sub       number of sub-ensembles N_R, >= 1.
 *   K1          number of DFT points K+1, a power of two in [2, 2^20].
 * The first call after make/reset fixes (n_sub, K1); later calls must pass
 * the same values (EINVAL otherwise).  Asynchronous on the network's stream
 * except for the first call's allocations.  Errors: EINVAL, ENOMEM, ECUDA,
 * ETIMEOUT.
 * A call cuts its trajectories into the fewest chunks of at most the
 * network's chunk size (gbs_network_info): chunks of ceil(E / chunks)
 * rounded up to a multiple of 128, the last one shorter; every sum runs in
 * a fixed order, so the same sequence of calls gives bitwise the same sums,
 * and so does a call split into calls at its own chunk boundaries (other
 * splits agree to rounding).  With the sampler folded into the GEMM
 * (gbs_set_sampler_fusion), when this call continues the network's
 * previous gbs_sample call (same seed, first_sample = that call's
 * first_sample + E), its last chunk's GEMM also draws the first chunk of a
 * following call on the same seed from first_sample + E, which that call
 * then does not draw again (the samples are the same either way): a stream
 * of consecutive calls then has no sampler launch, and a one-off call draws
 * nothing it does not use.
 */
int gbs_sample(gbs_net_t net, uint64_t seed, uint64_t first_sample, int64_t E, int n_sub,
               int K1);

/*
 * gbs_make_network_binned -- as gbs_make_network, with the output modes split
 * into d = 2..4 bins S_1 .. S_d for the joint distribution G(m_1, .., m_d)
 * of Eq. General_GCP with every mode binned ("Higher-dimensional binning").
 * bin: host, M ints, bin[i] in 0..d-1 (the bin of output mode i; d is the
 * largest value + 1), every bin non-empty.  Other arguments as
 * gbs_make_network.  The library stores the rows of each bin contiguously,
 * padded with zero rows to whole 64-mode tiles, so gbs_network_info reports
 * the padded M; gbs_sample still gives the total-count distribution.
 * Errors as gbs_make_network.
 */
int gbs_make_network_binned(int N, int M, const double *T, const double *r, const int *bin,
                            int precision, void *stream, gbs_net_t *out);

/*
 * gbs_sample_nd -- trajectories first..first+E-1 of a binned network into the
 * binned sums: per trajectory the generating function
 *   G_mP(z) = cosh(n + sum_b (z_b-1) n_Sb) / cosh(n),
 *   G_+P(z) = exp(sum_b (z_b-1) n_Sb),
 * n_Sb = sum over the output modes i of bin b of alpha'_i beta'_i, at
 * z_b = exp(2 pi i k_b / K_b) (the one-bin form of Eq. c-number-variable
 * with the exponent summed over the bins), summed per sub-ensemble (e mod
 * n_sub).  K: host, d powers of two >= 2 with prod K_b <= 2^22; the first
 * call fixes (n_sub, K) until gbs_reset.  Generating functions in FP64 (FP64
 * networks) or double-float (BF16 networks), summed in FP64.  Errors: EINVAL
 * (not a binned network, sizes), ENOMEM, ECUDA.
 */
int gbs_sample_nd(gbs_net_t net, uint64_t seed, uint64_t first_sample, int64_t E, int n_sub,
                  const int *K);

/*
 * gbs_binned_counts_nd -- the d-dimensional inverse DFT of the binned sums and
 * their statistics over sub-ensembles:
 *   P_r(m) = (1/prod K_b) sum_k <G>_r(z) prod_b z_b^{-m_b},
 * m_b = m_offset[b] .. m_offset[b] + K_b - 1, P = mean_r Re P_r, sigma =
 * std_r / sqrt(N_R).  m_offset: host, d values.  Host outputs of prod K_b
 * doubles each, row-major over (m_1, .., m_d); any may be NULL.
 * Synchronises the stream.  Errors: EINVAL, ECUDA.
 */
int gbs_binned_counts_nd(gbs_net_t net, const int64_t *m_offset, double *P_mP, double *sig_mP,
                         double *P_plusP, double *sig_plusP);

/*
 * gbs_sample_2d -- gbs_sample_nd for a network of two bins (grid K1 x K2):
 * trajectories first..first+E-1 into the two-bin sums, per trajectory the
 * generating function
 *   G_mP(z_1, z_2) = cosh(n + (z_1-1) n_S1 + (z_2-1) n_S2) / cosh(n),
 *   G_+P(z_1, z_2) = exp((z_1-1) n_S1 + (z_2-1) n_S2),
 * n_Sb = sum over the output modes i of bin b of alpha'_i beta'_i, at
 * z_b = exp(2 pi i k_b / K_b) (the one-bin form of Eq. c-number-variable
 * with the exponent summed over the bins), summed per sub-ensemble (e mod
 * n_sub).  K1, K2: powers of two, K1 K2 <= 2^22; the first call fixes
 * (n_sub, K1, K2) until gbs_reset.  Generating functions in FP64 (FP64
 * networks) or double-float (BF16 networks), summed in FP64.  Errors: EINVAL
 * (not a network of two bins, sizes), ENOMEM, ECUDA.
 */
int gbs_sample_2d(gbs_net_t net, uint64_t seed, uint64_t first_sample, int64_t E, int n_sub,
                  int K1, int K2);

/*
 * gbs_binned_counts_2d -- gbs_binned_counts_nd for a network of two bins:
 * the two-dimensional inverse DFT of the two-bin sums and their statistics
 * over sub-ensembles:
 *   P_r(m_1, m_2) = (1/(K1 K2)) sum_k <G>_r(z) z_1^{-m_1} z_2^{-m_2},
 * m_b = m_b_offset .. m_b_offset + K_b - 1, P = mean_r Re P_r, sigma =
 * std_r / sqrt(N_R).  Host outputs of K1*K2 doubles each, [m_1][m_2]
 * row-major; any may be NULL.  Synchronises the stream.  Errors: EINVAL,
 * ECUDA.
 */
int gbs_binned_counts_2d(gbs_net_t net, int64_t m1_offset, int64_t m2_offset, double *P_mP,
                         double *sig_mP, double *P_plusP, double *sig_plusP);

/*
 * gbs_moments -- normally-ordered moments and single-mode count marginals of
 * every output mode j ("Photon-counting observables") from trajectories
 * first..first+E-1 (the trajectories gbs_sample draws):
 *   Eq. moment, M = 2 parity case (Omega_00 = 1, T_0 = tanh n):
 *     <:n_j^m:> = < (n'_j)^m tanh(n)^(m mod 2) >  (matrix-P),
 *                 < (n'_j)^m >                    (+P),      m = 1..mmax;
 *   P_j(c) = < G(c) > with the projector of Eq. projection_op for S = {j},
 *     per trajectory Eq. c-number-variable with n_S = n'_j (matrix-P) and
 *     Eq. phase_space_projector (+P),                        c = 0..cmax;
 * n = sum_k alpha_k beta_k, n'_j = alpha'_j beta'_j.  Estimates are the mean
 * over sub-ensembles (trajectory e -> e mod n_sub) of the real part of the
 * sub-ensemble means, errors std_r / sqrt(n_sub) (0 for n_sub = 1).
 *   mmax   1..8;  cmax 0..15;  n_sub 1..65535 with E >= n_sub.
 *   mom, sig_mom     host, [2][M][mmax] (matrix-P first), m = 1..mmax;
 *   marg, sig_marg   host, [2][M][cmax + 1];  any output may be NULL.
 * Independent of the sub-ensemble sums of gbs_sample (nothing accumulates
 * across calls).  Per trajectory and mode in FP32 on the BF16 paths (FP64
 * for magnitudes |n'| > 40), FP64 on the FP64 path; sums in FP64.
 * Unbinned networks only.  Synchronises.  Errors: EINVAL, ENOMEM, ECUDA.
 */
int gbs_moments(gbs_net_t net, uint64_t seed, uint64_t first_sample, int64_t E, int n_sub,
                int mmax, int cmax, double *mom, double *sig_mom, double *marg, double *sig_marg);

/*
 * gbs_histogram -- probability densities of per-trajectory observables
 * (Appendix A, Eq. gen_probability_density): for trajectories
 * first..first+E-1 (the same trajectories gbs_sample would draw) and each
 * count m[q], the real parts of the matrix-P projector
 *   G_0(m) = [e^{-n_S} n_S^m e^{n} + e^{n_S} (-n_S)^m e^{-n}] / (m! 2 cosh n)
 * and of the +P projector G_+(m) = n_S^m e^{-n_S} / m! (Eq.
 * phase_space_projector) are counted in nbins equal bins of [lo, hi).
 *   m, nm     host, 1 <= nm <= 16 counts; 2 nm (nbins + 2) <= 12288.
 *   counts    host, [2][nm][nbins + 2] (matrix-P first); per row bin 0 counts
 *             values below lo (and NaN), bin nbins + 1 values >= hi.
 * Independent of the sub-ensemble sums.  Synchronises.  Errors: EINVAL,
 * ENOMEM, ECUDA.  The density of bin j is counts / (E * (hi - lo) / nbins).
 */
int gbs_histogram(gbs_net_t net, uint64_t seed, uint64_t first_sample, int64_t E, const int *m,
                  int nm, double lo, double hi, int nbins, int64_t *counts);

/*
 * gbs_binned_counts -- inverse DFT of the sub-ensemble means and the
 * statistics over sub-ensembles (Eq. total_counts; errors Appendix A):
 *   P_r(m) = (1/K1) sum_k <G>_r(z_k) z_k^{-m},  m = m_offset .. m_offset+K1-1,
 *   P(m) = mean_r Re P_r(m),  sigma(m) = std_r(Re P_r(m)) / sqrt(N_R)
 * (sample standard deviation; sigma = 0 when N_R = 1).  The result for bin m
 * is the aliased sum over m + j K1; choose K1 and m_offset to cover the
 * support.  Output arrays are host buffers of K1 doubles each; any of them
 * may be NULL to skip it.  Synchronises the network's stream.
 * Errors: EINVAL (no samples in some sub-ensemble), ETIMEOUT and ENONFINITE
 * (as gbs_check_finite), ECUDA.
 */
int gbs_binned_counts(gbs_net_t net, int64_t m_offset, double *P_mP, double *sig_mP,
                      double *P_plusP, double *sig_plusP);

/*
 * gbs_binned_counts_device -- as gbs_binned_counts, but writes into DEVICE
 * buffers and does not synchronise: out_dev holds 4*K1 doubles laid out as
 * [P_mP | sig_mP | P_plusP | sig_plusP].  No non-finite check is made (call
 * gbs_check_finite for it).  Errors: EINVAL, ECUDA.
 */
int gbs_binned_counts_device(gbs_net_t net, int64_t m_offset, double *out_dev);

/*
 * gbs_binned_counts_noalloc -- the same inversion and statistics as
 * gbs_binned_counts_device, for callers that must not allocate device
 * memory: for example a process whose device memory is owned entirely by
 * another allocator (a framework's caching pool or a pool reserved at
 * start-up), where a cudaMalloc outside that allocator fails or fragments
 * memory, or a latency-critical loop in which cudaMalloc/cudaFree would
 * synchronise the device.  The paper has no counterpart; it is a service of
 * this library.
 *   acc_dev     device, [2][n_sub][K1] complex sums as (re, im) doubles, the
 *               layout gbs_get_accumulators returns (estimator 0 = matrix-P).
 *   counts_dev  device, n_sub trajectory counts (each > 0; a zero count gives
 *               non-finite output).
 *   out_dev     device, 4*K1 doubles [P_mP | sig_mP | P_plusP | sig_plusP].
 *   stream      cudaStream_t (as void*) for the launches; asynchronous.
 * Work space is one fixed array inside the library (not allocated by the
 * call): 2 * n_sub * K1 <= 2^20 and K1 <= 2^16 (33 MB of device memory held
 * by every GPU that loads the library until exit); larger sizes return
 * GBS_EINVAL.  The first call on a device looks up the array's device address
 * (make it before capturing any stream) and keeps it for the life of the
 * process, so resetting the device (cudaDeviceReset) after that first call is
 * not supported.  Calls share the array: two calls that run at the same time
 * on one GPU race.  No network object is needed.
 */
int gbs_binned_counts_noalloc(const double *acc_dev, const int64_t *counts_dev, int n_sub,
                              int K1, int64_t m_offset, double *out_dev, void *stream);

/*
 * gbs_check_finite -- count non-finite entries of the sub-ensemble sums
 * (synchronises).  Returns GBS_OK and *count = 0 when all are finite,
 * GBS_ENONFINITE with *count > 0 otherwise.  Before counting it reads the
 * network's timeout flag: when a GEMM launch gave up waiting on its pipeline
 * since the last check (gbs_set_wait_limit), it clears the flag and returns
 * GBS_ETIMEOUT (*count = 0).
 */
int gbs_check_finite(gbs_net_t net, int64_t *count);

/*
 * gbs_debug_samples -- per-trajectory photon numbers for trajectories
 * e0 .. e0+count-1 of key `seed`, computed by the same kernels as gbs_sample
 * (for parity tests): n[count] (input total sum_j alpha_j beta_j) and
 * nS[2*count] (output total sum_i alpha'_i beta'_i as (re, im)), host
 * buffers.  Does not touch the sub-ensemble sums.  Synchronises.
 */
int gbs_debug_samples(gbs_net_t net, uint64_t seed, uint64_t e0, int64_t count, double *n,
                      double *nS);

/*
 * gbs_debug_windows -- the evaluation windows of the generating functions
 * for trajectories e0 .. e0+count-1 of key `seed` (measurement of the
 * generating-function work): w[2*count] as (w1, w2) per trajectory, host;
 * the terms e^{(z_k-1) n_S} are evaluated for the k within w1 of k = 0 and
 * matrix-P's e^{-(z_k-1) n_S - 2n} for the k within w2 of k = K1/2 (cyclic
 * distance; -1 = none, >= K1/2 = every k), every term outside below 2^-60
 * (GBS_FP64) or 2^-47 (the BF16 split paths, whose double-float evaluation
 * rounds terms of order one to 2^-46).
 * Needs K1 fixed by a gbs_sample call.  Does not touch the sub-ensemble
 * sums.  Synchronises.  Errors: EINVAL, ECUDA.
 */
int gbs_debug_windows(gbs_net_t net, uint64_t seed, uint64_t e0, int64_t count, int *w);

/*
 * gbs_debug_occupations -- the per-mode occupations n'_i = alpha'_i beta'_i
 * ("Applications to GBS") of trajectories e0 .. e0+count-1, as written by
 * the propagation GEMM's epilogue for gbs_moments: occ, host,
 * [M][count] complex as (re, im) pairs (FP32 values on the BF16 paths).
 * Unbinned networks only.  Synchronises.  Errors: EINVAL, ENOMEM, ECUDA.
 */
int gbs_debug_occupations(gbs_net_t net, uint64_t seed, uint64_t e0, int64_t count, double *occ);

/*
 * gbs_get_accumulators / gbs_set_accumulators -- the sub-ensemble sums as
 * host arrays: acc[2][n_sub][K1] complex (re, im) doubles (estimator 0 =
 * matrix-P, 1 = +P; each the SUM of G(z_k) over the sub-ensemble's
 * trajectories) and counts[n_sub] (trajectories per sub-ensemble).  Used for
 * checkpoint/resume and to combine runs.  gbs_set_accumulators also fixes
 * (n_sub, K1) like a first gbs_sample.  Both synchronise.
 */
int gbs_get_accumulators(gbs_net_t net, int *n_sub, int *K1, double *acc, int64_t *counts);
int gbs_set_accumulators(gbs_net_t net, int n_sub, int K1, const double *acc,
                         const int64_t *counts);

/* gbs_reset -- clear the sub-ensemble sums and unfix (n_sub, K1). */
int gbs_reset(gbs_net_t net);

/* gbs_network_info -- N, M, precision and the trajectories per internal chunk. */
int gbs_network_info(gbs_net_t net, int *N, int *M, int *precision, int64_t *chunk);

/*
 * gbs_set_gemm_config / gbs_gemm_config -- tile configuration of the tcgen05
 * propagation GEMM (BF16 paths; not part of the method: every configuration
 * gives bitwise the same sums).  pair = 1: one CTA per (64-mode tile,
 * 128-trajectory tile); 2: CTA pairs (cta_group::2, clusters of 2 CTAs) on
 * adjacent mode tiles of one trajectory tile, each CTA loading its own A
 * tile and half of the trajectory tile, the pair's MMA reading both halves.
 * band = 0: the tiles of one chunk in the plain order (all mode tiles of a
 * trajectory tile side by side); band > 0: in bands of `band` mode-tile
 * groups (a group = the 1 or 2 mode tiles of a CTA or pair), the trajectory
 * tiles of a band in order, so that a band's A tiles are read again from L2.
 * keep_a is a set of bits: 1 (with band > 0) loads the band's A tiles with
 * the evict-last L2 policy (4: for half of their lines); 2 loads the
 * trajectory tiles with the evict-first policy; 8 aligns the waves of CTAs:
 * before each tile of the second to the last full wave every CTA waits, for
 * at most 50 us, until all have issued the loads of their previous tile, so
 * that tiles shared within a wave are read while the L2 holds them (a wait
 * that times out is not an error: that CTA stops waiting for the rest of the
 * launch); 16 runs the operand ring in shared memory one stage shallower
 * than the deepest that fits (4 stages for one CTA and 6 for a pair with 3
 * products, 3 and 4 with 6 products).  None of them changes a result.
 * pair = 0 returns to the autotuner, which times the candidates (one CTA or
 * pairs; bands of 16 and 8 with and without the evict-last policy; the
 * plain order only where all of A fits in half the L2; each with the
 * deepest ring and with one stage less) on the first chunk
 * of each kind of launch (plain, and the one that also samples the next
 * chunk) in a loaded, interleaved sequence, keeps the fastest and adds the
 * wave alignment to banded orders (cached per size bucket of N and M for
 * the process).  gbs_gemm_config returns the configuration in use ((0, 0,
 * 0) before the first chunk).  EINVAL: FP64 network, pair not 0..2,
 * band < 0, keep_a not in 0..31, NULL pointers.
 */
int gbs_set_gemm_config(gbs_net_t net, int pair, int band, int keep_a);
int gbs_gemm_config(gbs_net_t net, int *pair, int *band, int *keep_a);

/*
 * gbs_set_pair_autotune -- whether the GEMM autotuner (and the batch's) also
 * times CTA pairs (on by default); process-wide, clears the autotuner's
 * cache.  Networks already configured keep their configuration.
 */
int gbs_set_pair_autotune(int enable);

/*
 * gbs_set_wait_limit -- bound, in nanoseconds, of every pipeline wait in the
 * network's tcgen05 GEMM launches (default 2e9; a wait that has not seen its
 * phase complete after that long raises the network's timeout flag, the
 * kernel stops issuing work, waits for what it already issued and returns).
 * The next synchronous read (gbs_binned_counts, gbs_check_finite,
 * gbs_moments) then returns GBS_ETIMEOUT and clears the flag; the sums of a
 * call that timed out are not meaningful (gbs_reset clears them).  A limit
 * of 0 exercises that path without a fault: each GEMM launch then first
 * waits on a barrier that nothing arrives on, gives up at once and issues
 * no MMA.  EINVAL: NULL network.
 */
int gbs_set_wait_limit(gbs_net_t net, uint64_t limit_ns);

/*
 * gbs_set_sampler_fusion / gbs_sampler_fusion -- sampling of the next chunk
 * inside the propagation GEMM (GBS_BF16X3 only).  When gbs_sample (also
 * gbs_sample_nd, gbs_moments and the rounds of gbs_sample_batch) covers more
 * than one chunk, the GEMM of chunk i also draws the samples of chunk i + 1
 * (the +P sampling of "Applications to GBS", Philox counters as in
 * gbs_sample) into a second sample operand allocated on first use (the size
 * of the first: about 1 GiB at N = 1000), so the sampler's arithmetic runs
 * in issue slots the tensor-core GEMM leaves idle.  mode = 0: never; 1 (the
 * default): for networks with at least 900 output modes (with fewer, the
 * GEMM of a chunk is too short to hide the sampling of the next); 2:
 * whenever the network can.  The samples and every sum are bitwise those of
 * mode 0.  Without room for the second operand, inside a stream capture
 * that would have to allocate it, or when the library's sampling GEMM was
 * not built with the register split it needs, the plain chunk loop runs.
 * gbs_sampler_fusion sets *active = 1 when the next call of more than one
 * chunk folds the sampler (the setting asks for it and the second operand
 * exists), else 0.  EINVAL: mode not 0, 1 or 2, NULL pointer.
 */
int gbs_set_sampler_fusion(gbs_net_t net, int mode);
int gbs_sampler_fusion(gbs_net_t net, int *active);

/*
 * Batches of networks of uneven size (many validations at once).  Each
 * network keeps its own sub-ensemble sums and is read out with
 * gbs_binned_counts; the batch only changes how the work is launched: per
 * round of one chunk per network, the samplers of all networks, ONE
 * persistent tcgen05 GEMM over the tiles of all networks (ordered by
 * decreasing K), then each network's generating-function sums.  All rounds
 * of a call are captured into one CUDA graph and launched once (on the
 * legacy default stream, which cannot be captured, they are issued
 * directly).  The batch GEMM's tile configuration is chosen by timing the
 * candidates on the first call's first round (gbs_set_batch_config).
 *
 * gbs_make_batch -- group `count` networks (1..4096) that share a BF16
 *   precision, a device and a stream.  The networks stay owned by the
 *   caller and must outlive the batch.
 * gbs_sample_batch -- as gbs_sample for every network i at once: seeds[i],
 *   first_sample[i], E[i], n_sub[i], K1[i] (host arrays of `count`).  The
 *   same trajectories as per-network gbs_sample calls are drawn.
 *   Synchronises the stream before capturing (descriptor upload).
 * gbs_set_batch_config -- the batch GEMM's configuration: pair 1 (one CTA
 *   per tile) or 2 (CTA pairs), band 0 (every network's tiles in the plain
 *   order) or > 0 (bands of that many mode-tile groups within each
 *   network), stages 0 (the deepest operand ring that fits in shared
 *   memory: 4 stages for one CTA and 6 for a pair with 3 products, 3 and 4
 *   with 6 products) or that depth, or one stage less; pair 0 returns to the
 *   autotuner, which times one CTA per tile and CTA pairs
 *   (gbs_set_pair_autotune), each with bands 0 and 8 and both ring depths,
 *   on the first call's first round.  Every configuration gives bitwise the
 *   same sums.  EINVAL: pair not 0..2, band < 0, stages not 0 or one of the
 *   two depths of (products, pair).
 * gbs_batch_info -- GEMM configuration in use (pair, band, ring stages;
 *   0, 0, 0 before the first call), rounds and GEMM tiles of the last call.
 * With phase timing enabled on the batch's first network (gbs_profile_enable),
 * gbs_sample_batch issues its rounds directly instead of as a graph and
 * attributes the grouped GEMM launches to that network's GEMM phase; each
 * network with phase timing enabled records its own generating-function
 * launches.
 * gbs_free_batch -- release the batch (not its networks).
 */
typedef struct gbs_batch *gbs_batch_t;
int gbs_make_batch(gbs_net_t *nets, int count, gbs_batch_t *out);
int gbs_sample_batch(gbs_batch_t batch, const uint64_t *seeds, const uint64_t *first_sample,
                     const int64_t *E, const int *n_sub, const int *K1);
int gbs_set_batch_config(gbs_batch_t batch, int pair, int band, int stages);
int gbs_batch_info(gbs_batch_t batch, int *pair, int *band, int *stages, int *rounds,
                   int64_t *tiles);
void gbs_free_batch(gbs_batch_t batch);

/*
 * Kernel-phase timing (instrumentation, not part of the method).  When
 * enabled, every kernel launch of the network is bracketed by CUDA events
 * recorded on the network's stream and attributed to a phase:
 */
#define GBS_PHASE_SAMPLE 0   /* phase-space input sampler */
#define GBS_PHASE_GEMM 1     /* propagation GEMM + occupation epilogue */
#define GBS_PHASE_FINALIZE 2 /* per-trajectory n_S sum and evaluation windows */
#define GBS_PHASE_GF 3       /* generating functions summed per sub-ensemble */
#define GBS_PHASE_INVERT 4   /* inverse DFT and statistics */
#define GBS_PHASE_MOMENTS 5  /* moments / marginals: per-trajectory parameters,
                                per-mode sums, statistics (gbs_moments) */
#define GBS_NPHASES 6
/* gbs_profile_enable -- start (enable != 0) or stop recording; starting
 * discards earlier records. */
int gbs_profile_enable(gbs_net_t net, int enable);
/* gbs_profile_read -- synchronise, then return per phase the summed event
 * time in milliseconds (ms[GBS_NPHASES]) and the number of kernel launches
 * (launches[GBS_NPHASES]) since the last enable/read; clears the records. */
int gbs_profile_read(gbs_net_t net, double *ms, int64_t *launches);

/*
 * gbs_measure_fp64_rate -- instrumentation, not part of the method: the
 * device's FP64 fused multiply-add rate in TFLOP/s (2 FLOP per FMA), timed
 * with CUDA events on `stream`.  Kernels of independent FMA chains (8, 16
 * or 32 accumulators per thread, 2 to 8 blocks of 256 threads per SM; as
 * outer-product updates with distinct operand registers and as recurrences
 * sharing one multiplier and addend) run 3 times each after a warm-up
 * launch; the best rate is returned.  It is the peak against which the FP64
 * path's propagation (k_gemm_fp64, bound by that rate) is reported, at the
 * clock the device ran the probe at.  Allocates small buffers
 * (stream-ordered) and synchronises `stream`.  Errors: EINVAL (NULL
 * tflops), ECUDA.
 */
int gbs_measure_fp64_rate(void *stream, double *tflops);

/* gbs_free_network -- synchronise the network's stream and release all memory
 * of the network (NULL is a no-op).  All device memory of a network (the
 * split T, the chunk workspace of sample operands, per-trajectory n, n_S,
 * windows and records -- about 1 GiB at N = 1000, twice that with the folded
 * sampler -- and the estimator's sums and tables) comes from the device's
 * default stream-ordered memory pool, allocated and freed on the network's
 * stream, so neither creating nor freeing a network synchronises the device;
 * the library raises that pool's release threshold once per device, so the
 * process keeps the memory for the next network instead of returning it to
 * the driver.  The stream must stay valid until this call. */
void gbs_free_network(gbs_net_t net);

/* gbs_last_error -- message of the last failure on this thread ("" if none). */
const char *gbs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GBS_H */
