// Two-dimensional binning ("Higher-dimensional binning", Eq. General_GCP with
// d = 2 and every output mode in one of the bins S_1, S_2): the joint
// distribution G(m_1, m_2) of the counts in the two bins.
//
// Per trajectory, with n = alpha.beta and n_Sb = sum_{i in S_b} alpha'_i
// beta'_i, the bin-total projectors have the generating function
//   G_mP(z_1, z_2) = cosh(n + L) / cosh(n),   G_+P(z_1, z_2) = e^{L},
//   L = (z_1 - 1) n_S1 + (z_2 - 1) n_S2,
// the one-bin form of Eq. c-number-variable with the exponent summed over
// the bins (the parity weight depends on m_1 + m_2).  The GEMM is the
// one-bin GEMM unchanged: the rows of each bin are contiguous and padded to
// whole 64-mode tiles, so its per-tile partials sum to n_S1 and n_S2.
//
// Evaluated on a (Ka x Kb) grid of z_b = e^{i theta_b} in FP64 (FP64
// networks) or in double-float on the FP32 pipes (BF16 networks, the
// one-bin kernel's table-driven exp and sin/cos, FP64 for arguments beyond
// their ranges); with
// L = l + i phi the same stable form as the one-bin kernels,
//   G_mP = [e^{l + c1} e^{i phi} + e^{-l + c2} e^{-i phi}] / (1 + e^{-2|n|}),
// c1 = min(0, 2n), c2 = -2 max(n, 0).  Terms below 2^-60 are skipped with
// per-dimension windows: for the e^{L} term the window in theta_1 uses the
// bound l_1(theta_1) <= -c x_1 + sqrt(2c) |y_1| (c = 1 - cos theta_1) with the
// threshold raised by the largest value of the theta_2 part, and likewise in
// theta_2 and for the e^{-L} term around (pi, pi).  Sub-ensemble sums are
// inverted by a two-dimensional FFT (rows, transpose, rows).
#include "gbs_internal.cuh"
#include "dfloat.cuh"

#include <cmath>

namespace gbs {
namespace {

constexpr double kTwoPi2 = 6.283185307179586476925286766559;
constexpr int kG2Threads = 128;
constexpr int kG2Tile = 128;

// max over c in [0, 2] of -c x + sqrt(2c) |y|
__device__ __forceinline__ double max_term1(double x, double y) {
    const double ay = fabs(y);
    if (x > 0.0) {
        const double cs = y * y / (2.0 * x * x);
        if (cs <= 2.0) return y * y / (2.0 * x);
    }
    return -2.0 * x + 2.0 * ay;
}

// max over c' in [0, 2] of (2 - c') x + sqrt(2c') |y|
__device__ __forceinline__ double max_term2(double x, double y) {
    const double ay = fabs(y);
    if (x > 0.0) {
        const double cs = y * y / (2.0 * x * x);
        if (cs <= 2.0) return 2.0 * x + y * y / (2.0 * x);
    }
    return 2.0 * ay;
}

__device__ __forceinline__ int half_width2(double cstar, int K) {
    const int half = K >> 1;
    if (!(cstar < 2.0)) return half;
    const double th = 2.0 * asin(sqrt(0.5 * cstar));
    const double w = floor(th * (double)K / kTwoPi2) + 1.0;
    return w >= (double)half ? half : (int)w;
}

// window of the e^{L} term in one dimension: -c x + sqrt(2c)|y| >= -T
__device__ __forceinline__ int win_term1(double x, double y, double T, int K) {
    if (!(x > 0.0)) return K >> 1;
    const double ay = fabs(y);
    const double u = (1.4142135623730951 * ay + sqrt(2.0 * y * y + 4.0 * x * T)) / (2.0 * x);
    return half_width2(u * u, K);
}

// window of the e^{-L} term around pi: (2 - c')x + sqrt(2c')|y| + c >= -T
__device__ __forceinline__ int win_term2(double x, double y, double c, double T, int K) {
    const double ay = fabs(y);
    if (!(x > 0.0)) return (2.0 * ay + c >= -T) ? (K >> 1) : -1;
    const double D = 2.0 * x + c + T;
    const double disc = 2.0 * y * y + 4.0 * x * D;
    if (disc < 0.0) return -1;
    const double u = (1.4142135623730951 * ay + sqrt(disc)) / (2.0 * x);
    return u < 0.0 ? -1 : half_width2(u * u, K);
}

__global__ void k_finalize2d(const double2 *__restrict__ part, int mtiles, int tile0, int64_t ld,
                             const double *__restrict__ n, int64_t count, int Ka, int Kb,
                             double2 *__restrict__ nS2, Window2 *__restrict__ win,
                             int *__restrict__ wmax) {
    int m[4] = {-1, -1, -1, -1};
    const double T = kSkipLog;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        double x1 = 0.0, y1 = 0.0, x2 = 0.0, y2 = 0.0;
        for (int t = 0; t < tile0; ++t) {
            const double2 p = part[(size_t)t * ld + i];
            x1 += p.x;
            y1 += p.y;
        }
        for (int t = tile0; t < mtiles; ++t) {
            const double2 p = part[(size_t)t * ld + i];
            x2 += p.x;
            y2 += p.y;
        }
        nS2[2 * i] = make_double2(x1, y1);
        nS2[2 * i + 1] = make_double2(x2, y2);
        const double c2 = -2.0 * fmax(n[i], 0.0);
        Window2 w;
        w.w1a = win_term1(x1, y1, T + max_term1(x2, y2), Ka);
        w.w1b = win_term1(x2, y2, T + max_term1(x1, y1), Kb);
        w.w2a = win_term2(x1, y1, c2 + max_term2(x2, y2), T, Ka);
        w.w2b = win_term2(x2, y2, c2 + max_term2(x1, y1), T, Kb);
        if (w.w2a < 0 || w.w2b < 0) w.w2a = w.w2b = -1;
        win[i] = w;
        m[0] = max(m[0], w.w1a);
        m[1] = max(m[1], w.w1b);
        m[2] = max(m[2], w.w2a);
        m[3] = max(m[3], w.w2b);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) m[q] = __reduce_max_sync(0xffffffffu, m[q]);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) atomicMax(&wmax[q], m[q]);
}

__device__ __forceinline__ int slots_of(int K, int W1, int W2) {
    const int half = K >> 1;
    const int n1 = W1 >= half ? K : 2 * W1 + 1;
    const int n2 = W2 < 0 ? 0 : (W2 >= half ? K : 2 * W2 + 1);
    return n1 + n2 >= K ? K : n1 + n2;
}

// k of slot i of one dimension: the window around 0 (k = -W1..W1), then the
// one around K/2; the whole range when they cover it.
__device__ __forceinline__ int slot_k(int i, int K, int W1, int W2) {
    const int half = K >> 1;
    const int n1 = W1 >= half ? K : 2 * W1 + 1;
    const int n2 = W2 < 0 ? 0 : (W2 >= half ? K : 2 * W2 + 1);
    if (n1 + n2 >= K) return i;
    if (i < n1) {
        const int k = i - W1;
        return k < 0 ? k + K : k;
    }
    return half - W2 + (i - n1);
}

__device__ __forceinline__ int d0(int k, int K) { return k <= (K >> 1) ? k : K - k; }
__device__ __forceinline__ int dpi(int k, int K) {
    const int d = k - (K >> 1);
    return d < 0 ? -d : d;
}

// One thread per (k_1, k_2) slot of the union window, one block row per
// sub-ensemble r; each thread adds its sub-ensemble's trajectories in
// increasing order.
__global__ void __launch_bounds__(kG2Threads)
    k_gf2d(const double *__restrict__ n_in, const double2 *__restrict__ nS2,
           const Window2 *__restrict__ win_in, const int *__restrict__ wmax, int64_t count,
           uint64_t e0, int n_sub, int Ka, int Kb, const double2 *__restrict__ tw,
           double2 *__restrict__ acc, int64_t *__restrict__ counts) {
    __shared__ double s_x1[kG2Tile], s_y1[kG2Tile], s_x2[kG2Tile], s_y2[kG2Tile];
    __shared__ double s_c1[kG2Tile], s_c2[kG2Tile], s_inv[kG2Tile];
    __shared__ Window2 s_w[kG2Tile];
    const int r = blockIdx.y;
    const int W1a = wmax[0], W1b = wmax[1], W2a = wmax[2], W2b = wmax[3];
    const int Sa = slots_of(Ka, W1a, W2a), Sb = slots_of(Kb, W1b, W2b);
    const int64_t slot = (int64_t)blockIdx.x * kG2Threads + threadIdx.x;
    const int64_t first = (int64_t)(((uint64_t)r + (uint64_t)n_sub - e0 % (uint64_t)n_sub) %
                                    (uint64_t)n_sub);
    const int64_t cnt_r = first < count ? (count - 1 - first) / n_sub + 1 : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[r] += cnt_r;
    if ((int64_t)blockIdx.x * kG2Threads >= (int64_t)Sa * Sb) return;  // block past the grid
    const bool valid = slot < (int64_t)Sa * Sb;
    const int k1 = valid ? slot_k((int)(slot / Sb), Ka, W1a, W2a) : 0;
    const int k2 = valid ? slot_k((int)(slot % Sb), Kb, W1b, W2b) : 0;
    const int a0 = valid ? d0(k1, Ka) : 0x3fffffff, b0 = valid ? d0(k2, Kb) : 0x3fffffff;
    const int api = valid ? dpi(k1, Ka) : 0x3fffffff, bpi = valid ? dpi(k2, Kb) : 0x3fffffff;
    const double2 ta = tw[k1], tb = tw[Ka + k2];
    double am_re = 0.0, am_im = 0.0, ap_re = 0.0, ap_im = 0.0;
    for (int64_t base = 0; base < cnt_r; base += kG2Tile) {
        const int64_t q = base + threadIdx.x;
        if (q < cnt_r) {
            const int64_t i = first + q * n_sub;
            const double nn = n_in[i];
            const double2 s1 = nS2[2 * i], s2 = nS2[2 * i + 1];
            s_x1[threadIdx.x] = s1.x;
            s_y1[threadIdx.x] = s1.y;
            s_x2[threadIdx.x] = s2.x;
            s_y2[threadIdx.x] = s2.y;
            s_c1[threadIdx.x] = fmin(0.0, 2.0 * nn);
            s_c2[threadIdx.x] = -2.0 * fmax(nn, 0.0);
            s_inv[threadIdx.x] = 1.0 / (1.0 + exp(-2.0 * fabs(nn)));
            s_w[threadIdx.x] = win_in[i];
        }
        __syncthreads();
        const int ntile = (cnt_r - base) < kG2Tile ? (int)(cnt_r - base) : kG2Tile;
        if (valid) {
            for (int j = 0; j < ntile; ++j) {
                const Window2 w = s_w[j];
                const bool in1 = a0 <= w.w1a && b0 <= w.w1b;
                const bool in2 = api <= w.w2a && bpi <= w.w2b;
                if (!(in1 || in2)) continue;
                const double x1 = s_x1[j], y1 = s_y1[j], x2 = s_x2[j], y2 = s_y2[j];
                const double l = (ta.x * x1 - ta.y * y1) + (tb.x * x2 - tb.y * y2);
                const double ph = (ta.y * x1 + ta.x * y1) + (tb.y * x2 + tb.x * y2);
                double sp, cp;
                sincos(ph, &sp, &cp);
                double e1 = 0.0, e2 = 0.0;
                if (in1) {
                    const double c1 = s_c1[j];
                    e1 = exp(l + c1);
                    const double gp = (c1 == 0.0) ? e1 : exp(l);
                    ap_re += gp * cp;
                    ap_im += gp * sp;
                }
                if (in2) e2 = exp(-l + s_c2[j]);
                const double inv = s_inv[j];
                am_re += (e1 + e2) * cp * inv;
                am_im += (e1 - e2) * sp * inv;
            }
        }
        __syncthreads();
    }
    if (valid) {
        const size_t grid = (size_t)Ka * Kb;
        const size_t o = (size_t)k1 * Kb + k2;
        double2 *p0 = acc + (size_t)r * grid + o;
        double2 *p1 = acc + ((size_t)n_sub + r) * grid + o;
        const double2 v0 = *p0, v1 = *p1;
        *p0 = make_double2(v0.x + am_re, v0.y + am_im);
        *p1 = make_double2(v1.x + ap_re, v1.y + ap_im);
    }
}

// The same sums in double-float arithmetic (BF16 networks).
__global__ void __launch_bounds__(kG2Threads)
    k_gf2d_df(const double *__restrict__ n_in, const double2 *__restrict__ nS2,
              const Window2 *__restrict__ win_in, const int *__restrict__ wmax, int64_t count,
              uint64_t e0, int n_sub, int Ka, int Kb, const double2 *__restrict__ tw,
              const DfConsts K, double2 *__restrict__ acc, int64_t *__restrict__ counts) {
    __shared__ df s_x1[kG2Tile], s_y1[kG2Tile], s_x2[kG2Tile], s_y2[kG2Tile];
    __shared__ df s_c1[kG2Tile], s_c2[kG2Tile], s_inv[kG2Tile];
    __shared__ double s_n[kG2Tile];
    __shared__ double2 s_s1[kG2Tile], s_s2[kG2Tile];
    __shared__ Window2 s_w[kG2Tile];
    __shared__ DfTables s_tab;
    const int r = blockIdx.y;
    const int W1a = wmax[0], W1b = wmax[1], W2a = wmax[2], W2b = wmax[3];
    const int Sa = slots_of(Ka, W1a, W2a), Sb = slots_of(Kb, W1b, W2b);
    const int64_t slot = (int64_t)blockIdx.x * kG2Threads + threadIdx.x;
    const int64_t first = (int64_t)(((uint64_t)r + (uint64_t)n_sub - e0 % (uint64_t)n_sub) %
                                    (uint64_t)n_sub);
    const int64_t cnt_r = first < count ? (count - 1 - first) / n_sub + 1 : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[r] += cnt_r;
    if ((int64_t)blockIdx.x * kG2Threads >= (int64_t)Sa * Sb) return;  // block past the grid
    if (threadIdx.x < 64) s_tab.exp2[threadIdx.x] = df{K.exp2_hi[threadIdx.x], K.exp2_lo[threadIdx.x]};
    if (threadIdx.x < 33) {
        s_tab.sn[threadIdx.x] = df{K.sin_hi[threadIdx.x], K.sin_lo[threadIdx.x]};
        s_tab.cs[threadIdx.x] = df{K.cos_hi[threadIdx.x], K.cos_lo[threadIdx.x]};
    }  // visible after the first __syncthreads of the tile loop
    const bool valid = slot < (int64_t)Sa * Sb;
    const int k1 = valid ? slot_k((int)(slot / Sb), Ka, W1a, W2a) : 0;
    const int k2 = valid ? slot_k((int)(slot % Sb), Kb, W1b, W2b) : 0;
    const int a0 = valid ? d0(k1, Ka) : 0x3fffffff, b0 = valid ? d0(k2, Kb) : 0x3fffffff;
    const int api = valid ? dpi(k1, Ka) : 0x3fffffff, bpi = valid ? dpi(k2, Kb) : 0x3fffffff;
    const double2 tad = tw[k1], tbd = tw[Ka + k2];
    const df cma = df_from_double(tad.x), sna = df_from_double(tad.y);
    const df cmb = df_from_double(tbd.x), snb = df_from_double(tbd.y);
    double am_re = 0.0, am_im = 0.0, ap_re = 0.0, ap_im = 0.0;
    for (int64_t base = 0; base < cnt_r; base += kG2Tile) {
        const int64_t q = base + threadIdx.x;
        if (q < cnt_r) {
            const int64_t i = first + q * n_sub;
            const double nn = n_in[i];
            const double2 v1 = nS2[2 * i], v2 = nS2[2 * i + 1];
            s_x1[threadIdx.x] = df_from_double(v1.x);
            s_y1[threadIdx.x] = df_from_double(v1.y);
            s_x2[threadIdx.x] = df_from_double(v2.x);
            s_y2[threadIdx.x] = df_from_double(v2.y);
            s_c1[threadIdx.x] = df_from_double(fmin(0.0, 2.0 * nn));
            s_c2[threadIdx.x] = df_from_double(-2.0 * fmax(nn, 0.0));
            s_inv[threadIdx.x] = df_from_double(1.0 / (1.0 + exp(-2.0 * fabs(nn))));
            s_n[threadIdx.x] = nn;
            s_s1[threadIdx.x] = v1;
            s_s2[threadIdx.x] = v2;
            s_w[threadIdx.x] = win_in[i];
        }
        __syncthreads();
        const int ntile = (cnt_r - base) < kG2Tile ? (int)(cnt_r - base) : kG2Tile;
        if (valid) {
            df pm_re = {0.0f, 0.0f}, pm_im = {0.0f, 0.0f}, pp_re = {0.0f, 0.0f},
               pp_im = {0.0f, 0.0f};
            for (int j = 0; j < ntile; ++j) {
                const Window2 w = s_w[j];
                const bool in1 = a0 <= w.w1a && b0 <= w.w1b;
                const bool in2 = api <= w.w2a && bpi <= w.w2b;
                if (!(in1 || in2)) continue;
                const df x1 = s_x1[j], y1 = s_y1[j], x2 = s_x2[j], y2 = s_y2[j];
                const df l = df_add(df_sub(df_mul(cma, x1), df_mul(sna, y1)),
                                    df_sub(df_mul(cmb, x2), df_mul(snb, y2)));
                const df ph = df_add(df_add(df_mul(sna, x1), df_mul(cma, y1)),
                                     df_add(df_mul(snb, x2), df_mul(cmb, y2)));
                const df c1 = s_c1[j];
                const df a1 = df_add(l, c1);
                const df a2 = df_add(df_neg(l), s_c2[j]);
                const bool big = fabsf(ph.hi) >= 6000.0f ||
                                 (in1 && (a1.hi >= 80.0f || l.hi >= 80.0f)) ||
                                 (in2 && a2.hi >= 80.0f);
                if (big) {
                    // outside the double-float ranges: this pair in FP64
                    const double2 v1 = s_s1[j], v2 = s_s2[j];
                    const double nn = s_n[j];
                    const double ld = (tad.x * v1.x - tad.y * v1.y) + (tbd.x * v2.x - tbd.y * v2.y);
                    const double pd = (tad.y * v1.x + tad.x * v1.y) + (tbd.y * v2.x + tbd.x * v2.y);
                    double sd, cd;
                    sincos(pd, &sd, &cd);
                    const double c1d = fmin(0.0, 2.0 * nn), c2d = -2.0 * fmax(nn, 0.0);
                    double e1d = 0.0, e2d = 0.0;
                    if (in1) {
                        e1d = exp(ld + c1d);
                        const double gp = (c1d == 0.0) ? e1d : exp(ld);
                        ap_re += gp * cd;
                        ap_im += gp * sd;
                    }
                    if (in2) e2d = exp(-ld + c2d);
                    const double inv = df_to_double(s_inv[j]);
                    am_re += (e1d + e2d) * cd * inv;
                    am_im += (e1d - e2d) * sd * inv;
                    continue;
                }
                df sp, cp;
                df_sincos_tab(ph, s_tab, K, sp, cp);
                const df inv = s_inv[j];
                df e1 = {0.0f, 0.0f}, e2 = {0.0f, 0.0f};
                if (in1) {
                    e1 = a1.hi < -87.0f ? df{0.0f, 0.0f} : df_exp_tab(a1, s_tab, K);
                    const df gp = (c1.hi == 0.0f)
                                      ? e1
                                      : (l.hi < -87.0f ? df{0.0f, 0.0f} : df_exp_tab(l, s_tab, K));
                    pp_re = df_add(pp_re, df_mul(gp, cp));
                    pp_im = df_add(pp_im, df_mul(gp, sp));
                }
                if (in2) e2 = a2.hi < -87.0f ? df{0.0f, 0.0f} : df_exp_tab(a2, s_tab, K);
                pm_re = df_add(pm_re, df_mul(df_mul(df_add(e1, e2), inv), cp));
                pm_im = df_add(pm_im, df_mul(df_mul(df_sub(e1, e2), inv), sp));
            }
            am_re += df_to_double(pm_re);
            am_im += df_to_double(pm_im);
            ap_re += df_to_double(pp_re);
            ap_im += df_to_double(pp_im);
        }
        __syncthreads();
    }
    if (valid) {
        const size_t grid = (size_t)Ka * Kb;
        const size_t o = (size_t)k1 * Kb + k2;
        double2 *p0 = acc + (size_t)r * grid + o;
        double2 *p1 = acc + ((size_t)n_sub + r) * grid + o;
        const double2 v0 = *p0, v1 = *p1;
        *p0 = make_double2(v0.x + am_re, v0.y + am_im);
        *p1 = make_double2(v1.x + ap_re, v1.y + ap_im);
    }
}

__global__ void k_tables2d(int Ka, int Kb, double2 *__restrict__ tw, double2 *__restrict__ wf) {
    const int total = Ka + Kb;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int K = i < Ka ? Ka : Kb;
        const int k = i < Ka ? i : i - Ka;
        const double f = (double)k / (double)K;
        double sh, ch, s2, c2;
        sincospi(f, &sh, &ch);
        sincospi(2.0 * f, &s2, &c2);
        tw[i] = make_double2(-2.0 * sh * sh, s2);  // (cos theta - 1, sin theta)
        wf[i] = make_double2(c2, -s2);             // e^{-i theta}
    }
}

// a = acc / (count_r Ka Kb) * e^{-i (theta_1 m1_off + theta_2 m2_off)}
__global__ void k_prep2d(const double2 *__restrict__ acc, const int64_t *__restrict__ counts,
                         int n_sub, int Ka, int Kb, int64_t mo1, int64_t mo2,
                         const double2 *__restrict__ wf, double2 *__restrict__ out) {
    const int64_t grid = (int64_t)Ka * Kb;
    const int64_t total = 2 * (int64_t)n_sub * grid;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = idx % grid;
        const int r = (int)((idx / grid) % n_sub);
        const int k1 = (int)(g / Kb), k2 = (int)(g % Kb);
        const double scale = 1.0 / ((double)counts[r] * (double)grid);
        const double2 w1 = wf[(int)(((int64_t)k1 * mo1) % Ka)];
        const double2 w2 = wf[Ka + (int)(((int64_t)k2 * mo2) % Kb)];
        const double2 w = make_double2(w1.x * w2.x - w1.y * w2.y, w1.x * w2.y + w1.y * w2.x);
        const double2 a = acc[idx];
        out[idx] = make_double2((a.x * w.x - a.y * w.y) * scale, (a.x * w.y + a.y * w.x) * scale);
    }
}

// [batch][R][C] -> [batch][C][R]
__global__ void k_transpose2d(const double2 *__restrict__ x, double2 *__restrict__ y, int R,
                              int C, int64_t batch) {
    const int64_t per = (int64_t)R * C;
    const int64_t total = batch * per;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / per;
        const int64_t g = idx % per;
        const int rr = (int)(g / C), cc = (int)(g % C);
        y[b * per + (int64_t)cc * R + rr] = x[idx];
    }
}

// x: [est][r][m2][m1] -> out [P_mP | sig_mP | P_pP | sig_pP], each [m1][m2]
__global__ void k_stats2d(const double2 *__restrict__ x, int n_sub, int Ka, int Kb,
                          double *__restrict__ out) {
    const int64_t grid = (int64_t)Ka * Kb;
    const int64_t total = 2 * grid;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int est = (int)(idx / grid);
        const int64_t g = idx % grid;
        const int m1 = (int)(g / Kb), m2 = (int)(g % Kb);
        const double2 *p = x + (size_t)est * n_sub * grid + (size_t)m2 * Ka + m1;
        double mean = 0.0;
        for (int r = 0; r < n_sub; ++r) mean += p[(size_t)r * grid].x;
        mean /= (double)n_sub;
        double var = 0.0;
        for (int r = 0; r < n_sub; ++r) {
            const double d = p[(size_t)r * grid].x - mean;
            var += d * d;
        }
        const double sd = n_sub > 1 ? sqrt(var / (double)(n_sub - 1)) : 0.0;
        out[(size_t)(2 * est) * grid + g] = mean;
        out[(size_t)(2 * est + 1) * grid + g] = sd / sqrt((double)n_sub);
    }
}

int blocks2(const gbs_net *net, int64_t work) {
    int64_t b = (work + 255) / 256;
    const int64_t cap = (int64_t)net->sm_count * 8;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

int launch_finalize2d(gbs_net *net, int64_t count) {
    if (count <= 0) return GBS_OK;
    GBS_CUDA_TRY(cudaMemsetAsync(net->d_wmax2, 0xff, 4 * sizeof(int), net->stream));
    k_finalize2d<<<blocks2(net, count), 256, 0, net->stream>>>(
        net->d_nS_part, net->mtiles, net->bin_tile0, net->chunk, net->d_n, count, net->Ka,
        net->Kb, net->d_nS2, net->d_win2, net->d_wmax2);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int launch_gf2d(gbs_net *net, uint64_t e0, int64_t count) {
    if (count <= 0) return GBS_OK;
    // blocks for the whole grid; blocks past the chunk's union window return
    const int64_t cells = (int64_t)net->Ka * net->Kb;
    dim3 grid((unsigned)((cells + kG2Threads - 1) / kG2Threads), (unsigned)net->n_sub2);
    if (net->precision == GBS_FP64) {
        k_gf2d<<<grid, kG2Threads, 0, net->stream>>>(net->d_n, net->d_nS2, net->d_win2,
                                                      net->d_wmax2, count, e0, net->n_sub2,
                                                      net->Ka, net->Kb, net->d_tw2, net->d_acc2,
                                                      net->d_counts2);
    } else {
        static const DfConsts K = make_df_consts();
        k_gf2d_df<<<grid, kG2Threads, 0, net->stream>>>(net->d_n, net->d_nS2, net->d_win2,
                                                         net->d_wmax2, count, e0, net->n_sub2,
                                                         net->Ka, net->Kb, net->d_tw2, K,
                                                         net->d_acc2, net->d_counts2);
    }
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int launch_tables2d(gbs_net *net) {
    const int total = net->Ka + net->Kb;
    k_tables2d<<<(total + 255) / 256, 256, 0, net->stream>>>(net->Ka, net->Kb, net->d_tw2,
                                                              net->d_wf2);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int launch_invert2d(gbs_net *net, int64_t m1_off, int64_t m2_off, double *out_dev) {
    const int Ka = net->Ka, Kb = net->Kb;
    const int64_t grid = (int64_t)Ka * Kb;
    const int64_t batch = 2 * (int64_t)net->n_sub2;
    int64_t mo1 = m1_off % Ka, mo2 = m2_off % Kb;
    if (mo1 < 0) mo1 += Ka;
    if (mo2 < 0) mo2 += Kb;
    k_prep2d<<<blocks2(net, batch * grid), 256, 0, net->stream>>>(
        net->d_acc2, net->d_counts2, net->n_sub2, Ka, Kb, mo1, mo2, net->d_wf2, net->d_f2a);
    GBS_LAUNCH_CHECK();
    int rc;
    double2 *res = nullptr;
    // DFT along k_2 (rows of Kb), transpose, DFT along k_1 (rows of Ka)
    if ((rc = launch_fft_rows(net->d_wf2 + Ka, Kb, batch * Ka, net->d_f2a, net->d_f2b, &res,
                              net->stream, net->sm_count)))
        return rc;
    double2 *other = res == net->d_f2a ? net->d_f2b : net->d_f2a;
    k_transpose2d<<<blocks2(net, batch * grid), 256, 0, net->stream>>>(res, other, Ka, Kb, batch);
    GBS_LAUNCH_CHECK();
    double2 *spare = other == net->d_f2a ? net->d_f2b : net->d_f2a;
    if ((rc = launch_fft_rows(net->d_wf2, Ka, batch * Kb, other, spare, &res, net->stream,
                              net->sm_count)))
        return rc;
    k_stats2d<<<blocks2(net, 2 * grid), 256, 0, net->stream>>>(res, net->n_sub2, Ka, Kb, out_dev);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace gbs
