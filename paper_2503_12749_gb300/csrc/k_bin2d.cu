// Binning into d = 2..4 output bins ("Higher-dimensional binning", Eq.
// General_GCP with every output mode in one of the bins S_1 .. S_d): the
// joint distribution G(m_1, .., m_d) of the counts in the bins.
//
// Per trajectory, with n = alpha.beta and n_Sb = sum_{i in S_b} alpha'_i
// beta'_i, the bin-total projectors have the generating function
//   G_mP(z) = cosh(n + L) / cosh(n),   G_+P(z) = e^{L},
//   L = sum_b (z_b - 1) n_Sb,
// the one-bin form of Eq. c-number-variable with the exponent summed over
// the bins (the parity weight depends on the total count).  The GEMM is the
// one-bin GEMM unchanged: the rows of each bin are contiguous and padded to
// whole 64-mode tiles, so its per-tile partials sum to every n_Sb.
//
// Evaluated on a K_1 x .. x K_d grid of z_b = e^{i theta_b} in FP64 (FP64
// networks) or in double-float on the FP32 pipes (BF16 networks, the
// one-bin kernel's table-driven exp and sin/cos, FP64 for arguments beyond
// their ranges); with L = l + i phi the same stable form as the one-bin
// kernels,
//   G_mP = [e^{l + c1} e^{i phi} + e^{-l + c2} e^{-i phi}] / (1 + e^{-2|n|}),
// c1 = min(0, 2n), c2 = -2 max(n, 0).  Terms below 2^-60 are skipped with
// per-dimension windows: for the e^{L} term the window in theta_b uses the
// bound l_b(theta_b) <= -c x_b + sqrt(2c) |y_b| (c = 1 - cos theta_b) with
// the threshold raised by the largest values of the other bins' parts, and
// likewise for the e^{-L} term around (pi, .., pi).  Sub-ensemble sums are
// inverted by a d-dimensional FFT: per dimension, FFTs along the innermost
// one and a rotation that moves it outermost.
#include "gbs_internal.cuh"
#include "dfloat.cuh"

#include <cmath>

namespace gbs {
namespace {

constexpr double kTwoPi2 = 6.283185307179586476925286766559;
constexpr int kG2Threads = 128;
constexpr int kG2Tile = 128;

// Shape of one launch over the grid (passed by value).
struct GridD {
    int d;                   // bins
    int K[kMaxBins];         // points per dimension
    int Koff[kMaxBins];      // offsets of each dimension's tables
    int tile[kMaxBins + 1];  // bin b = GEMM tiles [tile[b], tile[b + 1])
};

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

__global__ void k_finalize2d(const double2 *__restrict__ part, const GridD g, int64_t ld,
                             const double *__restrict__ n, int64_t count,
                             double2 *__restrict__ nSd, WindowD *__restrict__ win,
                             int *__restrict__ wmax) {
    int m[2 * kMaxBins];
#pragma unroll
    for (int q = 0; q < 2 * kMaxBins; ++q) m[q] = -1;
    const double T = kSkipLog;
    const int d = g.d;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        double x[kMaxBins] = {}, y[kMaxBins] = {}, M1[kMaxBins] = {}, M2[kMaxBins] = {};
        double s1 = 0.0, s2 = 0.0;
#pragma unroll
        for (int b = 0; b < kMaxBins; ++b) {
            if (b >= d) continue;
            for (int t = g.tile[b]; t < g.tile[b + 1]; ++t) {
                const double2 p = part[(size_t)t * ld + i];
                x[b] += p.x;
                y[b] += p.y;
            }
            nSd[(size_t)d * i + b] = make_double2(x[b], y[b]);
            M1[b] = max_term1(x[b], y[b]);
            M2[b] = max_term2(x[b], y[b]);
            s1 += M1[b];
            s2 += M2[b];
        }
        const double c2 = -2.0 * fmax(n[i], 0.0);
        WindowD w;
        bool none2 = false;
#pragma unroll
        for (int b = 0; b < kMaxBins; ++b) {
            w.w1[b] = -1;
            w.w2[b] = -1;
            if (b < d) {
                w.w1[b] = win_term1(x[b], y[b], T + (s1 - M1[b]), g.K[b]);
                w.w2[b] = win_term2(x[b], y[b], c2 + (s2 - M2[b]), T, g.K[b]);
                none2 = none2 || w.w2[b] < 0;
            }
        }
#pragma unroll
        for (int b = 0; b < kMaxBins; ++b) {
            if (none2) w.w2[b] = -1;
            m[b] = max(m[b], w.w1[b]);
            m[kMaxBins + b] = max(m[kMaxBins + b], w.w2[b]);
        }
        win[i] = w;
    }
#pragma unroll
    for (int q = 0; q < 2 * kMaxBins; ++q) m[q] = __reduce_max_sync(0xffffffffu, m[q]);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < 2 * kMaxBins; ++q) atomicMax(&wmax[q], m[q]);
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

// Slots of the union window per dimension.
struct Slots {
    int S[kMaxBins];
    int W1[kMaxBins], W2[kMaxBins];
};

__device__ __forceinline__ Slots slots_of_grid(const GridD &g, const int *wmax) {
    Slots s;
#pragma unroll
    for (int b = 0; b < kMaxBins; ++b) {
        s.W1[b] = wmax[b];
        s.W2[b] = wmax[kMaxBins + b];
        s.S[b] = b < g.d ? slots_of(g.K[b], s.W1[b], s.W2[b]) : 1;
    }
    return s;
}

// Dimensions [0, nb) of the flattened slot index idx (last of them fastest)
// -> k_b; returns the row-major grid index over those dimensions.
__device__ __forceinline__ int64_t slot_ks(const GridD &g, const Slots &s, int nb, int64_t idx,
                                           int (&k)[kMaxBins]) {
    int64_t rem = idx;
#pragma unroll
    for (int b = kMaxBins - 1; b >= 0; --b) {
        if (b >= nb) continue;
        const int sb = (int)(rem % s.S[b]);
        rem /= s.S[b];
        k[b] = slot_k(sb, g.K[b], s.W1[b], s.W2[b]);
    }
    int64_t o = 0;
#pragma unroll
    for (int b = 0; b < kMaxBins; ++b)
        if (b < nb) o = o * g.K[b] + k[b];
    return o;
}

// One thread per slot of the union window (FP64 networks), one block row
// per sub-ensemble r; each thread adds its sub-ensemble's trajectories in
// increasing order.
__global__ void __launch_bounds__(kG2Threads)
    k_gf2d(const double *__restrict__ n_in, const double2 *__restrict__ nSd,
           const WindowD *__restrict__ win_in, const int *__restrict__ wmax, int64_t count,
           uint64_t e0, int n_sub, const GridD g, const double2 *__restrict__ tw,
           double2 *__restrict__ acc, int64_t *__restrict__ counts) {
    __shared__ double s_x[kG2Tile][kMaxBins], s_y[kG2Tile][kMaxBins];
    __shared__ double s_c1[kG2Tile], s_c2[kG2Tile], s_inv[kG2Tile];
    __shared__ WindowD s_w[kG2Tile];
    const int d = g.d;
    const int r = blockIdx.y;
    const Slots sl = slots_of_grid(g, wmax);
    int64_t total = 1;
    for (int b = 0; b < d; ++b) total *= sl.S[b];
    const int64_t slot = (int64_t)blockIdx.x * kG2Threads + threadIdx.x;
    const int64_t first = (int64_t)(((uint64_t)r + (uint64_t)n_sub - e0 % (uint64_t)n_sub) %
                                    (uint64_t)n_sub);
    const int64_t cnt_r = first < count ? (count - 1 - first) / n_sub + 1 : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[r] += cnt_r;
    if ((int64_t)blockIdx.x * kG2Threads >= total) return;  // block past the grid
    const bool valid = slot < total;
    int k[kMaxBins] = {0, 0, 0, 0}, a0[kMaxBins], api[kMaxBins];
    int64_t o = 0;
    if (valid) o = slot_ks(g, sl, d, slot, k);
    double2 t[kMaxBins];
#pragma unroll
    for (int b = 0; b < kMaxBins; ++b) {
        a0[b] = (valid && b < d) ? d0(k[b], g.K[b]) : 0;
        api[b] = (valid && b < d) ? dpi(k[b], g.K[b]) : 0;
        t[b] = b < d ? tw[g.Koff[b] + k[b]] : make_double2(0.0, 0.0);
    }
    double am_re = 0.0, am_im = 0.0, ap_re = 0.0, ap_im = 0.0;
    for (int64_t base = 0; base < cnt_r; base += kG2Tile) {
        const int64_t q = base + threadIdx.x;
        if (q < cnt_r) {
            const int64_t i = first + q * n_sub;
            const double nn = n_in[i];
#pragma unroll
            for (int b = 0; b < kMaxBins; ++b) {
                const double2 v = b < d ? nSd[(size_t)d * i + b] : make_double2(0.0, 0.0);
                s_x[threadIdx.x][b] = v.x;
                s_y[threadIdx.x][b] = v.y;
            }
            s_c1[threadIdx.x] = fmin(0.0, 2.0 * nn);
            s_c2[threadIdx.x] = -2.0 * fmax(nn, 0.0);
            s_inv[threadIdx.x] = 1.0 / (1.0 + exp(-2.0 * fabs(nn)));
            s_w[threadIdx.x] = win_in[i];
        }
        __syncthreads();
        const int ntile = (cnt_r - base) < kG2Tile ? (int)(cnt_r - base) : kG2Tile;
        if (valid) {
            for (int j = 0; j < ntile; ++j) {
                const WindowD &w = s_w[j];
                bool in1 = true, in2 = true;
#pragma unroll
                for (int b = 0; b < kMaxBins; ++b)
                    if (b < d) {
                        in1 = in1 && a0[b] <= w.w1[b];
                        in2 = in2 && api[b] <= w.w2[b];
                    }
                if (!(in1 || in2)) continue;
                double l = 0.0, ph = 0.0;
#pragma unroll
                for (int b = 0; b < kMaxBins; ++b)
                    if (b < d) {
                        l += t[b].x * s_x[j][b] - t[b].y * s_y[j][b];
                        ph += t[b].y * s_x[j][b] + t[b].x * s_y[j][b];
                    }
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
        int64_t grid = 1;
        for (int b = 0; b < d; ++b) grid *= g.K[b];
        double2 *p0 = acc + (size_t)r * grid + o;
        double2 *p1 = acc + ((size_t)n_sub + r) * grid + o;
        const double2 v0 = *p0, v1 = *p1;
        *p0 = make_double2(v0.x + am_re, v0.y + am_im);
        *p1 = make_double2(v1.x + ap_re, v1.y + ap_im);
    }
}

// The same sums in double-float arithmetic (BF16 networks), from the
// factorisation of the exponent by bins.  Bins 1..d-1 form the first factor
// (their exponents summed, their slots flattened) and bin d the second; with
// l_A + i phi_A = sum_{b<d} (z_b - 1) n_Sb and l_B + i phi_B = (z_d - 1) n_Sd,
//   e^{L}  = [e^{l_A + M_B} e^{i phi_A}] [e^{l_B - M_B} e^{i phi_B}],
//   inv e^{-L + c2} = [e^{-l_A + M'_B + c2 + log inv} e^{-i phi_A}]
//                     [e^{-l_B - M'_B} e^{-i phi_B}],
// M_B = max over theta of l_B (max_term1), M'_B = max of -l_B (max_term2),
// inv = 1 / (1 + e^{-2|n|}): every second factor is at most 1 and every
// first factor at most e^{M_A + M_B} (or e^{M'_A + M'_B + c2 + log inv}), M_A
// and M'_A the sums of the first bins' maxima.  A trajectory is therefore a
// pair of vectors per factor on a CTA's slots, and its terms on the CTA's
// tile are outer products:
//   G_+P = A_1 A_2,   G_mP = inv e^{c1} A_1 A_2 + B_1 B_2.
// Per grid point this is one or two double-float complex products instead
// of an exponential and a sine/cosine.  Factors below FP32's normal range
// (e^-87) are flushed to zero: with the exponents capped at 40 (else the
// trajectory takes the per-point FP64 route), a flushed factor drops only
// terms below e^{40 - 87} < 2^-60, the threshold of the windows.  The sums
// are kept as +P and (matrix-P - +P): the difference needs only the B_1 B_2
// term when inv e^{c1} = 1.  A trajectory's A (or B) outer product is left
// out on a tile where its largest factors multiply to below 2^-63, and
// formed in FP32 where they multiply to below 2^-25.
//
// CTA: a tile of 32 x 32 (first-factor slot, last-bin slot) of one
// sub-ensemble, 256 threads of 2 x 2 points; rounds of 16 trajectories: the
// factor vectors of the round on the tile's slots are evaluated into shared
// memory (double-float table exp and sin/cos), then each thread accumulates
// its points in double-float, renormalised every round and added to FP64
// accumulators every 4 rounds, trajectories in increasing order.
constexpr int kSepTile = 32;     // slots per factor per CTA
constexpr int kSepThreads = 256; // 16 x 16 threads, 2 x 2 points each
constexpr int kSepRound = 16;    // trajectories per round

// Per-trajectory constants of the factorised evaluation (one pass per chunk):
// the bins' n_S in double-float and the exponent offsets.
struct __align__(16) SepTraj {
    df x[kMaxBins], y[kMaxBins];  // n_Sb
    df m2, mp2;         // M_B, M'_B (offsets of the second factors)
    df o1a, o1b;        // offsets of the first factors: +M_B, +M'_B + c2 + log inv
    df rA;              // inv e^{c1} (<= 1)
    int flags;          // 2: per-point FP64 route, 4: B term used, 8: rA == 1
    int pad;
};

__global__ void k_sep_prep(const double *__restrict__ n_in, const double2 *__restrict__ nSd,
                           int64_t count, int d, SepTraj *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double nn = n_in[i];
        SepTraj st;
        double MA = 0.0, PA = 0.0, phA = 0.0, MB = 0.0, PB = 0.0, phB = 0.0;
        bool bad = false;
#pragma unroll
        for (int b = 0; b < kMaxBins; ++b) {
            const double2 v = b < d ? nSd[(size_t)d * i + b] : make_double2(0.0, 0.0);
            st.x[b] = df_from_double(v.x);
            st.y[b] = df_from_double(v.y);
            if (b >= d) continue;
            const double m1 = max_term1(v.x, v.y), m2 = max_term2(v.x, v.y);
            const double ph = fabs(v.x) + 2.0 * fabs(v.y);
            bad = bad || !(m1 >= 0.0);
            if (b < d - 1) {
                MA += m1;
                PA += m2;
                phA += ph;
            } else {
                MB = m1;
                PB = m2;
                phB = ph;
            }
        }
        const double c1 = fmin(0.0, 2.0 * nn), c2 = -2.0 * fmax(nn, 0.0);
        const double linv = -log1p(exp(-2.0 * fabs(nn)));
        const double lwB = PA + PB + c2 + linv;
        const bool big = bad || phA >= 6000.0 || phB >= 6000.0 || MA + MB > 40.0 || lwB > 40.0;
        st.m2 = df_from_double(MB);
        st.mp2 = df_from_double(PB);
        st.o1a = df_from_double(MB);
        st.o1b = df_from_double(PB + c2 + linv);
        const double rA = exp(c1 + linv);
        st.rA = df_from_double(rA);
        st.flags = (big ? 2 : 0) | (lwB >= -42.0 ? 4 : 0) | (rA == 1.0 ? 8 : 0);
        st.pad = 0;
        out[i] = st;
    }
}

// Complex double-float numbers with the real and imaginary parts side by
// side on the packed FP32x2 instructions (per lane the scalar double-float
// operations): hi = (re.hi, im.hi), lo = (re.lo, im.lo), stored as float4
// (re.hi, im.hi, re.lo, im.lo).

// The lane pairs a complex product reads of its left factor a ...
struct CLeft {
    float2 rr_hi, ii_hi, rr_lo, ii_lo;  // (re, re), (im, im) of hi and lo
};
__device__ __forceinline__ CLeft c_left(const float4 v) {
    return {f2(v.x, v.x), f2(v.y, v.y), f2(v.z, v.z), f2(v.w, v.w)};
}
// ... and of its right factor b
struct CRight {
    float2 h, hs, l, ls;  // (re, im) and (im, re) of hi and lo
};
__device__ __forceinline__ CRight c_right(const float4 v) {
    return {f2(v.x, v.y), f2(v.y, v.x), f2(v.z, v.w), f2(v.w, v.z)};
}

// unnormalised double-float complex product a b: the real part
// (ar br - ai bi) in lane x, the imaginary part (ar bi + ai br) in lane y;
// the two-products' errors and the cross terms of the low parts in FP32
__device__ __forceinline__ df2 c_mul(const CLeft &a, const CRight &b) {
    const float2 p13 = f2_mul(a.rr_hi, b.h);   // (ar br, ar bi)
    const float2 e13 = f2_fma(a.rr_hi, b.h, f2_neg(p13));
    const float2 p24 = f2_mul(a.ii_hi, b.hs);  // (ai bi, ai br)
    const float2 e24 = f2_fma(a.ii_hi, b.hs, f2_neg(p24));
    const float2 sg = f2(-1.0f, 1.0f);
    const df2 s = df2_two_sum(p13, f2_mul(p24, sg));
    const float2 l1 = f2_fma(a.rr_hi, b.l, f2_fma(a.rr_lo, b.h, e13));
    const float2 l2 = f2_fma(a.ii_hi, b.ls, f2_fma(a.ii_lo, b.hs, e24));
    return {s.hi, f2_add(f2_fma(l2, sg, l1), s.lo)};
}

// acc += t (both unnormalised)
__device__ __forceinline__ void c_acc(df2 &acc, const df2 t) {
    const df2 r = df2_two_sum(acc.hi, t.hi);
    acc = {r.hi, f2_add(f2_add(acc.lo, t.lo), r.lo)};
}

__device__ __forceinline__ df2 c_norm(const df2 a) { return df2_fast_two_sum(a.hi, a.lo); }

constexpr int kSepFlush = 4;  // rounds between additions to the FP64 sums

template <int D>
__global__ void __launch_bounds__(kSepThreads, 2)
    k_gf2d_df(const SepTraj *__restrict__ sep, const double *__restrict__ n_in,
              const double2 *__restrict__ nSd, const int *__restrict__ wmax, int64_t count,
              uint64_t e0, int n_sub, const GridD g, const double2 *__restrict__ tw,
              const DfConsts K, double2 *__restrict__ acc, int64_t *__restrict__ counts) {
    __shared__ float4 sA1[kSepRound][kSepTile], sB1[kSepRound][kSepTile];
    __shared__ float4 sA2[kSepRound][kSepTile], sB2[kSepRound][kSepTile];
    __shared__ SepTraj s_t[kSepRound];
    // the tile's twiddles: first factor [slot][component bin], second [slot]
    __shared__ df s_cmA[kSepTile][kMaxBins - 1], s_snA[kSepTile][kMaxBins - 1];
    __shared__ df s_cmB[kSepTile], s_snB[kSepTile];
    __shared__ int s_ok[2][kSepTile];
    __shared__ float s_mx[kSepRound][2][2];  // largest |factor| on the tile: [j][factor][A, B]
    __shared__ DfTables s_tab;
    constexpr int d = D;
    const int r = blockIdx.y;
    const int tid = threadIdx.x;
    const int64_t first = (int64_t)(((uint64_t)r + (uint64_t)n_sub - e0 % (uint64_t)n_sub) %
                                    (uint64_t)n_sub);
    const int64_t cnt_r = first < count ? (count - 1 - first) / n_sub + 1 : 0;
    if (blockIdx.x == 0 && tid == 0) counts[r] += cnt_r;
    const Slots sl = slots_of_grid(g, wmax);
    int64_t Sa = 1;
    for (int b = 0; b < d - 1; ++b) Sa *= sl.S[b];
    const int Sb = sl.S[d - 1];
    const int64_t nta = (Sa + kSepTile - 1) / kSepTile;
    const int ntb = (Sb + kSepTile - 1) / kSepTile;
    if ((int64_t)blockIdx.x >= nta * ntb) return;  // past the union window
    const int64_t sa0 = ((int64_t)blockIdx.x / ntb) * kSepTile;
    const int sb0 = ((int)(blockIdx.x % ntb)) * kSepTile;
    const int KB = g.K[d - 1];
    if (tid < 64) s_tab.exp2[tid] = df{K.exp2_hi[tid], K.exp2_lo[tid]};
    if (tid < 33) {
        s_tab.sn[tid] = df{K.sin_hi[tid], K.sin_lo[tid]};
        s_tab.cs[tid] = df{K.cos_hi[tid], K.cos_lo[tid]};
    }
    if (tid < kSepTile) {
        const int64_t s = sa0 + tid;
        const bool ok = s < Sa;
        int k[kMaxBins] = {0, 0, 0, 0};
        if (ok) slot_ks(g, sl, d - 1, s, k);
#pragma unroll
        for (int b = 0; b < kMaxBins - 1; ++b) {
            const double2 t = b < d - 1 ? tw[g.Koff[b] + k[b]] : make_double2(0.0, 0.0);
            s_cmA[tid][b] = df_from_double(t.x);
            s_snA[tid][b] = df_from_double(t.y);
        }
        s_ok[0][tid] = ok;
    } else if (tid < 2 * kSepTile) {
        const int j2 = tid - kSepTile;
        const int s = sb0 + j2;
        const bool ok = s < Sb;
        const int kk = ok ? slot_k(s, KB, sl.W1[d - 1], sl.W2[d - 1]) : 0;
        const double2 t = tw[g.Koff[d - 1] + kk];
        s_cmB[j2] = df_from_double(t.x);
        s_snB[j2] = df_from_double(t.y);
        s_ok[1][j2] = ok;
    }
    // this thread's points: first-factor slots sa0 + 2 ty + p, last-bin
    // slots sb0 + 2 tx + q
    const int tx = tid & 15, ty = tid >> 4;
    int64_t oA[2];
    int kB[2];
    bool v1[2], v2[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int64_t sa = sa0 + 2 * ty + p;
        const int sb = sb0 + 2 * tx + p;
        v1[p] = sa < Sa;
        v2[p] = sb < Sb;
        int k[kMaxBins] = {0, 0, 0, 0};
        oA[p] = v1[p] ? slot_ks(g, sl, d - 1, sa, k) : 0;
        kB[p] = v2[p] ? slot_k(sb, KB, sl.W1[d - 1], sl.W2[d - 1]) : 0;
    }
    double dP[2][2][2] = {}, dX[2][2][2] = {};  // +P and (matrix-P - +P), (re, im)
    df2 aP[2][2], aX[2][2];  // double-float sums (re, im side by side)
    float2 fP[2][2], fX[2][2];  // FP32 sums of the terms below 2^-24
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            aP[p][q] = {f2(0.f, 0.f), f2(0.f, 0.f)};
            aX[p][q] = aP[p][q];
            fP[p][q] = make_float2(0.f, 0.f);
            fX[p][q] = fP[p][q];
        }

    int round = 0;
    for (int64_t base = 0; base < cnt_r; base += kSepRound, ++round) {
        const int nr = (int)((cnt_r - base) < kSepRound ? (cnt_r - base) : kSepRound);
        if (tid < kSepRound) {
            SepTraj st = {};
            st.flags = 2 | 16;  // 16: no trajectory
            if (tid < nr) st = sep[first + (base + tid) * n_sub];
            s_t[tid] = st;
        }
        __syncthreads();
        // factor vectors of the round on the tile's slots: item =
        // (trajectory, factor, slot); A and B share l, phi and the sine/cosine
        for (int it = tid; it < kSepRound * 2 * kSepTile; it += kSepThreads) {
            const int j = it / (2 * kSepTile);
            const int fac = (it / kSepTile) & 1;
            const int sidx = it % kSepTile;
            const SepTraj &st = s_t[j];
            float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A;
            if (!(st.flags & 2) && s_ok[fac][sidx]) {
                df l = {0.f, 0.f}, ph = {0.f, 0.f};
                if (fac == 0) {
#pragma unroll
                    for (int b = 0; b < d - 1; ++b) {
                        const df cm1 = s_cmA[sidx][b], sn = s_snA[sidx][b];
                        const df lb = df_sub(df_mul(cm1, st.x[b]), df_mul(sn, st.y[b]));
                        const df pb = df_add(df_mul(sn, st.x[b]), df_mul(cm1, st.y[b]));
                        l = b == 0 ? lb : df_add(l, lb);
                        ph = b == 0 ? pb : df_add(ph, pb);
                    }
                } else {
                    const df cm1 = s_cmB[sidx], sn = s_snB[sidx];
                    l = df_sub(df_mul(cm1, st.x[d - 1]), df_mul(sn, st.y[d - 1]));
                    ph = df_add(df_mul(sn, st.x[d - 1]), df_mul(cm1, st.y[d - 1]));
                }
                df sp, cp;
                df_sincos_tab(ph, s_tab, K, sp, cp);
                // exponents: first factor: l + M_B and -l + M'_B + c2 + log inv;
                // second: l - M_B and -l - M'_B
                const df ea = fac == 0 ? df_add(l, st.o1a) : df_sub(l, st.m2);
                const df eb = fac == 0 ? df_sub(st.o1b, l) : df_sub(df_neg(l), st.mp2);
                if (ea.hi >= -87.0f) {
                    const df e = df_exp_tab(ea, s_tab, K);
                    const df re = df_mul(e, cp), im = df_mul(e, sp);
                    A = make_float4(re.hi, im.hi, re.lo, im.lo);
                }
                if ((st.flags & 4) && eb.hi >= -87.0f) {
                    const df e = df_exp_tab(eb, s_tab, K);
                    const df re = df_mul(e, cp), im = df_mul(e, sp);
                    B = make_float4(re.hi, -im.hi, re.lo, -im.lo);
                }
            }
            if (fac == 0) {
                sA1[j][sidx] = A;
                sB1[j][sidx] = B;
            } else {
                sA2[j][sidx] = A;
                sB2[j][sidx] = B;
            }
            // the 32 slots of one (trajectory, factor) are one warp's items
            const unsigned ma = __float_as_uint(fmaxf(fabsf(A.x), fabsf(A.y)));
            const unsigned mb = __float_as_uint(fmaxf(fabsf(B.x), fabsf(B.y)));
            const unsigned wa = __reduce_max_sync(0xffffffffu, ma);
            const unsigned wb = __reduce_max_sync(0xffffffffu, mb);
            if (sidx == 0) {
                s_mx[j][fac][0] = __uint_as_float(wa);
                s_mx[j][fac][1] = __uint_as_float(wb);
            }
        }
        __syncthreads();
        for (int j = 0; j < nr; ++j) {
            const int flags = s_t[j].flags;
            if (flags & 2) {
                // per-point FP64 route (huge phases or exponents)
                const int64_t i = first + (base + j) * n_sub;
                const double nn = n_in[i];
                const double c1d = fmin(0.0, 2.0 * nn), c2d = -2.0 * fmax(nn, 0.0);
                const double inv = 1.0 / (1.0 + exp(-2.0 * fabs(nn)));
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        if (!(v1[p] && v2[q])) continue;
                        double ld = 0.0, pd = 0.0;
                        int64_t rem = oA[p];  // row-major over the first d - 1 bins
#pragma unroll
                        for (int b = d - 1; b >= 0; --b) {
                            int kb;
                            if (b == d - 1) {
                                kb = kB[q];
                            } else {
                                kb = (int)(rem % g.K[b]);
                                rem /= g.K[b];
                            }
                            const double2 t = tw[g.Koff[b] + kb];
                            const double2 v = nSd[(size_t)d * i + b];
                            ld += t.x * v.x - t.y * v.y;
                            pd += t.y * v.x + t.x * v.y;
                        }
                        double sd, cd;
                        sincos(pd, &sd, &cd);
                        const double gp = ld >= -745.0 ? exp(ld) : 0.0;
                        const double e1 = ld + c1d >= -745.0 ? exp(ld + c1d) : 0.0;
                        const double e2 = -ld + c2d >= -745.0 ? exp(-ld + c2d) : 0.0;
                        const double mre = (e1 + e2) * cd * inv, mim = (e1 - e2) * sd * inv;
                        dP[p][q][0] += gp * cd;
                        dP[p][q][1] += gp * sd;
                        dX[p][q][0] += mre - gp * cd;
                        dX[p][q][1] += mim - gp * sd;
                    }
                continue;
            }
            // a term whose largest product on the tile is below 2^-63 (so
            // every complex product below 2^-62) is left out, as the windows
            // leave out terms below 2^-60; below 2^-25 (products below
            // 2^-24) it is formed and summed in FP32, whose rounding
            // (< 2^-48 per term) is far below the double-float needs of the
            // large terms
            const float mA = s_mx[j][0][0] * s_mx[j][1][0];
            const float mB = (flags & 4) ? s_mx[j][0][1] * s_mx[j][1][1] : 0.0f;
            const bool rA1 = (flags & 8) != 0;
            if (mA >= 0x1p-63f && mA < 0x1p-25f) {
                const float4 A1[2] = {sA1[j][2 * ty], sA1[j][2 * ty + 1]};
                const float4 A2[2] = {sA2[j][2 * tx], sA2[j][2 * tx + 1]};
                const float rm1 = rA1 ? 0.0f : s_t[j].rA.hi - 1.0f + s_t[j].rA.lo;
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float tr = fmaf(A1[p].x, A2[q].x, -A1[p].y * A2[q].y);
                        const float ti = fmaf(A1[p].x, A2[q].y, A1[p].y * A2[q].x);
                        fP[p][q].x += tr;
                        fP[p][q].y += ti;
                        if (!rA1) {
                            fX[p][q].x = fmaf(rm1, tr, fX[p][q].x);
                            fX[p][q].y = fmaf(rm1, ti, fX[p][q].y);
                        }
                    }
            } else if (mA >= 0x1p-25f) {
                const CLeft L[2] = {c_left(sA1[j][2 * ty]), c_left(sA1[j][2 * ty + 1])};
                const CRight R[2] = {c_right(sA2[j][2 * tx]), c_right(sA2[j][2 * tx + 1])};
                const df rAm1 = rA1 ? df{0.f, 0.f} : df_add_f(s_t[j].rA, -1.0f);
                const df2 rAm1x2 = df2_make(rAm1, rAm1);
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const df2 t = c_mul(L[p], R[q]);
                        c_acc(aP[p][q], t);
                        // the matrix-P A term is rA t: (rA - 1) t into the difference
                        if (!rA1) c_acc(aX[p][q], df2_mul(t, rAm1x2));
                    }
            }
            if (mB >= 0x1p-63f) {
                const float4 B1[2] = {sB1[j][2 * ty], sB1[j][2 * ty + 1]};
                const float4 B2[2] = {sB2[j][2 * tx], sB2[j][2 * tx + 1]};
                if (mB < 0x1p-25f) {
#pragma unroll
                    for (int p = 0; p < 2; ++p)
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            fX[p][q].x = fmaf(B1[p].x, B2[q].x, fmaf(-B1[p].y, B2[q].y, fX[p][q].x));
                            fX[p][q].y = fmaf(B1[p].x, B2[q].y, fmaf(B1[p].y, B2[q].x, fX[p][q].y));
                        }
                } else {
                    const CLeft L[2] = {c_left(B1[0]), c_left(B1[1])};
                    const CRight R[2] = {c_right(B2[0]), c_right(B2[1])};
#pragma unroll
                    for (int p = 0; p < 2; ++p)
#pragma unroll
                        for (int q = 0; q < 2; ++q) c_acc(aX[p][q], c_mul(L[p], R[q]));
                }
            }
        }
        // renormalise every round, add to the FP64 sums every kSepFlush rounds
        const bool flush = (round + 1) % kSepFlush == 0 || base + kSepRound >= cnt_r;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                aP[p][q] = c_norm(aP[p][q]);
                aX[p][q] = c_norm(aX[p][q]);
                if (flush) {
                    dP[p][q][0] += (double)aP[p][q].hi.x + (double)aP[p][q].lo.x + (double)fP[p][q].x;
                    dP[p][q][1] += (double)aP[p][q].hi.y + (double)aP[p][q].lo.y + (double)fP[p][q].y;
                    dX[p][q][0] += (double)aX[p][q].hi.x + (double)aX[p][q].lo.x + (double)fX[p][q].x;
                    dX[p][q][1] += (double)aX[p][q].hi.y + (double)aX[p][q].lo.y + (double)fX[p][q].y;
                    aP[p][q] = {f2(0.f, 0.f), f2(0.f, 0.f)};
                    aX[p][q] = aP[p][q];
                    fP[p][q] = make_float2(0.f, 0.f);
                    fX[p][q] = fP[p][q];
                }
            }
        __syncthreads();
    }
    int64_t grid = 1;
    for (int b = 0; b < d; ++b) grid *= g.K[b];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (!(v1[p] && v2[q])) continue;
            const size_t o = (size_t)oA[p] * KB + kB[q];
            double2 *pm = acc + (size_t)r * grid + o;
            double2 *pp = acc + ((size_t)n_sub + r) * grid + o;
            const double2 vm = *pm, vp = *pp;
            *pm = make_double2(vm.x + (dP[p][q][0] + dX[p][q][0]), vm.y + (dP[p][q][1] + dX[p][q][1]));
            *pp = make_double2(vp.x + dP[p][q][0], vp.y + dP[p][q][1]);
        }
}

__global__ void k_tables2d(const GridD g, int total, double2 *__restrict__ tw,
                           double2 *__restrict__ wf) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int b = 0;
        while (b + 1 < g.d && i >= g.Koff[b + 1]) ++b;
        const int K = g.K[b];
        const int k = i - g.Koff[b];
        const double f = (double)k / (double)K;
        double sh, ch, s2, c2;
        sincospi(f, &sh, &ch);
        sincospi(2.0 * f, &s2, &c2);
        tw[i] = make_double2(-2.0 * sh * sh, s2);  // (cos theta - 1, sin theta)
        wf[i] = make_double2(c2, -s2);             // e^{-i theta}
    }
}

// a = acc / (count_r prod K) * e^{-i sum_b theta_b m_off_b}
__global__ void k_prep2d(const double2 *__restrict__ acc, const int64_t *__restrict__ counts,
                         int n_sub, const GridD g, int64_t grid, const int64_t *__restrict__ mo,
                         const double2 *__restrict__ wf, double2 *__restrict__ out) {
    const int64_t total = 2 * (int64_t)n_sub * grid;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t gi = idx % grid;
        const int r = (int)((idx / grid) % n_sub);
        const double scale = 1.0 / ((double)counts[r] * (double)grid);
        double2 w = make_double2(1.0, 0.0);
        for (int b = g.d - 1; b >= 0; --b) {
            const int k = (int)(gi % g.K[b]);
            gi /= g.K[b];
            const double2 wb = wf[g.Koff[b] + (int)(((int64_t)k * mo[b]) % g.K[b])];
            w = make_double2(w.x * wb.x - w.y * wb.y, w.x * wb.y + w.y * wb.x);
        }
        const double2 a = acc[idx];
        out[idx] = make_double2((a.x * w.x - a.y * w.y) * scale, (a.x * w.y + a.y * w.x) * scale);
    }
}

// [batch][R][C] -> [batch][C][R]
__global__ void k_transpose2d(const double2 *__restrict__ x, double2 *__restrict__ y, int64_t R,
                              int C, int64_t batch) {
    const int64_t per = R * C;
    const int64_t total = batch * per;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / per;
        const int64_t gidx = idx % per;
        const int64_t rr = gidx / C;
        const int cc = (int)(gidx % C);
        y[b * per + (int64_t)cc * R + rr] = x[idx];
    }
}

// x: [est][r][grid] -> out [P_mP | sig_mP | P_pP | sig_pP], each [grid]
__global__ void k_stats2d(const double2 *__restrict__ x, int n_sub, int64_t grid,
                          double *__restrict__ out) {
    const int64_t total = 2 * grid;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int est = (int)(idx / grid);
        const int64_t gi = idx % grid;
        const double2 *p = x + (size_t)est * n_sub * grid + gi;
        double mean = 0.0;
        for (int r = 0; r < n_sub; ++r) mean += p[(size_t)r * grid].x;
        mean /= (double)n_sub;
        double var = 0.0;
        for (int r = 0; r < n_sub; ++r) {
            const double dd = p[(size_t)r * grid].x - mean;
            var += dd * dd;
        }
        const double sd = n_sub > 1 ? sqrt(var / (double)(n_sub - 1)) : 0.0;
        out[(size_t)(2 * est) * grid + gi] = mean;
        out[(size_t)(2 * est + 1) * grid + gi] = sd / sqrt((double)n_sub);
    }
}

int blocks2(const gbs_net *net, int64_t work) {
    int64_t b = (work + 255) / 256;
    const int64_t cap = (int64_t)net->sm_count * 8;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

GridD grid_of(const gbs_net *net) {
    GridD g = {};
    g.d = net->nbins;
    int off = 0;
    for (int b = 0; b < kMaxBins; ++b) {
        g.K[b] = b < g.d ? net->Kd[b] : 1;
        g.Koff[b] = off;
        if (b < g.d) off += net->Kd[b];
    }
    for (int b = 0; b <= kMaxBins; ++b) g.tile[b] = net->bin_tiles[b];
    return g;
}

}  // namespace

size_t sep2_bytes_per_trajectory() { return sizeof(SepTraj); }

int launch_finalize2d(gbs_net *net, int64_t count) {
    if (count <= 0) return GBS_OK;
    GBS_CUDA_TRY(cudaMemsetAsync(net->d_wmax2, 0xff, 2 * kMaxBins * sizeof(int), net->stream));
    k_finalize2d<<<blocks2(net, count), 256, 0, net->stream>>>(
        net->d_nS_part, grid_of(net), net->chunk, net->d_n, count, net->d_nS2, net->d_win2,
        net->d_wmax2);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int launch_gf2d(gbs_net *net, uint64_t e0, int64_t count) {
    if (count <= 0) return GBS_OK;
    const GridD g = grid_of(net);
    if (simt_precision(net->precision)) {
        // blocks for the whole grid; blocks past the chunk's union window return
        dim3 grid((unsigned)((net->grid2 + kG2Threads - 1) / kG2Threads), (unsigned)net->n_sub2);
        k_gf2d<<<grid, kG2Threads, 0, net->stream>>>(net->d_n, net->d_nS2, net->d_win2,
                                                      net->d_wmax2, count, e0, net->n_sub2, g,
                                                      net->d_tw2, net->d_acc2, net->d_counts2);
    } else {
        static const DfConsts K = make_df_consts();
        // tiles of 32 x 32 slots over the whole grid; tiles past the chunk's
        // union window return at once
        const int KB = net->Kd[net->nbins - 1];
        const int64_t KA = net->grid2 / KB;
        const int64_t tiles = ((KA + kSepTile - 1) / kSepTile) * ((KB + kSepTile - 1) / kSepTile);
        dim3 g2((unsigned)tiles, (unsigned)net->n_sub2);
        SepTraj *sep = static_cast<SepTraj *>(net->d_sep2);
        k_sep_prep<<<blocks2(net, count), 256, 0, net->stream>>>(net->d_n, net->d_nS2, count,
                                                                 net->nbins, sep);
        GBS_LAUNCH_CHECK();
        auto kern = net->nbins == 2 ? k_gf2d_df<2> : net->nbins == 3 ? k_gf2d_df<3> : k_gf2d_df<4>;
        kern<<<g2, kSepThreads, 0, net->stream>>>(sep, net->d_n, net->d_nS2, net->d_wmax2, count,
                                                   e0, net->n_sub2, g, net->d_tw2, K, net->d_acc2,
                                                   net->d_counts2);
    }
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int launch_tables2d(gbs_net *net) {
    const GridD g = grid_of(net);
    int total = 0;
    for (int b = 0; b < g.d; ++b) total += g.K[b];
    k_tables2d<<<(total + 255) / 256, 256, 0, net->stream>>>(g, total, net->d_tw2, net->d_wf2);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int launch_invert2d(gbs_net *net, const int64_t *m_off, double *out_dev, int *launches) {
    const GridD g = grid_of(net);
    const int64_t grid = net->grid2;
    const int64_t batch = 2 * (int64_t)net->n_sub2;
    int64_t mo[kMaxBins] = {0, 0, 0, 0};
    for (int b = 0; b < g.d; ++b) {
        mo[b] = m_off[b] % g.K[b];
        if (mo[b] < 0) mo[b] += g.K[b];
    }
    // pageable source: the copy is staged before the call returns
    GBS_CUDA_TRY(cudaMemcpyAsync(net->d_mo2, mo, sizeof(mo), cudaMemcpyHostToDevice, net->stream));
    k_prep2d<<<blocks2(net, batch * grid), 256, 0, net->stream>>>(
        net->d_acc2, net->d_counts2, net->n_sub2, g, grid, net->d_mo2, net->d_wf2, net->d_f2a);
    GBS_LAUNCH_CHECK();
    int nl = 1;
    double2 *cur = net->d_f2a;
    // per dimension, innermost first: FFTs along it, then rotate it outermost
    for (int b = g.d - 1; b >= 0; --b) {
        double2 *other = cur == net->d_f2a ? net->d_f2b : net->d_f2a;
        double2 *res = nullptr;
        int rc;
        if ((rc = launch_fft_rows(net->d_wf2 + g.Koff[b], g.K[b], batch * (grid / g.K[b]), cur,
                                  other, &res, net->stream, net->sm_count)))
            return rc;
        for (int v = g.K[b]; v > 1; v >>= 1) ++nl;
        double2 *dst = res == net->d_f2a ? net->d_f2b : net->d_f2a;
        k_transpose2d<<<blocks2(net, batch * grid), 256, 0, net->stream>>>(res, dst, grid / g.K[b],
                                                                            g.K[b], batch);
        GBS_LAUNCH_CHECK();
        ++nl;
        cur = dst;
    }
    k_stats2d<<<blocks2(net, 2 * grid), 256, 0, net->stream>>>(cur, net->n_sub2, grid, out_dev);
    GBS_LAUNCH_CHECK();
    ++nl;
    if (launches) *launches = nl;
    return GBS_OK;
}

}  // namespace gbs
