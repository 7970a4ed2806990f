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

// The same sums in double-float arithmetic (BF16 networks), from the
// factorisation of the exponent by bins.  With l_b + i phi_b = (z_b - 1) n_Sb,
//   e^{L}  = [e^{l_1 + M_2} e^{i phi_1}] [e^{l_2 - M_2} e^{i phi_2}],
//   inv e^{-L + c2} = [e^{-l_1 + M'_2 + c2 + log inv} e^{-i phi_1}]
//                     [e^{-l_2 - M'_2} e^{-i phi_2}],
// M_b = max over theta of l_b (max_term1), M'_b = max of -l_b (max_term2),
// inv = 1 / (1 + e^{-2|n|}): every bin-2 factor is at most 1 and every
// bin-1 factor at most e^{M_1 + M_2} (or e^{M'_1 + M'_2 + c2 + log inv}).
// A trajectory is therefore a pair of vectors per bin on the CTA's slots, and
// its terms on the CTA's (k_1, k_2) tile are outer products:
//   G_+P = A_1 A_2,   G_mP = inv e^{c1} A_1 A_2 + B_1 B_2.
// Per pair this is one or two double-float complex products instead of an
// exponential and a sine/cosine.  Factors below FP32's normal range (e^-87)
// are flushed to zero: with the exponents capped at 40 (else the trajectory
// takes the per-pair FP64 route), a flushed factor drops only terms below
// e^{40 - 87} < 2^-60, the threshold of the windows.  The sums are kept as
// +P and (matrix-P - +P): the difference needs only the B_1 B_2 term when
// inv e^{c1} = 1.
//
// A trajectory's A (or B) outer product is left out on a tile where its
// largest factors multiply to below 2^-63, and formed in FP32 where they
// multiply to below 2^-25.
// CTA: a tile of 32 x 32 (k_1, k_2) slots of one sub-ensemble, 256 threads of
// 2 x 2 pairs; rounds of 16 trajectories: the bin vectors of the round on the
// tile's slots are evaluated into shared memory (double-float table exp and
// sin/cos), then each thread accumulates its pairs in double-float and adds
// the round to FP64 accumulators, trajectories in increasing order.
constexpr int kSepTile = 32;     // slots per bin per CTA
constexpr int kSepThreads = 256; // 16 x 16 threads, 2 x 2 pairs each
constexpr int kSepRound = 16;    // trajectories per round

// Per-trajectory constants of the factorised evaluation (one pass per chunk):
// the bins' n_S in double-float and the exponent offsets.
struct __align__(16) SepTraj {
    df x1, y1, x2, y2;  // n_S1, n_S2
    df m2, mp2;         // M_2, M'_2 (offsets of the bin-2 factors)
    df o1a, o1b;        // offsets of the bin-1 factors: +M_2, +M'_2 + c2 + log inv
    df rA;              // inv e^{c1} (<= 1)
    int flags;          // 2: per-pair FP64 route, 4: B term used, 8: rA == 1
    int pad;
};

__global__ void k_sep_prep(const double *__restrict__ n_in, const double2 *__restrict__ nS2,
                           int64_t count, SepTraj *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double nn = n_in[i];
        const double2 a = nS2[2 * i], b = nS2[2 * i + 1];
        const double M1 = max_term1(a.x, a.y), M2 = max_term1(b.x, b.y);
        const double P1 = max_term2(a.x, a.y), P2 = max_term2(b.x, b.y);
        const double c1 = fmin(0.0, 2.0 * nn), c2 = -2.0 * fmax(nn, 0.0);
        const double linv = -log1p(exp(-2.0 * fabs(nn)));
        const double lwB = P1 + P2 + c2 + linv;
        const bool big = fabs(a.x) + 2.0 * fabs(a.y) >= 6000.0 ||
                         fabs(b.x) + 2.0 * fabs(b.y) >= 6000.0 || M1 + M2 > 40.0 || lwB > 40.0 ||
                         !(M1 + M2 >= 0.0);
        SepTraj st;
        st.x1 = df_from_double(a.x);
        st.y1 = df_from_double(a.y);
        st.x2 = df_from_double(b.x);
        st.y2 = df_from_double(b.y);
        st.m2 = df_from_double(M2);
        st.mp2 = df_from_double(P2);
        st.o1a = df_from_double(M2);
        st.o1b = df_from_double(P2 + c2 + linv);
        const double rA = exp(c1 + linv);
        st.rA = df_from_double(rA);
        st.flags = (big ? 2 : 0) | (lwB >= -42.0 ? 4 : 0) | (rA == 1.0 ? 8 : 0);
        st.pad = 0;
        out[i] = st;
    }
}

// unnormalised double-float complex product a b: (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ float4 dfc_mul(const float4 a, const float4 b) {
    const float p1 = a.x * b.x, e1 = fmaf(a.x, b.x, -p1);
    const float p2 = a.z * b.z, e2 = fmaf(a.z, b.z, -p2);
    const df sr = df_two_sum(p1, -p2);
    const float lr = fmaf(a.x, b.y, fmaf(a.y, b.x, e1)) - fmaf(a.z, b.w, fmaf(a.w, b.z, e2)) + sr.lo;
    const float p3 = a.x * b.z, e3 = fmaf(a.x, b.z, -p3);
    const float p4 = a.z * b.x, e4 = fmaf(a.z, b.x, -p4);
    const df si = df_two_sum(p3, p4);
    const float li = fmaf(a.x, b.w, fmaf(a.y, b.z, e3)) + fmaf(a.z, b.y, fmaf(a.w, b.x, e4)) + si.lo;
    return make_float4(sr.hi, lr, si.hi, li);
}

// acc += t (both unnormalised double-float complex)
__device__ __forceinline__ void dfc_acc(float4 &acc, const float4 t) {
    const df r = df_two_sum(acc.x, t.x);
    const df i = df_two_sum(acc.z, t.z);
    acc = make_float4(r.hi, acc.y + t.y + r.lo, i.hi, acc.w + t.w + i.lo);
}

__device__ __forceinline__ float4 dfc_scale(const float4 a, const df s) {
    const df re = df_mul(df{a.x, a.y}, s), im = df_mul(df{a.z, a.w}, s);
    return make_float4(re.hi, re.lo, im.hi, im.lo);
}

__device__ __forceinline__ float4 dfc_norm(const float4 a) {
    const df re = df_fast_two_sum(a.x, a.y), im = df_fast_two_sum(a.z, a.w);
    return make_float4(re.hi, re.lo, im.hi, im.lo);
}

constexpr int kSepFlush = 4;  // rounds between additions to the FP64 sums

__global__ void __launch_bounds__(kSepThreads, 2)
    k_gf2d_df(const SepTraj *__restrict__ sep, const double *__restrict__ n_in,
              const double2 *__restrict__ nS2, const int *__restrict__ wmax, int64_t count,
              uint64_t e0, int n_sub, int Ka, int Kb, const double2 *__restrict__ tw,
              const DfConsts K, double2 *__restrict__ acc, int64_t *__restrict__ counts) {
    __shared__ float4 sA1[kSepRound][kSepTile], sB1[kSepRound][kSepTile];
    __shared__ float4 sA2[kSepRound][kSepTile], sB2[kSepRound][kSepTile];
    __shared__ SepTraj s_t[kSepRound];
    __shared__ df s_cm[2][kSepTile], s_sn[2][kSepTile];  // the tile's twiddles per bin
    __shared__ int s_ok[2][kSepTile];
    __shared__ float s_mx[kSepRound][2][2];  // largest |factor| on the tile: [j][bin][A, B]
    __shared__ DfTables s_tab;
    const int r = blockIdx.y;
    const int tid = threadIdx.x;
    const int64_t first = (int64_t)(((uint64_t)r + (uint64_t)n_sub - e0 % (uint64_t)n_sub) %
                                    (uint64_t)n_sub);
    const int64_t cnt_r = first < count ? (count - 1 - first) / n_sub + 1 : 0;
    if (blockIdx.x == 0 && tid == 0) counts[r] += cnt_r;
    const int W1a = wmax[0], W1b = wmax[1], W2a = wmax[2], W2b = wmax[3];
    const int Sa = slots_of(Ka, W1a, W2a), Sb = slots_of(Kb, W1b, W2b);
    const int nta = (Sa + kSepTile - 1) / kSepTile, ntb = (Sb + kSepTile - 1) / kSepTile;
    if ((int)blockIdx.x >= nta * ntb) return;  // past the union window
    const int sa0 = (blockIdx.x / ntb) * kSepTile, sb0 = (blockIdx.x % ntb) * kSepTile;
    if (tid < 64) s_tab.exp2[tid] = df{K.exp2_hi[tid], K.exp2_lo[tid]};
    if (tid < 33) {
        s_tab.sn[tid] = df{K.sin_hi[tid], K.sin_lo[tid]};
        s_tab.cs[tid] = df{K.cos_hi[tid], K.cos_lo[tid]};
    }
    if (tid < 2 * kSepTile) {
        const int bin = tid / kSepTile, sl = tid % kSepTile;
        const int slot = (bin == 0 ? sa0 : sb0) + sl;
        const bool ok = slot < (bin == 0 ? Sa : Sb);
        const int kk = !ok ? 0 : (bin == 0 ? slot_k(slot, Ka, W1a, W2a) : slot_k(slot, Kb, W1b, W2b));
        const double2 t = tw[(bin == 0 ? 0 : Ka) + kk];
        s_cm[bin][sl] = df_from_double(t.x);
        s_sn[bin][sl] = df_from_double(t.y);
        s_ok[bin][sl] = ok;
    }
    // this thread's pairs: bin-1 slots sa0 + 2 ty + p, bin-2 slots sb0 + 2 tx + q
    const int tx = tid & 15, ty = tid >> 4;
    int k1[2], k2[2];
    bool v1[2], v2[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int sa = sa0 + 2 * ty + p, sb = sb0 + 2 * tx + p;
        v1[p] = sa < Sa;
        v2[p] = sb < Sb;
        k1[p] = v1[p] ? slot_k(sa, Ka, W1a, W2a) : 0;
        k2[p] = v2[p] ? slot_k(sb, Kb, W1b, W2b) : 0;
    }
    double dP[2][2][2] = {}, dX[2][2][2] = {};  // +P and (matrix-P - +P), (re, im)
    float4 aP[2][2], aX[2][2];  // double-float sums
    float2 fP[2][2], fX[2][2];  // FP32 sums of the terms below 2^-24
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            aP[p][q] = make_float4(0.f, 0.f, 0.f, 0.f);
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
        // bin vectors of the round on the tile's slots: item = (trajectory,
        // bin, slot); A and B share l, phi and the sine/cosine
        for (int it = tid; it < kSepRound * 2 * kSepTile; it += kSepThreads) {
            const int j = it / (2 * kSepTile);
            const int bin = (it / kSepTile) & 1;
            const int sl = it % kSepTile;
            const SepTraj &st = s_t[j];
            float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A;
            if (!(st.flags & 2) && s_ok[bin][sl]) {
                const df cm1 = s_cm[bin][sl], sn = s_sn[bin][sl];
                const df x = bin == 0 ? st.x1 : st.x2, y = bin == 0 ? st.y1 : st.y2;
                const df l = df_sub(df_mul(cm1, x), df_mul(sn, y));
                const df ph = df_add(df_mul(sn, x), df_mul(cm1, y));
                df sp, cp;
                df_sincos_tab(ph, s_tab, K, sp, cp);
                // exponents: bin 1: l + M_2 and -l + M'_2 + c2 + log inv;
                // bin 2: l - M_2 and -l - M'_2
                const df ea = bin == 0 ? df_add(l, st.o1a) : df_sub(l, st.m2);
                const df eb = bin == 0 ? df_sub(st.o1b, l) : df_sub(df_neg(l), st.mp2);
                if (ea.hi >= -87.0f) {
                    const df e = df_exp_tab(ea, s_tab, K);
                    const df re = df_mul(e, cp), im = df_mul(e, sp);
                    A = make_float4(re.hi, re.lo, im.hi, im.lo);
                }
                if ((st.flags & 4) && eb.hi >= -87.0f) {
                    const df e = df_exp_tab(eb, s_tab, K);
                    const df re = df_mul(e, cp), im = df_mul(e, sp);
                    B = make_float4(re.hi, re.lo, -im.hi, -im.lo);
                }
            }
            if (bin == 0) {
                sA1[j][sl] = A;
                sB1[j][sl] = B;
            } else {
                sA2[j][sl] = A;
                sB2[j][sl] = B;
            }
            // the 32 slots of one (trajectory, bin) are one warp's items
            const unsigned ma = __float_as_uint(fmaxf(fabsf(A.x), fabsf(A.z)));
            const unsigned mb = __float_as_uint(fmaxf(fabsf(B.x), fabsf(B.z)));
            const unsigned wa = __reduce_max_sync(0xffffffffu, ma);
            const unsigned wb = __reduce_max_sync(0xffffffffu, mb);
            if (sl == 0) {
                s_mx[j][bin][0] = __uint_as_float(wa);
                s_mx[j][bin][1] = __uint_as_float(wb);
            }
        }
        __syncthreads();
        for (int j = 0; j < nr; ++j) {
            const int flags = s_t[j].flags;
            if (flags & 2) {
                // per-pair FP64 route (huge phases or exponents)
                const int64_t i = first + (base + j) * n_sub;
                const double nn = n_in[i];
                const double2 a = nS2[2 * i], b = nS2[2 * i + 1];
                const double c1d = fmin(0.0, 2.0 * nn), c2d = -2.0 * fmax(nn, 0.0);
                const double inv = 1.0 / (1.0 + exp(-2.0 * fabs(nn)));
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        if (!(v1[p] && v2[q])) continue;
                        const double2 ta = tw[k1[p]], tb = tw[Ka + k2[q]];
                        const double ld = (ta.x * a.x - ta.y * a.y) + (tb.x * b.x - tb.y * b.y);
                        const double pd = (ta.y * a.x + ta.x * a.y) + (tb.y * b.x + tb.x * b.y);
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
                        const float tr = fmaf(A1[p].x, A2[q].x, -A1[p].z * A2[q].z);
                        const float ti = fmaf(A1[p].x, A2[q].z, A1[p].z * A2[q].x);
                        fP[p][q].x += tr;
                        fP[p][q].y += ti;
                        if (!rA1) {
                            fX[p][q].x = fmaf(rm1, tr, fX[p][q].x);
                            fX[p][q].y = fmaf(rm1, ti, fX[p][q].y);
                        }
                    }
            } else if (mA >= 0x1p-25f) {
                const float4 A1[2] = {sA1[j][2 * ty], sA1[j][2 * ty + 1]};
                const float4 A2[2] = {sA2[j][2 * tx], sA2[j][2 * tx + 1]};
                const df rAm1 = rA1 ? df{0.f, 0.f} : df_add_f(s_t[j].rA, -1.0f);
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float4 t = dfc_mul(A1[p], A2[q]);
                        dfc_acc(aP[p][q], t);
                        // the matrix-P A term is rA t: (rA - 1) t into the difference
                        if (!rA1) dfc_acc(aX[p][q], dfc_scale(t, rAm1));
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
                            fX[p][q].x = fmaf(B1[p].x, B2[q].x, fmaf(-B1[p].z, B2[q].z, fX[p][q].x));
                            fX[p][q].y = fmaf(B1[p].x, B2[q].z, fmaf(B1[p].z, B2[q].x, fX[p][q].y));
                        }
                } else {
#pragma unroll
                    for (int p = 0; p < 2; ++p)
#pragma unroll
                        for (int q = 0; q < 2; ++q) dfc_acc(aX[p][q], dfc_mul(B1[p], B2[q]));
                }
            }
        }
        // renormalise every round, add to the FP64 sums every kSepFlush rounds
        const bool flush = (round + 1) % kSepFlush == 0 || base + kSepRound >= cnt_r;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                aP[p][q] = dfc_norm(aP[p][q]);
                aX[p][q] = dfc_norm(aX[p][q]);
                if (flush) {
                    dP[p][q][0] += (double)aP[p][q].x + (double)aP[p][q].y + (double)fP[p][q].x;
                    dP[p][q][1] += (double)aP[p][q].z + (double)aP[p][q].w + (double)fP[p][q].y;
                    dX[p][q][0] += (double)aX[p][q].x + (double)aX[p][q].y + (double)fX[p][q].x;
                    dX[p][q][1] += (double)aX[p][q].z + (double)aX[p][q].w + (double)fX[p][q].y;
                    aP[p][q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    aX[p][q] = aP[p][q];
                    fP[p][q] = make_float2(0.f, 0.f);
                    fX[p][q] = fP[p][q];
                }
            }
        __syncthreads();
    }
    const size_t grid = (size_t)Ka * Kb;
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (!(v1[p] && v2[q])) continue;
            const size_t o = (size_t)k1[p] * Kb + k2[q];
            double2 *pm = acc + (size_t)r * grid + o;
            double2 *pp = acc + ((size_t)n_sub + r) * grid + o;
            const double2 vm = *pm, vp = *pp;
            *pm = make_double2(vm.x + (dP[p][q][0] + dX[p][q][0]), vm.y + (dP[p][q][1] + dX[p][q][1]));
            *pp = make_double2(vp.x + dP[p][q][0], vp.y + dP[p][q][1]);
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

size_t sep2_bytes_per_trajectory() { return sizeof(SepTraj); }

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
        // tiles of 32 x 32 slots over the whole grid; tiles past the chunk's
        // union window return at once
        const int64_t tiles = (int64_t)((net->Ka + kSepTile - 1) / kSepTile) *
                              ((net->Kb + kSepTile - 1) / kSepTile);
        dim3 g2((unsigned)tiles, (unsigned)net->n_sub2);
        SepTraj *sep = static_cast<SepTraj *>(net->d_sep2);
        k_sep_prep<<<blocks2(net, count), 256, 0, net->stream>>>(net->d_n, net->d_nS2, count, sep);
        GBS_LAUNCH_CHECK();
        k_gf2d_df<<<g2, kSepThreads, 0, net->stream>>>(sep, net->d_n, net->d_nS2, net->d_wmax2,
                                                        count, e0, net->n_sub2, net->Ka, net->Kb,
                                                        net->d_tw2, K, net->d_acc2,
                                                        net->d_counts2);
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
