// K4: per-trajectory generating functions and their sub-ensemble sums.
//
// For trajectory e with input total n = alpha.beta (real) and output total
// n_S = alpha'.beta' = x + i y, and z_k = e^{i theta_k}, theta_k = 2 pi k / K1,
// the c-number projector of Eq. c-number-variable summed over m gives
//   G_mP(z) = cosh(n + (z-1) n_S) / cosh(n)               (matrix-P, M = 2)
//   G_+P(z) = exp((z-1) n_S)                              (+P, g_0 = 1)
// With L = (z-1) n_S = l1 + i phi,
//   l1  = (cos theta - 1) x - sin theta y,  phi = sin theta x + (cos theta - 1) y,
// and numerator and denominator of cosh(n+L)/cosh(n) multiplied by e^{-|n|}:
//   G_mP = [e^{l1 + c1} e^{i phi} + e^{-l1 + c2} e^{-i phi}] / (1 + e^{-2|n|}),
//   c1 = min(0, 2n),  c2 = -2 max(n, 0),
//   G_+P = e^{l1} e^{i phi}.
// Terms below 2^-60 (FP64 kernel) or 2^-47 (double-float kernel) are
// skipped: per trajectory, finalize() derives from (n, x, y) two windows of
// k (around theta = 0 for the e^{l1} terms, around theta = pi for the
// e^{-l1} term) outside which each term is provably smaller than that,
// using |sin theta| <= sqrt(2 (1 - cos theta)).
//
// Work split (FP64 kernel): one thread per k, one block per (256
// consecutive k, sub-ensemble r); each thread loops over the sub-ensemble's
// trajectories of the chunk in increasing order and adds its sums to
// acc[est][r][k], so every sum is formed in a fixed order (bitwise
// reproducible for a fixed chunking).  The double-float kernel gives each
// lane the mirror pair k, K1 - k and splits the trajectories over 8
// half-warps (see k_gf_df).  Trajectory e belongs to sub-ensemble e mod n_sub.
#include "gbs_internal.cuh"
#include "dfloat.cuh"

#include <algorithm>
#include <cmath>

namespace gbs {
namespace {

// The windows are bounds, so FP32 serves (GB300's FP64 pipe is narrow and
// its asin and sqrt are slow): every FP32 step below errs by a few ulp, in
// all below 4e-6 relative in theta, and the k count is rounded up by that
// plus a margin of 2 (one for the floor, one for the rounding).
__device__ __forceinline__ int half_width(float cstar, int K1) {
    // largest |delta theta| with 1 - cos(delta theta) <= cstar, in k units
    const int half = K1 >> 1;
    if (!(cstar < 2.0f)) return half;  // also catches NaN
    const float th = 2.0f * asinf(sqrtf(0.5f * cstar));
    const float v = th * (float)K1 * 0.159154943f;  // K1 / (2 pi)
    const float w = floorf(v * (1.0f + 4e-6f)) + 2.0f;
    return w >= (float)half ? half : (int)w;
}

__device__ __forceinline__ Window windows_for(double n, double xd, double yd, int K1, double Td) {
    const float x = (float)xd, y = (float)yd, T = (float)Td;
    const float ay = fabsf(y);
    const int half = K1 >> 1;
    Window w;
    // e^{l1} terms: l1 <= -c x + sqrt(2c)|y|, c = 1 - cos theta
    if (!(xd > 0.0)) {
        w.w1 = half;
    } else {
        const float u = (1.41421356f * ay + sqrtf(2.0f * y * y + 4.0f * x * T)) / (2.0f * x);
        w.w1 = half_width(u * u, K1);
    }
    // e^{-l1 + c2} term: -l1 + c2 <= (2 - c')x + sqrt(2c')|y| + c2, c' = 1 + cos theta;
    // D = 2 x + c2 + T = 2 (x - max(n, 0)) + T with the difference taken in
    // FP64, T raised by 1/4 so that FP32 rounding near disc = 0 cannot drop
    // a window
    const double c2 = -2.0 * fmax(n, 0.0);
    if (!(xd > 0.0)) {
        w.w2 = ((double)ay + c2 >= -Td) ? half : -1;
    } else {
        const float D = (float)(2.0 * xd + c2) + (T + 0.25f);
        const float disc = 2.0f * y * y + 4.0f * x * D;
        if (disc < 0.0f) {
            w.w2 = -1;
        } else {
            const float u = (1.41421356f * ay + sqrtf(disc)) / (2.0f * x);
            w.w2 = (u < 0.0f) ? -1 : half_width(u * u, K1);
        }
    }
    return w;
}

// Per-trajectory constants of the double-float generating functions:
// n_S = x + i y, c1 = min(0, 2n), c2 = -2 max(n, 0), 1 / (1 + e^{-2|n|}) as
// double-float, the FP64 values for the pairs outside the double-float
// ranges, and the windows.
struct __align__(16) GfRec {
    double xd, yd, c1d, c2d;
    df x, y, c1, c2, inv;
    int w1, w2;
};
static_assert(sizeof(GfRec) == 80, "generating-function record layout");

__global__ void k_finalize(const double2 *__restrict__ part, int mtiles, int64_t ld,
                           const double *__restrict__ n, int64_t count, int K1,
                           double2 *__restrict__ nS, Window *__restrict__ win,
                           int *__restrict__ wmax, GfRec *__restrict__ rec) {
    int m1 = -1, m2 = -1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int t = 0; t < mtiles; ++t) {
            const double2 p = part[(size_t)t * ld + i];
            re += p.x;
            im += p.y;
        }
        nS[i] = make_double2(re, im);
        const double nn = n[i];
        const Window w = windows_for(nn, re, im, K1, rec ? kSkipLogDf : kSkipLog);
        win[i] = w;
        if (rec) {
            GfRec g;
            g.xd = re;
            g.yd = im;
            g.c1d = fmin(0.0, 2.0 * nn);
            g.c2d = -2.0 * fmax(nn, 0.0);
            g.x = df_from_double(re);
            g.y = df_from_double(im);
            g.c1 = df_from_double(g.c1d);
            g.c2 = df_from_double(g.c2d);
            // 1 + e^{-2|n|} rounds to 1 for |n| > 20 (e^{-40} < 2^-54): no
            // FP64 exponential for those (GB300's FP64 pipe is narrow)
            const double an = fabs(nn);
            g.inv = df_from_double(an > 20.0 ? 1.0 : 1.0 / (1.0 + exp(-2.0 * an)));
            g.w1 = w.w1;
            g.w2 = w.w2;
            rec[i] = g;
        }
        m1 = max(m1, w.w1);
        m2 = max(m2, w.w2);
    }
    // union of the chunk's windows: the generating-function kernel only
    // assigns threads to k inside it
    m1 = __reduce_max_sync(0xffffffffu, m1);
    m2 = __reduce_max_sync(0xffffffffu, m2);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&wmax[0], m1);
        atomicMax(&wmax[1], m2);
    }
}

__device__ __forceinline__ int dist0(int k, int K1) { return k <= (K1 >> 1) ? k : K1 - k; }

__device__ __forceinline__ int dist_pi(int k, int K1) {
    const int d = k - (K1 >> 1);
    return d < 0 ? -d : d;
}

// FP64 evaluation (GBS_FP64).
__global__ void __launch_bounds__(256) k_gf_fp64(const double *__restrict__ n_in,
                                                 const double2 *__restrict__ nS_in,
                                                 const Window *__restrict__ win_in,
                                                 int64_t count, uint64_t e0, int n_sub, int K1,
                                                 const double2 *__restrict__ tw,
                                                 double2 *__restrict__ acc,
                                                 int64_t *__restrict__ counts) {
    __shared__ double s_x[256], s_y[256], s_c1[256], s_c2[256], s_inv[256];
    __shared__ int s_w1[256], s_w2[256];

    const int r = blockIdx.y;
    const int kb0 = blockIdx.x * 256;
    const int kb1 = min(kb0 + 256, K1);
    const int k = kb0 + threadIdx.x;
    const bool kvalid = k < K1;
    const int d0 = kvalid ? dist0(k, K1) : 0x3fffffff;
    const int dpi = kvalid ? dist_pi(k, K1) : 0x3fffffff;
    // block-wide minimum distances (for tile skipping)
    const int bd0 = min(dist0(kb0, K1), dist0(kb1 - 1, K1));
    const int half = K1 >> 1;
    const int bdpi = (half >= kb0 && half < kb1) ? 0 : min(dist_pi(kb0, K1), dist_pi(kb1 - 1, K1));

    const int64_t first = (int64_t)(((uint64_t)r + (uint64_t)n_sub - e0 % (uint64_t)n_sub) %
                                    (uint64_t)n_sub);
    const int64_t cnt_r = first < count ? (count - 1 - first) / n_sub + 1 : 0;

    double2 t = kvalid ? tw[k] : make_double2(0.0, 0.0);
    const double cm1 = t.x, sn = t.y;
    double am_re = 0.0, am_im = 0.0, ap_re = 0.0, ap_im = 0.0;

    for (int64_t base = 0; base < cnt_r; base += 256) {
        const int64_t q = base + threadIdx.x;
        int hit = 0;
        if (q < cnt_r) {
            const int64_t i = first + q * n_sub;
            const double nn = n_in[i];
            const double2 s = nS_in[i];
            const Window w = win_in[i];
            s_x[threadIdx.x] = s.x;
            s_y[threadIdx.x] = s.y;
            s_c1[threadIdx.x] = fmin(0.0, 2.0 * nn);
            s_c2[threadIdx.x] = -2.0 * fmax(nn, 0.0);
            s_inv[threadIdx.x] = 1.0 / (1.0 + exp(-2.0 * fabs(nn)));
            s_w1[threadIdx.x] = w.w1;
            s_w2[threadIdx.x] = w.w2;
            hit = (bd0 <= w.w1) || (bdpi <= w.w2);
        }
        if (!__syncthreads_or(hit)) continue;
        const int ntile = (cnt_r - base) < 256 ? (int)(cnt_r - base) : 256;
        if (kvalid) {
            for (int j = 0; j < ntile; ++j) {
                const bool in1 = d0 <= s_w1[j];
                const bool in2 = dpi <= s_w2[j];
                if (!(in1 || in2)) continue;
                const double x = s_x[j], y = s_y[j];
                const double l1 = cm1 * x - sn * y;
                const double ph = sn * x + cm1 * y;
                double sp, cp;
                sincos(ph, &sp, &cp);
                double e1 = 0.0, e2 = 0.0;
                if (in1) {
                    const double c1 = s_c1[j];
                    e1 = exp(l1 + c1);
                    const double gp = (c1 == 0.0) ? e1 : exp(l1);
                    ap_re += gp * cp;
                    ap_im += gp * sp;
                }
                if (in2) e2 = exp(-l1 + s_c2[j]);
                const double inv = s_inv[j];
                am_re += (e1 + e2) * cp * inv;
                am_im += (e1 - e2) * sp * inv;
            }
        }
        __syncthreads();
    }
    if (kvalid) {
        double2 *a0 = acc + (size_t)r * K1 + k;
        double2 *a1 = acc + ((size_t)n_sub + r) * K1 + k;
        const double2 o0 = *a0, o1 = *a1;
        *a0 = make_double2(o0.x + am_re, o0.y + am_im);
        *a1 = make_double2(o1.x + ap_re, o1.y + ap_im);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[r] += cnt_r;
}

// Double-float evaluation (BF16 split paths).  Each generating-function
// term enters the sub-ensemble sums, so its rounding error is an absolute
// error of P(m) at every m; the far-tail bins have sampling errors of
// 1e-10 and below, so the terms need FP64-class accuracy.  GB300's FP64 rate
// is low, so the same formulas are evaluated in double-float arithmetic on
// the FP32 pipes (dfloat.cuh, ~2^-46 relative): l1, phi, e^{l1 + c1},
// e^{-l1 + c2}, e^{l1}, sin phi, cos phi, so that the absolute error of
// every term stays at the 2^-46 the double-float rounding commits on terms
// of order one; terms below 2^-27 reach that with FP32 exp and sin/cos
// (small_term below).  Arguments outside the double-float ranges (|phi| >=
// 6000, exponents >= 80: only the +P heavy tail) are evaluated in FP64 and
// added to the FP64 sums directly.  Per warp lane, double-float partial sums
// over 32 trajectories are added to FP64 accumulators.
__device__ __forceinline__ df df_exp_small(df a, const DfTables &T, const DfConsts &K) {
    return a.hi < -87.0f ? df{0.0f, 0.0f} : df_exp_tab(a, T, K);  // below 1e-37: nothing
}

// Pieces of pi/64 for a one-stage Cody-Waite reduction of phi: the first
// four have at most 7 significant bits, so their products with the table
// index J (|J| < 2^17 for |phi| < 6000) are exact; the fifth is the float
// nearest the rest (what remains is below 4e-20, times |J| below 5e-15).
constexpr float kPi64a = 0x1.94p-5f, kPi64b = -0x1.ep-13f, kPi64c = -0x1.2cp-23f,
                kPi64d = 0x1.1p-31f, kPi64e = 0x1.0b4612p-39f;

// The common case's term e^{l1} (cos phi, sin phi) in double-float with the
// independent halves side by side on the packed FP32x2 instructions: phi =
// J pi/64 + r (|r| <= pi/128) beside l1 = (64 m + j) ln2/64 + r' (Tang's
// exponential, as df_exp_tab), the sine and cosine of r by their Taylor
// series (as df_sincos_tab), combined with the full-circle table
// circ[J mod 128] = (sin, cos)(J pi/64) by angle addition, and the final
// products.  Returns (re, im) as (x, y).
__device__ __forceinline__ df2 cexp_pair(df l1, df ph, const DfTables &T, const float4 *circ,
                                         const DfConsts &K) {
    const float jf = rintf(ph.hi * 20.371832715762604f);  // 64 / pi
    const float kf = rintf(l1.hi * 92.33248261689366f);   // 64 / ln 2
    const float2 nq = f2(-jf, -kf);
    df2 r = df2_two_sum(f2_fma(nq, f2(kPi64a, K.ln2_64_1), f2(ph.hi, l1.hi)),
                        f2(ph.lo, l1.lo));                    // exact products
    r = df2_add_f(r, f2_mul(nq, f2(kPi64b, K.ln2_64_2)));   // exact products
    r = df2_add_f(r, f2_mul(nq, f2(kPi64c, K.ln2_64_3)));
    df rr = df_add_f(df2_x(r), -jf * kPi64d);               // exact product
    rr = df_add_f(rr, -jf * kPi64e);
    const df er = df2_y(r);
    const df r2 = df_mul(rr, rr);
    const float x = r2.hi;
    const float ts = x * x * fmaf(-x, 1.0f / 5040.0f, 1.0f / 120.0f);
    const float tc = x * x * fmaf(fmaf(x, 1.0f / 40320.0f, -1.0f / 720.0f), x, 1.0f / 24.0f);
    const df sixth = {-0x1.555556p-3f, 0x1.555556p-28f};  // -1/6
    df2 w = df2_make(df_mul(r2, sixth), df{-0.5f * r2.hi, -0.5f * r2.lo});
    w = df2_add_f(df2_add_f(w, f2(ts, tc)), f2(1.0f, 1.0f));
    const df sr = df_mul(rr, df2_x(w)), cr = df2_y(w);
    const float4 tb = circ[((int)jf) & 127];  // (sin hi, sin lo, cos hi, cos lo)
    const df S = {tb.x, tb.y}, C = {tb.z, tb.w};
    const df2 P = df2_mul(df2_make(S, C), df2_make(cr, cr));  // (S cr, C cr)
    df2 Q = df2_mul(df2_make(C, S), df2_make(sr, sr));        // (C sr, S sr)
    Q.hi.y = -Q.hi.y;
    Q.lo.y = -Q.lo.y;
    const df2 sc = df2_add(P, Q);  // (sin phi, cos phi)
    // e^{l1} by the 2^(j/64) table
    const float xe = er.hi;
    const float qt = xe * fmaf(fmaf(xe, 1.0f / 120.0f, 1.0f / 24.0f), xe, 1.0f / 6.0f);
    const df q = df_fast_two_sum(0.5f, qt);
    const df pe = df_add_f(df_add(er, df_mul(df_mul(er, er), q)), 1.0f);
    const int n = (int)kf;
    const df t = df_mul(T.exp2[n & 63], pe);
    const float scale = __int_as_float(((n >> 6) + 127) << 23);
    const df e1 = l1.hi < -87.0f ? df{0.0f, 0.0f} : df{t.hi * scale, t.lo * scale};
    return df2_mul(df2_make(e1, e1), df2_make(df2_y(sc), df2_x(sc)));
}

// Terms below 2^-27 (exponent l1 below kSmallLog) need no double-float
// result: their absolute error stays below 2^-46, what the double-float
// evaluation commits on terms of order one, when
//   e^{l1} = expf(l1.hi) (1 + l1.lo)   (expf: 2 ulp),
//   phi = 2 pi q + r in double-float (Cody-Waite with the 12-bit pieces of
//   pi/2 times 4: |q| < 1000, so every product is exact), then the SFU sine
//   and cosine of r.hi in [-pi, pi] (absolute error 2^-21.41) corrected to
//   first order by r.lo,
// i.e. a relative error below 2^-20.5 on a term below 2^-27.  Such terms
// are summed in FP32 (at most 32 per warp lane between flushes, each below
// 2^-27) and added to the FP64 sums with the double-float partials.
constexpr float kSmallLog = -18.72f;  // just below ln 2^-27 = -18.7150

__device__ __forceinline__ void small_term(df l1, df ph, const DfConsts &K, float &re, float &im) {
    const float qf = rintf(ph.hi * 0.15915494309189535f);  // 1 / (2 pi)
    df r = df_two_sum(fmaf(-qf, 4.0f * K.pio2_1, ph.hi), ph.lo);  // exact product
    r = df_add_f(r, -qf * (4.0f * K.pio2_2));                      // exact product
    r = df_add_f(r, -qf * (4.0f * K.pio2_3));
    r = df_add_f(r, -qf * (4.0f * K.pio2_4));
    float sn, cs;
    __sincosf(r.hi, &sn, &cs);
    const float s1 = fmaf(cs, r.lo, sn);
    const float c1 = fmaf(-sn, r.lo, cs);
    const float e = expf(l1.hi);
    const float m = fmaf(e, l1.lo, e);
    re = fmaf(m, c1, re);
    im = fmaf(m, s1, im);
}

// Mirror pairs.  theta_{K1-k} = -theta_k, so with
//   a = (cos theta - 1) x,  b = sin theta y,  c = sin theta x,  d = (cos theta - 1) y
// the exponents at k and K1 - k are
//   (z_k - 1) n_S      = (a - b) + i (c + d),
//   (z_{K1-k} - 1) n_S = (a + b) + i (d - c),
// and both terms share E = e^a e^{ic}:
//   e^{(z_k - 1) n_S}      = E       e^{-b + i d},
//   e^{(z_{K1-k} - 1) n_S} = conj(E) e^{ b + i d}.
// n_S is real for uniform loss (T = t U: alpha'.beta' = t^2 alpha.beta) up
// to the GEMM's rounding, so b and d are usually tiny.  With
// omega = -b + i d = y w, w = i (z_k - 1) (a constant of the lane), the two
// terms are E e^{omega} and conj(E e^{-omega}), so the lane's sums at k and
// K1 - k are X + Z and conj(X - Z) with
//   X = sum E cosh(omega) = S0 + (w^2 / 2) S2,
//   Z = sum E sinh(omega) = w S1 + (w^3 / 6) S3,   S_j = sum E y^j
// (|omega| <= 2^-12.5, so omega^4/24 < 2^-54 is left out): one table-driven
// complex exponential and four accumulations per trajectory serve both k,
// and the lane's factors w^j are applied once per tile.  S0 and S1 are
// double-float sums; S2 and S3 FP32, since w^2 S2 / 2 and w^3 S3 / 6 are
// below 2^-26 |E| and 2^-37 |E| per term.  Every lane of the double-float
// kernel holds such a pair of k.

// (p.x + i p.y) (q.x + i q.y) in double-float.
__device__ __forceinline__ df2 cmul_df2(df2 p, df2 q) {
    const df2 s = df2_mul(p, df2_make(df2_x(q), df2_x(q)));                // (px qx, py qx)
    df2 t = df2_mul(df2_make(df2_y(p), df2_x(p)), df2_make(df2_y(q), df2_y(q)));  // (py qy, px qy)
    t.hi.x = -t.hi.x;
    t.lo.x = -t.lo.x;
    return df2_add(s, t);
}

// Moment sums of one lane's mirror pairs over a tile (see above).
struct MirrorSums {
    df2 s0, s1;       // sum E, sum E y (double-float)
    float2 s2, s3;    // sum E y^2, sum E y^3 (FP32)
};

__device__ __forceinline__ void mirror_add(MirrorSums &m, df2 E, df y) {
    m.s0 = df2_add(m.s0, E);
    // E y: the product of the high parts exact, the cross terms in FP32
    const float2 yh = f2(y.hi, y.hi);
    const float2 p = f2_mul(E.hi, yh);
    const float2 e = f2_fma(E.hi, f2(y.lo, y.lo), f2_fma(E.lo, yh, f2_fma(E.hi, yh, f2_neg(p))));
    m.s1 = df2_add(m.s1, df2{p, e});
    const float y2 = y.hi * y.hi;
    m.s2 = f2_fma(E.hi, f2(y2, y2), m.s2);
    m.s3 = f2_fma(E.hi, f2(y2 * y.hi, y2 * y.hi), m.s3);
}

// (X + Z, conj(X - Z)) from the moment sums and the lane's w = i (z - 1).
__device__ __forceinline__ void mirror_finish(const MirrorSums &m, df2 w, df2 &at_k, df2 &at_mk) {
    const float wr = w.hi.x, wi = w.hi.y;
    const float w2r = wr * wr - wi * wi, w2i = 2.0f * wr * wi;
    const float w3r = w2r * wr - w2i * wi, w3i = w2r * wi + w2i * wr;
    const float2 c2 = f2(0.5f * (w2r * m.s2.x - w2i * m.s2.y), 0.5f * (w2r * m.s2.y + w2i * m.s2.x));
    const float2 c3 = f2((w3r * m.s3.x - w3i * m.s3.y) * (1.0f / 6.0f),
                         (w3r * m.s3.y + w3i * m.s3.x) * (1.0f / 6.0f));
    const df2 X = df2_add_f(m.s0, c2);
    df2 Z = df2_add_f(cmul_df2(w, m.s1), c3);
    at_k = df2_add(X, Z);
    Z.hi = f2_neg(Z.hi);
    Z.lo = f2_neg(Z.lo);
    at_mk = df2_add(X, Z);
    at_mk.hi.y = -at_mk.hi.y;
    at_mk.lo.y = -at_mk.lo.y;
}

// Pair slots of the union window: slot s holds k = s and K1 - s for
// s = 0..W1 (around theta = 0), then k = K1/2 + s and K1/2 - s for
// s = 0..W2 (around theta = pi); when the two windows cover the circle,
// s = 0..K1/2.  k = 0 and k = K1/2 pair with themselves.
__device__ __forceinline__ int pair_slot_count(int K1, int W1, int W2, bool &whole) {
    const int half = K1 >> 1;
    const int n1 = W1 >= half ? K1 : 2 * W1 + 1;
    const int n2 = W2 < 0 ? 0 : (W2 >= half ? K1 : 2 * W2 + 1);
    whole = n1 + n2 >= K1;
    if (whole) return half + 1;
    return (W1 < 0 ? 0 : W1 + 1) + (W2 < 0 ? 0 : W2 + 1);
}

// (k, K1 - k) of pair slot i (whole: the windows cover the circle), or
// kp = -1 past the end.
__device__ __forceinline__ void pair_slot_to_k(int i, int K1, int W1, int W2, bool whole, int &kp,
                                               int &km) {
    const int half = K1 >> 1;
    kp = km = -1;
    if (whole) {
        if (i <= half) {
            kp = i;
            km = (K1 - i) & (K1 - 1);
        }
        return;
    }
    const int p1 = W1 < 0 ? 0 : W1 + 1;
    const int p2 = W2 < 0 ? 0 : W2 + 1;
    if (i < p1) {
        kp = i;
        km = (K1 - i) & (K1 - 1);
    } else if (i < p1 + p2) {
        kp = half + (i - p1);
        km = half - (i - p1);
    }
}

constexpr int kGfSlots = 16;   // pair slots per block (the lanes of each half-warp)
#ifndef GBS_GF_MINBLOCKS
#define GBS_GF_MINBLOCKS 5     // resident blocks per SM the register budget is sized for
#endif
constexpr int kGfGroups = 8;   // trajectory groups per block, one half-warp each
constexpr int kGfPer = 32;     // trajectories per half-warp and tile
constexpr int kGfTile = kGfGroups * kGfPer;  // trajectories per tile
#ifndef GBS_GF_FLUSH_TILES
#define GBS_GF_FLUSH_TILES 2   // tiles between flushes of the partials to FP64
#endif
constexpr int kGfFlushTiles = GBS_GF_FLUSH_TILES;

// Double-float partial sums of one k over the trajectories of one tile.
struct SidePartial {
    df2 both;                         // terms common to both estimators (re, im)
    df pm_re, pm_im, pp_re, pp_im;    // general formulas: matrix-P, +P
    float sm_re, sm_im;               // terms below 2^-27, both estimators
    bool gen;                         // a general-formula term was added
};

__device__ __forceinline__ void side_clear(SidePartial &s) {
    s.both = {f2(0.0f, 0.0f), f2(0.0f, 0.0f)};
    s.pm_re = s.pm_im = s.pp_re = s.pp_im = df{0.0f, 0.0f};
    s.sm_re = s.sm_im = 0.0f;
    s.gen = false;
}

// The lane's FP64 sums in shared memory, f[c * kGfSlots]: c = 0, 1 the
// terms common to both estimators (re, im), c = 2, 3 matrix-P's own, c = 4,
// 5 +P's own; matrix-P's generating function is the sum of c = 0, 1 and 2,
// 3, +P's of c = 0, 1 and 4, 5.
constexpr int kGfSums = 6;

// One (trajectory, k) term with exponent (l1, ph) = (z_k - 1) n_S: FP64
// outside the double-float ranges (straight into the lane's FP64 sums f),
// FP32 below 2^-27, the term shared by both estimators when `plain`, else
// the general formulas.  (cm1d, snd) = (cos theta_k - 1, sin theta_k) in
// FP64.
__device__ __forceinline__ void side_term(df l1, df ph, bool in1, bool in2, bool plain,
                                          const GfRec &g, double cm1d, double snd,
                                          const DfTables &T, const float4 *circ,
                                          const DfConsts &K, SidePartial &s,
                                          double *f) {
    const df c1 = g.c1;
    df a1 = l1, a2 = {0.0f, 0.0f};
    bool big = fabsf(ph.hi) >= 6000.0f || (in1 && l1.hi >= 80.0f);
    if (!plain) {
        a1 = df_add(l1, c1);
        a2 = df_add(df_neg(l1), g.c2);
        big = big || (in1 && a1.hi >= 80.0f) || (in2 && a2.hi >= 80.0f);
    }
    if (big) {
        // outside the double-float ranges (+P heavy tail, huge phases):
        // this term in FP64, straight into the FP64 sums
        const double xd = g.xd, yd = g.yd;
        const double l1d = cm1d * xd - snd * yd;
        double sd, cd;
        sincos(snd * xd + cm1d * yd, &sd, &cd);
        double e1d = 0.0, e2d = 0.0;
        if (in1) {
            e1d = exp(l1d + g.c1d);
            const double gp = (g.c1d == 0.0) ? e1d : exp(l1d);
            f[4 * kGfSlots] += gp * cd;
            f[5 * kGfSlots] += gp * sd;
        }
        if (in2) e2d = exp(-l1d + g.c2d);
        const double dinv = df_to_double(g.inv);
        f[2 * kGfSlots] += (e1d + e2d) * cd * dinv;
        f[3 * kGfSlots] += (e1d - e2d) * sd * dinv;
        return;
    }
    if (plain && l1.hi < kSmallLog) {
        small_term(l1, ph, K, s.sm_re, s.sm_im);
        return;
    }
    if (plain) {
        s.both = df2_add(s.both, cexp_pair(l1, ph, T, circ, K));
        return;
    }
    df sp, cp;
    df_sincos_tab(ph, T, K, sp, cp);
    df e1 = {0.0f, 0.0f}, e2 = {0.0f, 0.0f};
    s.gen = true;
    if (in1) {
        e1 = df_exp_small(a1, T, K);
        const df gp = (c1.hi == 0.0f) ? e1 : df_exp_small(l1, T, K);
        s.pp_re = df_add(s.pp_re, df_mul(gp, cp));
        s.pp_im = df_add(s.pp_im, df_mul(gp, sp));
    }
    if (in2) e2 = df_exp_small(a2, T, K);
    s.pm_re = df_add(s.pm_re, df_mul(df_mul(df_add(e1, e2), g.inv), cp));
    s.pm_im = df_add(s.pm_im, df_mul(df_mul(df_sub(e1, e2), g.inv), sp));
}

// The FP32 small-term sums (at most kGfPer terms each) into the
// double-float partials, on the FP32 pipes.
__device__ __forceinline__ void side_fold_small(SidePartial &s) {
    s.both = df2_add_f(s.both, f2(s.sm_re, s.sm_im));
    s.sm_re = s.sm_im = 0.0f;
}

// The partials (small sums folded in) into the lane's FP64 sums f.  GB300's
// FP64 pipe is narrow: the general formulas' partials are converted only
// when used.
__device__ __forceinline__ void side_flush(const SidePartial &s, double *f) {
    f[0] += df_to_double(df2_x(s.both));
    f[kGfSlots] += df_to_double(df2_y(s.both));
    if (s.gen) {
        f[2 * kGfSlots] += df_to_double(s.pm_re);
        f[3 * kGfSlots] += df_to_double(s.pm_im);
        f[4 * kGfSlots] += df_to_double(s.pp_re);
        f[5 * kGfSlots] += df_to_double(s.pp_im);
    }
}

// One block per (16 pair slots of the union window, sub-ensemble r): the 8
// half-warps hold the same 32 k and split the sub-ensemble's trajectories
// (trajectory q to half-warp q mod 8), so they carry the same work and need
// no barrier until the final fixed-order sum of their 8 partials.  Each
// warp stages the 64 trajectories of its two half-warps in a 256-trajectory
// tile (records written by the finalize kernel); each half-warp walks its
// 32 in order, flushing its double-float partials to FP64 after each tile.
// Grid: x = sub-ensemble (fast), y = block of pair slots from k = 0
// outwards, so the heaviest blocks start first and the last wave holds the
// lightest; blocks of 16 pair slots (32 k) keep that tail short.
struct GfShared {
    GfRec rec[kGfGroups / 2][2 * kGfPer];  // per warp: its two half-warps' trajectories
    double sum[kGfGroups][2][kGfSums][kGfSlots];  // FP64 sums: [group][k, K1 - k][c]
    DfTables tab;
    float4 circ[128];  // (sin, cos)(j pi/64) as double-float, j = 0..127
};

// One block's work: sub-ensemble r, pair-slot block y of one chunk of one
// network.
__device__ __forceinline__ void gf_df_block(const GfRec *__restrict__ rec,
                                            const int *__restrict__ wmax, int64_t count,
                                            uint64_t e0, int n_sub, int K1,
                                            const double2 *__restrict__ tw, const DfConsts &K,
                                            double2 *__restrict__ acc,
                                            int64_t *__restrict__ counts, int r, int y,
                                            GfShared &sh) {
    const int W1 = wmax[0], W2 = wmax[1];
    const int lane = threadIdx.x & 31;
    const int slot = threadIdx.x & (kGfSlots - 1);
    const int grp = threadIdx.x / kGfSlots;  // half-warp
    const int warp = threadIdx.x >> 5;
    const int64_t first = (int64_t)(((uint64_t)r + (uint64_t)n_sub - e0 % (uint64_t)n_sub) %
                                    (uint64_t)n_sub);
    const int64_t cnt_r = first < count ? (count - 1 - first) / n_sub + 1 : 0;
    bool whole;
    const int nslots = pair_slot_count(K1, W1, W2, whole);
    if (y * kGfSlots >= nslots && y > 0) return;  // past the union window (block 0 always runs)
    int kp, km;
    pair_slot_to_k(y * kGfSlots + slot, K1, W1, W2, whole, kp, km);
    const bool kvalid = kp >= 0;
    const bool self = kp == km;  // k = 0 or K1/2
    const int d0 = kvalid ? dist0(kp, K1) : 0x3fffffff;     // the same for km
    const int dpi = kvalid ? dist_pi(kp, K1) : 0x3fffffff;
    for (int t = threadIdx.x; t < 64; t += blockDim.x)
        sh.tab.exp2[t] = df{K.exp2_hi[t], K.exp2_lo[t]};
    for (int t = threadIdx.x; t < 33; t += blockDim.x) {
        sh.tab.sn[t] = df{K.sin_hi[t], K.sin_lo[t]};
        sh.tab.cs[t] = df{K.cos_hi[t], K.cos_lo[t]};
    }
    for (int t = threadIdx.x; t < 128; t += blockDim.x)
        sh.circ[t] = make_float4(K.circ[t][0], K.circ[t][1], K.circ[t][2], K.circ[t][3]);
    double *fp = sh.sum[grp][0][0] + slot;  // f[c] at fp[c * kGfSlots]
    double *fm = sh.sum[grp][1][0] + slot;
#pragma unroll
    for (int c = 0; c < kGfSums; ++c) fp[c * kGfSlots] = fm[c * kGfSlots] = 0.0;
    __syncthreads();

    const double2 t = kvalid ? tw[kp] : make_double2(0.0, 0.0);
    const double cm1d = t.x, snd = t.y;
    const df cm1 = df_from_double(t.x), sn = df_from_double(t.y);
    const df2 cs_pair = df2_make(cm1, sn), sc_pair = df2_make(sn, cm1);
    // |b|, |d| <= |y| max(|sin|, 1 - cos); the factor rounded up
    const float ymul = fmaxf(fabsf(sn.hi), fabsf(cm1.hi)) * (1.0f + 0x1p-20f);
    const df2 w_lane = df2_make(df_neg(sn), cm1);  // i (z_k - 1)
    const GfRec *mine = sh.rec[warp] + kGfPer * (lane / kGfSlots);

    // double-float partials over kGfFlushTiles tiles (the FP32 small-term
    // sums folded into them after every tile), then into the FP64 sums
    SidePartial sp_, sm_;
    side_clear(sp_);
    side_clear(sm_);
    MirrorSums ms;
    ms.s0 = ms.s1 = {f2(0.0f, 0.0f), f2(0.0f, 0.0f)};
    ms.s2 = ms.s3 = f2(0.0f, 0.0f);
    bool mirror = false;
    int pending = 0;
    for (int64_t base = 0; base < cnt_r; base += kGfTile) {
#pragma unroll
        for (int e = lane; e < 2 * kGfPer; e += 32) {
            // entry e: trajectory j = e mod kGfPer of half-warp 2 warp + e / kGfPer
            const int64_t q = base + 2 * warp + e / kGfPer + kGfGroups * (e % kGfPer);
            if (q < cnt_r) sh.rec[warp][e] = rec[first + q * n_sub];
        }
        __syncwarp();
        const int ntile = (cnt_r - base) < kGfTile ? (int)(cnt_r - base) : kGfTile;
        const int nmine = ntile > grp ? (ntile - grp + kGfGroups - 1) / kGfGroups : 0;
        if (kvalid) {
            for (int m = 0; m < nmine; ++m) {
                const GfRec &g = mine[m];
                const bool in1 = d0 <= g.w1;
                const bool in2 = dpi <= g.w2;
                if (!(in1 || in2)) continue;
                // (a, c) = (cos - 1, sin) x
                const df2 A = df2_mul(cs_pair, df2_make(g.x, g.x));
                // n >= 0 with e^{-2n} below double rounding and no term near
                // theta = pi: both estimators add e^{l1} e^{i phi} (the
                // general formulas give the same value), summed once
                const bool plain = in1 && !in2 && g.c1.hi == 0.0f && g.inv.hi == 1.0f &&
                                   g.inv.lo == 0.0f;
                if (plain && !self && fabsf(g.y.hi) * ymul <= 0x1p-13f &&
                    A.hi.x >= kSmallLog + 0x1p-10f && A.hi.x < 79.0f &&
                    fabsf(A.hi.y) < 5999.0f) {
                    // both k from one complex exponential (|b|, |d| <=
                    // 2^-13 keep both exponents on the double-float side of
                    // kSmallLog and inside the double-float ranges)
                    mirror_add(ms, cexp_pair(df2_x(A), df2_y(A), sh.tab, sh.circ, K), g.y);
                    mirror = true;
                    continue;
                }
                // each k by the general rules: (l1, phi) = (a - b, c + d) at
                // k and (a + b, d - c) at K1 - k, (b, d) = (sin, cos - 1) y
                const df2 B = df2_mul(sc_pair, df2_make(g.y, g.y));
                df2 Bn = B;
                Bn.hi.x = -Bn.hi.x;
                Bn.lo.x = -Bn.lo.x;
                const df2 lp = df2_add(A, Bn);
                side_term(df2_x(lp), df2_y(lp), in1, in2, plain, g, cm1d, snd, sh.tab, sh.circ,
                          K, sp_, fp);
                if (!self) {
                    df2 An = A;
                    An.hi.y = -An.hi.y;
                    An.lo.y = -An.lo.y;
                    const df2 lm = df2_add(An, B);
                    side_term(df2_x(lm), df2_y(lm), in1, in2, plain, g, cm1d, -snd, sh.tab,
                              sh.circ, K, sm_, fm);
                }
            }
            side_fold_small(sp_);
            side_fold_small(sm_);
            if (++pending == kGfFlushTiles || base + kGfTile >= cnt_r) {
                if (mirror) {
                    df2 at_k, at_mk;
                    mirror_finish(ms, w_lane, at_k, at_mk);
                    sp_.both = df2_add(sp_.both, at_k);
                    sm_.both = df2_add(sm_.both, at_mk);
                    ms.s0 = ms.s1 = {f2(0.0f, 0.0f), f2(0.0f, 0.0f)};
                    ms.s2 = ms.s3 = f2(0.0f, 0.0f);
                    mirror = false;
                }
                side_flush(sp_, fp);
                if (!self) side_flush(sm_, fm);
                side_clear(sp_);
                side_clear(sm_);
                pending = 0;
            }
        }
        __syncwarp();
    }
    // combine the trajectory groups in a fixed order
    __syncthreads();
    if (grp == 0 && kvalid) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            if (side == 1 && self) break;
            double v[kGfSums];
#pragma unroll
            for (int c = 0; c < kGfSums; ++c) {
                double t = 0.0;
#pragma unroll
                for (int gi = 0; gi < kGfGroups; ++gi) t += sh.sum[gi][side][c][slot];
                v[c] = t;
            }
            v[2] += v[0];  // matrix-P: common + own
            v[3] += v[1];
            v[4] += v[0];  // +P: common + own
            v[5] += v[1];
            const int k = side ? km : kp;
            double2 *a0 = acc + (size_t)r * K1 + k;
            double2 *a1 = acc + ((size_t)n_sub + r) * K1 + k;
            const double2 o0 = *a0, o1 = *a1;
            *a0 = make_double2(o0.x + v[2], o0.y + v[3]);
            *a1 = make_double2(o1.x + v[4], o1.y + v[5]);
        }
    }
    if (y == 0 && threadIdx.x == 0) counts[r] += cnt_r;
}

__global__ void __launch_bounds__(kGfSlots * kGfGroups, GBS_GF_MINBLOCKS)
    k_gf_df(const GfRec *__restrict__ rec, const int *__restrict__ wmax, int64_t count,
            uint64_t e0, int n_sub, int K1, const double2 *__restrict__ tw, const DfConsts K,
            double2 *__restrict__ acc, int64_t *__restrict__ counts) {
    __shared__ GfShared sh;
    gf_df_block(rec, wmax, count, e0, n_sub, K1, tw, K, acc, counts, blockIdx.x, blockIdx.y, sh);
}

}  // namespace

// Float pieces of ln 2 and pi/2 for exact Cody-Waite products (12
// significant bits each except the last), split from the constants'
// decimal expansions at 80 digits; factorial reciprocals as double-float.
DfConsts make_df_consts() {
    DfConsts K;
    K.ln2_1 = 0x1.62ep-1f;
    K.ln2_2 = 0x1.0cp-15f;
    K.ln2_3 = -0x1.05c61p-29f;
    K.pio2_1 = 0x1.922p+0f;
    K.pio2_2 = -0x1.2aep-18f;
    K.pio2_3 = -0x1.deap-31f;
    K.pio2_4 = 0x1.184698p-44f;
    double f = 1.0;
    for (int k = 0; k < 18; ++k) {
        if (k > 0) f *= (double)k;
        const double v = 1.0 / f;
        K.inv_fact_hi[k] = (float)v;
        K.inv_fact_lo[k] = (float)(v - (double)K.inv_fact_hi[k]);
    }
    // ln 2 / 64 and pi / 64 in pieces whose products with the table index
    // (|n| < 2^13, |j| <= 16) are exact, from 60-digit expansions
    K.ln2_64_1 = 0x1.63p-7f;
    K.ln2_64_2 = -0x1.bdp-19f;
    K.ln2_64_3 = -0x1.05c61p-35f;
    K.pi64_1 = 0x1.921f8p-5f;
    K.pi64_2 = 0x1.aa22p-24f;
    K.pi64_3 = 0x1.68c234p-44f;
    for (int j = 0; j < 64; ++j) {
        const double v = std::exp2((double)j / 64.0);
        K.exp2_hi[j] = (float)v;
        K.exp2_lo[j] = (float)(v - (double)K.exp2_hi[j]);
    }
    const double pi = 3.14159265358979323846264338327950288;
    for (int j = 0; j < 128; ++j) {
        const double sv = std::sin((double)j * pi / 64.0), cv = std::cos((double)j * pi / 64.0);
        K.circ[j][0] = (float)sv;
        K.circ[j][1] = (float)(sv - (double)K.circ[j][0]);
        K.circ[j][2] = (float)cv;
        K.circ[j][3] = (float)(cv - (double)K.circ[j][2]);
    }
    for (int j = -16; j <= 16; ++j) {
        const double sv = std::sin((double)j * pi / 64.0), cv = std::cos((double)j * pi / 64.0);
        K.sin_hi[j + 16] = (float)sv;
        K.sin_lo[j + 16] = (float)(sv - (double)K.sin_hi[j + 16]);
        K.cos_hi[j + 16] = (float)cv;
        K.cos_lo[j + 16] = (float)(cv - (double)K.cos_hi[j + 16]);
    }
    return K;
}

namespace {

__global__ void k_tables(int K1, double2 *__restrict__ tw, double2 *__restrict__ wfft) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K1; k += gridDim.x * blockDim.x) {
        const double f = (double)k / (double)K1;
        double sh, ch, s2, c2;
        sincospi(f, &sh, &ch);        // theta/2 = pi k / K1
        sincospi(2.0 * f, &s2, &c2);  // theta = 2 pi k / K1
        tw[k] = make_double2(-2.0 * sh * sh, s2);  // (cos theta - 1, sin theta)
        wfft[k] = make_double2(c2, -s2);           // e^{-i theta}
    }
}

}  // namespace

int launch_finalize(gbs_net *net, int64_t count) {
    if (count <= 0) return GBS_OK;
    GBS_CUDA_TRY(cudaMemsetAsync(net->d_wmax, 0xff, 2 * sizeof(int), net->stream));  // -1, -1
    int blocks = (int)std::min<int64_t>((count + 255) / 256, (int64_t)net->sm_count * 8);
    k_finalize<<<blocks, 256, 0, net->stream>>>(net->d_nS_part, net->mtiles, net->chunk, net->d_n,
                                                 count, net->K1, net->d_nS, net->d_win,
                                                 net->d_wmax, static_cast<GfRec *>(net->d_gfrec));
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int launch_gf(gbs_net *net, uint64_t e0, int64_t count) {
    if (count <= 0) return GBS_OK;
    dim3 grid((unsigned)((net->K1 + 255) / 256), (unsigned)net->n_sub);
    if (simt_precision(net->precision)) {
        k_gf_fp64<<<grid, 256, 0, net->stream>>>(net->d_n, net->d_nS, net->d_win, count, e0,
                                                   net->n_sub, net->K1, net->d_tw, net->d_acc,
                                                   net->d_counts);
    } else {
        static const DfConsts K = make_df_consts();
        dim3 g2((unsigned)net->n_sub, (unsigned)((net->K1 / 2 + 1 + kGfSlots - 1) / kGfSlots));
        if (!net->d_gfrec) return set_error(GBS_EINVAL, "network has no generating-function records");
        k_gf_df<<<g2, kGfSlots * kGfGroups, 0, net->stream>>>(
            static_cast<const GfRec *>(net->d_gfrec), net->d_wmax, count, e0, net->n_sub,
            net->K1, net->d_tw, K, net->d_acc, net->d_counts);
    }
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

size_t gf_record_bytes() { return sizeof(GfRec); }

int launch_tables(gbs_net *net) {
    const int blocks = (net->K1 + 255) / 256;
    k_tables<<<blocks, 256, 0, net->stream>>>(net->K1, net->d_tw, net->d_wfft);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace gbs
