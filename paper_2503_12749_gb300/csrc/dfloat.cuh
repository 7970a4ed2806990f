// Double-float arithmetic on the FP32 pipes: a value is the unevaluated sum
// hi + lo of two floats (|lo| <= ulp(hi)/2), giving ~2^-46 relative
// precision at FP32 issue rates.  Error-free transformations: Knuth's
// two-sum, Dekker's fast two-sum, and the two-product via a fused
// multiply-add (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2).  exp and sin/cos are
// Cody-Waite range reductions (constants split into 12-bit pieces on the
// host so that k * piece is exact) followed by Taylor series of the
// reduced argument, evaluated by Horner's rule: the leading terms in
// double-float, the terms below 2^-28 of the result in plain FP32.
#pragma once

#include <cstdint>

namespace gbs {

struct df {
    float hi, lo;
};

// Range-reduction constants, computed on the host (see make_df_consts()).
struct DfConsts {
    float ln2_1, ln2_2, ln2_3;             // ln 2 = ln2_1 + ln2_2 + ln2_3
    float pio2_1, pio2_2, pio2_3, pio2_4;  // pi / 2 = sum of the four
    float inv_fact_hi[18], inv_fact_lo[18];  // 1 / k! as double-float, k = 0..17
    // table-driven functions (df_exp_tab, df_sincos_tab)
    float ln2_64_1, ln2_64_2, ln2_64_3;    // ln 2 / 64 in pieces of <= 11 bits (+ rest)
    float pi64_1, pi64_2, pi64_3;          // pi / 64 in pieces of <= 18 bits (+ rest)
    float exp2_hi[64], exp2_lo[64];        // 2^(j/64), j = 0..63
    float sin_hi[33], sin_lo[33];          // sin(j pi/64), j = -16..16 (index j + 16)
    float cos_hi[33], cos_lo[33];          // cos(j pi/64)
    float circ[128][4];                    // (sin hi, sin lo, cos hi, cos lo)(j pi/64), j = 0..127
};

// The constants and tables above (host; k_gf.cu).
DfConsts make_df_consts();

// The tables of DfConsts copied into shared memory (lanes index them with
// different j).
struct DfTables {
    df exp2[64];
    df sn[33], cs[33];
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    const float e = b - (s - a);
    return {s, e};
}

__device__ __forceinline__ df df_two_prod(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ df df_add(df x, df y) {
    const df s = df_two_sum(x.hi, y.hi);
    const float e = s.lo + (x.lo + y.lo);
    return df_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_add_f(df x, float y) {
    const df s = df_two_sum(x.hi, y);
    return df_fast_two_sum(s.hi, s.lo + x.lo);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_mul(df x, df y) {
    const df p = df_two_prod(x.hi, y.hi);
    const float e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
    return df_fast_two_sum(p.hi, e);
}

__device__ __forceinline__ df df_mul_f(df x, float y) {
    const df p = df_two_prod(x.hi, y);
    return df_fast_two_sum(p.hi, fmaf(x.lo, y, p.lo));
}

__device__ __forceinline__ df df_from_double(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ df df_fact(const DfConsts &K, int k) {
    return {K.inv_fact_hi[k], K.inv_fact_lo[k]};
}

// e^a for a.hi in [-87, 88].  a = k ln2 + r, |r| <= ln2/2 + tiny;
// e^r = sum_{j<=13} r^j/j! (remainder < 4e-18): j <= 8 in double-float,
// j = 9..13 in FP32.  Then scaled by 2^k.
__device__ __forceinline__ df df_exp(df a, const DfConsts &K) {
    const float kf = rintf(a.hi * 1.44269504088896340736f);
    df r = df_two_sum(fmaf(-kf, K.ln2_1, a.hi), a.lo);  // first product exact
    r = df_add_f(r, -kf * K.ln2_2);                      // exact product
    r = df_add_f(r, -kf * K.ln2_3);
    const float x = r.hi;
    // FP32 tail: sum_{j=9..13} x^{j-9}/j!
    float t = K.inv_fact_hi[13];
    t = fmaf(t, x, K.inv_fact_hi[12]);
    t = fmaf(t, x, K.inv_fact_hi[11]);
    t = fmaf(t, x, K.inv_fact_hi[10]);
    t = fmaf(t, x, K.inv_fact_hi[9]);
    df p = df_add_f(df_fact(K, 8), t * x);
#pragma unroll
    for (int j = 7; j >= 0; --j) p = df_add(df_fact(K, j), df_mul(p, r));
    const int ki = (int)kf;
    const float scale = __int_as_float((ki + 127) << 23);
    return {p.hi * scale, p.lo * scale};
}

// sin and cos of phi for |phi.hi| < 6000 (quadrant count < 2^12, so the
// products with the 12-bit pieces of pi/2 are exact).  phi = q pi/2 + s,
// |s| <= pi/4; with x = s^2 (<= 0.62):
//   sin s = s (1 - x/3! + x^2/5! - ... + x^8/17!),  remainder < 1e-19,
//   cos s = 1 - x/2! + x^2/4! - ... + x^8/16!,      remainder < 3e-18,
// the terms from x^5/11! (sin) and x^6/12! (cos) on in FP32.
__device__ __forceinline__ void df_sincos(df phi, const DfConsts &K, df &s_out, df &c_out) {
    const float qf = rintf(phi.hi * 0.636619772367581343076f);
    df s = df_two_sum(fmaf(-qf, K.pio2_1, phi.hi), phi.lo);
    s = df_add_f(s, -qf * K.pio2_2);
    s = df_add_f(s, -qf * K.pio2_3);
    s = df_add_f(s, -qf * K.pio2_4);
    const df x = df_mul(s, s);
    const float xf = x.hi;
    // sine: FP32 tail 1/11! - x (1/13! - x (1/15! - x/17!))
    float t = K.inv_fact_hi[17];
    t = fmaf(-t, xf, K.inv_fact_hi[15]);
    t = fmaf(-t, xf, K.inv_fact_hi[13]);
    t = fmaf(-t, xf, K.inv_fact_hi[11]);
    df ps = df_add_f(df_fact(K, 9), -t * xf);
    ps = df_sub(df_fact(K, 7), df_mul(ps, x));
    ps = df_sub(df_fact(K, 5), df_mul(ps, x));
    ps = df_sub(df_fact(K, 3), df_mul(ps, x));
    ps = df_sub(df_fact(K, 1), df_mul(ps, x));
    const df sn = df_mul(ps, s);
    // cosine: FP32 tail 1/12! - x (1/14! - x/16!)
    float u = K.inv_fact_hi[16];
    u = fmaf(-u, xf, K.inv_fact_hi[14]);
    u = fmaf(-u, xf, K.inv_fact_hi[12]);
    df pc = df_add_f(df_fact(K, 10), -u * xf);
    pc = df_sub(df_fact(K, 8), df_mul(pc, x));
    pc = df_sub(df_fact(K, 6), df_mul(pc, x));
    pc = df_sub(df_fact(K, 4), df_mul(pc, x));
    pc = df_sub(df_fact(K, 2), df_mul(pc, x));
    pc = df_sub(df_fact(K, 0), df_mul(pc, x));
    switch (((int)qf) & 3) {
        case 0: s_out = sn; c_out = pc; break;
        case 1: s_out = pc; c_out = df_neg(sn); break;
        case 2: s_out = df_neg(sn); c_out = df_neg(pc); break;
        default: s_out = df_neg(pc); c_out = sn; break;
    }
}

// Table-driven e^a for a.hi in [-87, 88] (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15, 1989): a = (64 m + j) ln2/64 + r, |r| <= ln2/128,
// e^a = 2^m 2^(j/64) e^r with e^r = 1 + r + r^2 (1/2 + r/6 + r^2/24 + r^3/120)
// (remainder < 4e-17); r^2 and the leading terms in double-float, the
// bracket beyond 1/2 in FP32.
__device__ __forceinline__ df df_exp_tab(df a, const DfTables &T, const DfConsts &K) {
    const float kf = rintf(a.hi * 92.33248261689366f);  // 64 / ln 2
    df r = df_two_sum(fmaf(-kf, K.ln2_64_1, a.hi), a.lo);  // exact product
    r = df_add_f(r, -kf * K.ln2_64_2);                      // exact product
    r = df_add_f(r, -kf * K.ln2_64_3);
    const float x = r.hi;
    const float qt = x * fmaf(fmaf(x, 1.0f / 120.0f, 1.0f / 24.0f), x, 1.0f / 6.0f);
    const df q = df_fast_two_sum(0.5f, qt);
    const df p = df_add_f(df_add(r, df_mul(df_mul(r, r), q)), 1.0f);
    const int n = (int)kf;
    const df t = df_mul(T.exp2[n & 63], p);
    const float scale = __int_as_float(((n >> 6) + 127) << 23);
    return {t.hi * scale, t.lo * scale};
}

// Table-driven sin and cos of phi for |phi.hi| < 6000: phi = q pi/2 + s
// (Cody-Waite, as df_sincos), s = j pi/64 + r with |j| <= 16, |r| <= pi/128;
// sin s = S_j cos r + C_j sin r, cos s = C_j cos r - S_j sin r with
//   sin r = r (1 - r^2/6 + r^4/120 - r^6/5040),
//   cos r = 1 - r^2/2 + r^4/24 - r^6/720 + r^8/40320
// (remainders < 1e-19 relative); the angle-addition table method (e.g.
// J.-M. Muller, "Elementary Functions", ch. 6).
__device__ __forceinline__ void df_sincos_tab(df phi, const DfTables &T, const DfConsts &K,
                                              df &s_out, df &c_out) {
    const float qf = rintf(phi.hi * 0.636619772367581343076f);
    df s = df_two_sum(fmaf(-qf, K.pio2_1, phi.hi), phi.lo);
    s = df_add_f(s, -qf * K.pio2_2);
    s = df_add_f(s, -qf * K.pio2_3);
    s = df_add_f(s, -qf * K.pio2_4);
    float jf = rintf(s.hi * 20.371832715762604f);  // 64 / pi
    jf = fminf(fmaxf(jf, -16.0f), 16.0f);
    df r = df_two_sum(fmaf(-jf, K.pi64_1, s.hi), s.lo);  // exact product
    r = df_add_f(r, -jf * K.pi64_2);                      // exact product
    r = df_add_f(r, -jf * K.pi64_3);
    const df r2 = df_mul(r, r);
    const float x = r2.hi;
    const float ts = x * x * fmaf(-x, 1.0f / 5040.0f, 1.0f / 120.0f);
    const df sixth = {-0x1.555556p-3f, 0x1.555556p-28f};  // -1/6
    const df sr = df_mul(r, df_add_f(df_add_f(df_mul(r2, sixth), ts), 1.0f));
    const float tc = x * x * fmaf(fmaf(x, 1.0f / 40320.0f, -1.0f / 720.0f), x, 1.0f / 24.0f);
    const df cr = df_add_f(df_add_f(df{-0.5f * r2.hi, -0.5f * r2.lo}, tc), 1.0f);
    const int j = (int)jf + 16;
    const df S = T.sn[j], C = T.cs[j];
    const df sn = df_add(df_mul(S, cr), df_mul(C, sr));
    const df cs = df_sub(df_mul(C, cr), df_mul(S, sr));
    switch (((int)qf) & 3) {
        case 0: s_out = sn; c_out = cs; break;
        case 1: s_out = cs; c_out = df_neg(sn); break;
        case 2: s_out = df_neg(sn); c_out = df_neg(cs); break;
        default: s_out = df_neg(cs); c_out = sn; break;
    }
}

// ---------------------------------------------------------------------------
// Two double-float numbers side by side (lane x and lane y of each float2),
// on the packed FP32x2 instructions: every operation below performs, per
// lane, exactly the IEEE operations of its scalar counterpart above (a - b
// as fma(b, -1, a), one rounding), with half the instructions.
// ---------------------------------------------------------------------------
struct df2 {
    float2 hi, lo;
};

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 f2_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ df2 df2_make(df x, df y) { return {f2(x.hi, y.hi), f2(x.lo, y.lo)}; }
__device__ __forceinline__ df df2_x(df2 v) { return {v.hi.x, v.lo.x}; }
__device__ __forceinline__ df df2_y(df2 v) { return {v.hi.y, v.lo.y}; }

__device__ __forceinline__ df2 df2_two_sum(float2 a, float2 b) {
    const float2 s = f2_add(a, b);
    const float2 bb = f2_sub(s, a);
    const float2 e = f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb));
    return {s, e};
}

__device__ __forceinline__ df2 df2_fast_two_sum(float2 a, float2 b) {  // |a| >= |b|
    const float2 s = f2_add(a, b);
    const float2 e = f2_sub(b, f2_sub(s, a));
    return {s, e};
}

__device__ __forceinline__ df2 df2_add(df2 x, df2 y) {
    const df2 s = df2_two_sum(x.hi, y.hi);
    const float2 e = f2_add(s.lo, f2_add(x.lo, y.lo));
    return df2_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df2 df2_add_f(df2 x, float2 y) {
    const df2 s = df2_two_sum(x.hi, y);
    return df2_fast_two_sum(s.hi, f2_add(s.lo, x.lo));
}

__device__ __forceinline__ df2 df2_mul(df2 x, df2 y) {
    const float2 p = f2_mul(x.hi, y.hi);
    const float2 pe = f2_fma(x.hi, y.hi, f2_neg(p));
    const float2 e = f2_fma(x.hi, y.lo, f2_fma(x.lo, y.hi, pe));
    return df2_fast_two_sum(p, e);
}

}  // namespace gbs
