// Device code of the BF16 phase-space sampler, shared by the standalone
// sampler kernel (k_sampler.cu) and the sampler warps of the propagation
// GEMM (k_gemm_tc.cu), which fill the next chunk's sample operand while the
// tensor cores work on the current one.  Both run the same instructions on
// the same counters, so the operand they write is bitwise the same.
//
// Squeezed-vacuum inputs ("Applications to GBS"): per mode the +P density
// xi(alpha) xi(beta) e^{alpha beta} on the real plane is a bivariate Gaussian
// with covariance [[sinh r cosh r, sinh^2 r], [sinh^2 r, sinh r cosh r]],
// whose eigen-decomposition gives
//   alpha = sqrt(s+/2) w1 + sqrt(s-/2) w2,  beta = sqrt(s+/2) w1 - sqrt(s-/2) w2,
//   s+- = sinh(r) e^{+-r},  w1, w2 independent standard normals.
// The normals of trajectory e, input mode j come from one Philox-4x32-10 call
// (Salmon et al., SC'11) at counter (e_lo, e_hi, j, 0) with key (seed_lo,
// seed_hi): two 53-bit uniforms, then Box-Muller.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

#include "gbs_internal.cuh"

namespace gbs {
namespace samp {

// Philox-4x32-10: ten rounds of two 32x32->64 multiplies (multipliers
// 0xD2511F53, 0xCD9E8D57) with the Weyl key schedule (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ void philox4x32_10(uint32_t &c0, uint32_t &c1, uint32_t &c2,
                                              uint32_t &c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// The 53-bit uniform (27 high bits of a, 26 high bits of b, +1/2 unit)
// rounded to FP32 (relative error ~2^-24 also near 0).
__device__ __forceinline__ float uniform53_f(uint32_t a, uint32_t b) {
    const float lo = ((float)(b >> 6) + 0.5f) * 1.1102230246251565e-16f;  // 2^-53
    return fmaf((float)(a >> 5), 7.450580596923828e-09f, lo);             // 2^-27
}

__device__ __forceinline__ void normals_fp32(uint64_t seed, uint64_t e, uint32_t j, float &w1,
                                             float &w2) {
    uint32_t c0 = (uint32_t)e, c1 = (uint32_t)(e >> 32), c2 = j, c3 = 0u;
    philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    // ln(u1): for u1 > 1/2 use log1p(-(1 - u1)); 1 - u1 is the same 53-bit
    // construction applied to the complemented words, so it is formed exactly
    // before rounding and keeps full FP32 relative precision near u1 = 1.
    const float u1 = uniform53_f(c0, c1);
    const float v1 = uniform53_f(~c0, ~c1);
    const float lnu = (v1 < 0.5f) ? log1pf(-v1) : logf(u1);
    const float u2 = uniform53_f(c2, c3);
    const float rho = sqrtf(-2.0f * lnu);
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    w1 = rho * c;
    w2 = rho * s;
}

// The same normals with the SFU approximations of ln and sin/cos (absolute
// errors ~2^-21 on these arguments) for the 3-product BF16 path, whose sample
// operand keeps two BF16 planes (~16 significant bits) of each amplitude:
// 2 pi u2 is shifted to [-pi, pi) (sin and cos change sign) where the SFU
// sine and cosine are specified.
__device__ __forceinline__ void normals_fp32_sfu(uint64_t seed, uint64_t e, uint32_t j, float &w1,
                                                 float &w2) {
    uint32_t c0 = (uint32_t)e, c1 = (uint32_t)(e >> 32), c2 = j, c3 = 0u;
    philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float u1 = uniform53_f(c0, c1);
    const float u2 = uniform53_f(c2, c3);
    const float rho = sqrtf(-2.0f * __logf(u1));
    float s, c;
    __sincosf(6.283185307179586f * (u2 - 0.5f), &s, &c);
    w1 = -rho * c;
    w2 = -rho * s;
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16 &h0, __nv_bfloat16 &h1,
                                       __nv_bfloat16 &h2) {
    h0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h0);
    h1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(h1);
    h2 = __float2bfloat16_rn(r2);
}

// Trajectory i of the job by one warp (lanes stride over input modes, 4
// modes per lane and step).  Layout written: per 128-trajectory tile, 256
// rows (128 alpha rows, then 128 beta rows); planes B0 = bf16(x), B1 =
// bf16(x - B0), B2 = bf16(x - B0 - B1) stored plane-major, each plane
// K-blocked [ldK / 32][rows][32] (mode j of row q at ((j / 32) * rows + q) *
// 32 + j % 32); n_e = sum_j alpha_j beta_j (Kahan-compensated FP32 partials
// per lane, summed in FP64).  kSfu: the 2-plane (3-product) operand, SFU ln
// and sin/cos.  kStream: stores that L2 evicts first (the operand is read
// again only by the next GEMM).
template <bool kSfu, bool kStream>
__device__ __forceinline__ void sample_trajectory_bf16(const SampleJob &jb, int64_t i, int lane) {
    const int planes = kSfu ? 2 : jb.planesB;
    const uint64_t e = jb.e0 + (uint64_t)i;
    const int64_t tile = i >> 7;
    const int q = (int)(i & 127);
    const size_t row_a = (size_t)(tile * 256 + q) * 32;
    const size_t row_b = (size_t)(tile * 256 + 128 + q) * 32;
    float s = 0.0f, comp = 0.0f;
    // modes N..ldK-1 (the K padding) are written as zeros, so the operand
    // needs no clearing before its first use
    for (int j0 = 4 * lane; j0 < jb.ldK; j0 += 128) {
        __align__(8) __nv_bfloat16 a0[4], a1[4], a2[4], b0[4], b1[4], b2[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = j0 + t;
            float a = 0.0f, b = 0.0f;
            if (j < jb.N) {
                float w1, w2;
                if (kSfu)
                    normals_fp32_sfu(jb.seed, e, (uint32_t)j, w1, w2);
                else
                    normals_fp32(jb.seed, e, (uint32_t)j, w1, w2);
                const float2 c = jb.sq[j];
                a = fmaf(c.x, w1, c.y * w2);
                b = fmaf(c.x, w1, -c.y * w2);
                const float y = fmaf(a, b, -comp);
                const float tsum = s + y;
                comp = (tsum - s) - y;
                s = tsum;
            }
            split3(a, a0[t], a1[t], a2[t]);
            split3(b, b0[t], b1[t], b2[t]);
        }
        if (j0 + 3 < jb.ldK) {
            // ldK is a multiple of 32 and j0 of 4: the 4 modes lie in one
            // K block, 8-byte aligned
            const size_t blk = (size_t)(j0 >> 5) * jb.rows * 32 + (size_t)(j0 & 31);
            const size_t oa = blk + row_a, ob = blk + row_b;
            auto put = [&](size_t o, const __nv_bfloat16 *v) {
                const uint2 w = *reinterpret_cast<const uint2 *>(v);
                uint2 *p = reinterpret_cast<uint2 *>(jb.B + o);
                if (kStream) __stcs(p, w);
                else *p = w;
            };
            put(oa, a0);
            put(ob, b0);
            if (planes > 1) {
                put(jb.plane_stride + oa, a1);
                put(jb.plane_stride + ob, b1);
            }
            if (planes > 2) {
                put(2 * jb.plane_stride + oa, a2);
                put(2 * jb.plane_stride + ob, b2);
            }
        }
    }
    double part = (double)s - (double)comp;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if (lane == 0) jb.n_out[i] = part;
}

// Trajectories warp, warp + nwarps, ... of the job, one warp each.
template <bool kSfu, bool kStream>
__device__ __forceinline__ void sample_warps_bf16(const SampleJob &jb, int64_t warp, int64_t nwarps,
                                                  int lane) {
    for (int64_t i = warp; i < jb.count; i += nwarps) sample_trajectory_bf16<kSfu, kStream>(jb, i, lane);
}

}  // namespace samp
}  // namespace gbs
