// K1: phase-space input sampler.
//
// Squeezed-vacuum inputs ("Applications to GBS"): per mode the +P density
// xi(alpha) xi(beta) e^{alpha beta} on the real plane is a bivariate Gaussian
// with covariance [[sinh r cosh r, sinh^2 r], [sinh^2 r, sinh r cosh r]],
// whose eigen-decomposition gives
//   alpha = sqrt(s+/2) w1 + sqrt(s-/2) w2,  beta = sqrt(s+/2) w1 - sqrt(s-/2) w2,
//   s+- = sinh(r) e^{+-r},  w1, w2 independent standard normals.
// The normals of trajectory e, input mode j come from one Philox-4x32-10 call
// (Salmon et al., SC'11) at counter (e_lo, e_hi, j, 0) with key (seed_lo,
// seed_hi): two 53-bit uniforms, then Box-Muller.  The same draws feed the
// matrix-P and +P estimators (both use the +P sampling procedure).
//
// Layouts written:
//   FP64 path: B[e][c][N] doubles, c = 0 (alpha), 1 (beta).
//   BF16 path: per 128-trajectory tile, 256 rows (128 alpha rows, then 128
//   beta rows); planes B0 = bf16(x), B1 = bf16(x - B0), B2 = bf16(x - B0 -
//   B1) stored plane-major, each plane K-blocked [ldK / 32][rows][32]
//   (mode j of row q at ((j / 32) * rows + q) * 32 + j % 32).
// Both also write n_e = sum_j alpha_j beta_j (FP64 result).
#include "gbs_internal.cuh"

namespace gbs {
namespace {

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

// 53-bit uniform in (0,1): 27 high bits of a, 26 high bits of b, +1/2 unit.
__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
    const double hi = (double)(a >> 5);
    const double lo = (double)(b >> 6);
    return (hi * 67108864.0 + lo + 0.5) * (1.0 / 9007199254740992.0);
}

// The same uniform rounded to FP32 (relative error ~2^-24 also near 0).
__device__ __forceinline__ float uniform53_f(uint32_t a, uint32_t b) {
    const float lo = ((float)(b >> 6) + 0.5f) * 1.1102230246251565e-16f;  // 2^-53
    return fmaf((float)(a >> 5), 7.450580596923828e-09f, lo);             // 2^-27
}

__device__ __forceinline__ void normals_fp64(uint64_t seed, uint64_t e, uint32_t j, double &w1,
                                             double &w2) {
    uint32_t c0 = (uint32_t)e, c1 = (uint32_t)(e >> 32), c2 = j, c3 = 0u;
    philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1 = uniform53(c0, c1);
    const double u2 = uniform53(c2, c3);
    const double rho = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    w1 = rho * c;
    w2 = rho * s;
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

// ---------------------------------------------------------------------------
// FP64 path: one warp per trajectory, lanes stride over input modes.
// ---------------------------------------------------------------------------
__global__ void k_sample_fp64(const double2 *__restrict__ sq, int N, uint64_t seed, uint64_t e0,
                              int64_t count, double *__restrict__ B, double *__restrict__ n_out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < count; i += nwarps) {
        const uint64_t e = e0 + (uint64_t)i;
        double *row_a = B + (size_t)i * 2 * N;
        double *row_b = row_a + N;
        double part = 0.0;
        for (int j = lane; j < N; j += 32) {
            double w1, w2;
            normals_fp64(seed, e, (uint32_t)j, w1, w2);
            const double2 q = sq[j];
            const double a = q.x * w1 + q.y * w2;
            const double b = q.x * w1 - q.y * w2;
            row_a[j] = a;
            row_b[j] = b;
            part += a * b;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if (lane == 0) n_out[i] = part;
    }
}

// ---------------------------------------------------------------------------
// BF16 split path: FP32 arithmetic; each lane handles 4 consecutive modes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split3(float x, __nv_bfloat16 &h0, __nv_bfloat16 &h1,
                                       __nv_bfloat16 &h2) {
    h0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h0);
    h1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(h1);
    h2 = __float2bfloat16_rn(r2);
}

template <bool kSfu>
__global__ void k_sample_bf16(const float2 *__restrict__ sq, int N, int ldK, int planesB,
                              size_t plane_stride, size_t rows, uint64_t seed, uint64_t e0,
                              int64_t count, __nv_bfloat16 *__restrict__ B,
                              double *__restrict__ n_out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < count; i += nwarps) {
        const uint64_t e = e0 + (uint64_t)i;
        const int64_t tile = i >> 7;
        const int q = (int)(i & 127);
        const size_t row_a = (size_t)(tile * 256 + q) * 32;
        const size_t row_b = (size_t)(tile * 256 + 128 + q) * 32;
        // Kahan-compensated FP32 partial of sum_j alpha_j beta_j
        float s = 0.0f, comp = 0.0f;
        for (int j0 = 4 * lane; j0 < N; j0 += 128) {
            __align__(8) __nv_bfloat16 a0[4], a1[4], a2[4], b0[4], b1[4], b2[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int j = j0 + t;
                float a = 0.0f, b = 0.0f;
                if (j < N) {
                    float w1, w2;
                    if (kSfu)
                        normals_fp32_sfu(seed, e, (uint32_t)j, w1, w2);
                    else
                        normals_fp32(seed, e, (uint32_t)j, w1, w2);
                    const float2 c = sq[j];
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
            if (j0 + 3 < ldK) {
                // ldK is a multiple of 32 and j0 of 4: the 4 modes lie in one
                // K block, 8-byte aligned
                const size_t blk = (size_t)(j0 >> 5) * rows * 32 + (size_t)(j0 & 31);
                const size_t oa = blk + row_a, ob = blk + row_b;
                *reinterpret_cast<uint2 *>(B + oa) = *reinterpret_cast<uint2 *>(a0);
                *reinterpret_cast<uint2 *>(B + ob) = *reinterpret_cast<uint2 *>(b0);
                if (planesB > 1) {
                    *reinterpret_cast<uint2 *>(B + plane_stride + oa) =
                        *reinterpret_cast<uint2 *>(a1);
                    *reinterpret_cast<uint2 *>(B + plane_stride + ob) =
                        *reinterpret_cast<uint2 *>(b1);
                }
                if (planesB > 2) {
                    *reinterpret_cast<uint2 *>(B + 2 * plane_stride + oa) =
                        *reinterpret_cast<uint2 *>(a2);
                    *reinterpret_cast<uint2 *>(B + 2 * plane_stride + ob) =
                        *reinterpret_cast<uint2 *>(b2);
                }
            }
        }
        double part = (double)s - (double)comp;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if (lane == 0) n_out[i] = part;
    }
}

int grid_for_warps(gbs_net *net, int64_t warps_needed, int threads) {
    const int64_t per_block = threads / 32;
    int64_t blocks = (warps_needed + per_block - 1) / per_block;
    const int64_t cap = (int64_t)net->sm_count * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

}  // namespace

int launch_sample_fp64(gbs_net *net, uint64_t seed, uint64_t e0, int64_t count) {
    if (count <= 0) return GBS_OK;
    const int threads = 256;
    k_sample_fp64<<<grid_for_warps(net, count, threads), threads, 0, net->stream>>>(
        net->d_sq64, net->N, seed, e0, count, static_cast<double *>(net->d_B), net->d_n);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int launch_sample_bf16(gbs_net *net, uint64_t seed, uint64_t e0, int64_t count) {
    if (count <= 0) return GBS_OK;
    const int threads = 256;
    const int64_t tiles = (net->chunk + kTcTileSamples - 1) / kTcTileSamples;
    const size_t rows = (size_t)tiles * 256;
    const size_t plane_stride = rows * net->ldK;
    auto kern = net->planesB == 2 ? k_sample_bf16<true> : k_sample_bf16<false>;
    kern<<<grid_for_warps(net, count, threads), threads, 0, net->stream>>>(
        net->d_sq32, net->N, net->ldK, net->planesB, plane_stride, rows, seed, e0, count,
        static_cast<__nv_bfloat16 *>(net->d_B), net->d_n);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace gbs
