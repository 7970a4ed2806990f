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
// Both also write n_e = sum_j alpha_j beta_j (FP64 result).  The BF16 path's
// device code (sampler_dev.cuh) also runs in the spare warps of the
// 3-product GEMM, which sample the next chunk.
#include "gbs_internal.cuh"
#include "sampler_dev.cuh"

namespace gbs {
namespace {

// 53-bit uniform in (0,1): 27 high bits of a, 26 high bits of b, +1/2 unit.
__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
    const double hi = (double)(a >> 5);
    const double lo = (double)(b >> 6);
    return (hi * 67108864.0 + lo + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ void normals_fp64(uint64_t seed, uint64_t e, uint32_t j, double &w1,
                                             double &w2) {
    uint32_t c0 = (uint32_t)e, c1 = (uint32_t)(e >> 32), c2 = j, c3 = 0u;
    samp::philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1 = uniform53(c0, c1);
    const double u2 = uniform53(c2, c3);
    const double rho = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    w1 = rho * c;
    w2 = rho * s;
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
template <bool kSfu>
__global__ void k_sample_bf16(const SampleJob job) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    samp::sample_warps_bf16<kSfu, false>(job, warp, nwarps, lane);
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
    net->pre_valid = false;  // the operands are overwritten
    if (count <= 0) return GBS_OK;
    const int threads = 256;
    k_sample_fp64<<<grid_for_warps(net, count, threads), threads, 0, net->stream>>>(
        net->d_sq64, net->N, seed, e0, count, static_cast<double *>(net->d_B), net->d_n);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

SampleJob sample_job_bf16(gbs_net *net, void *B, double *n, uint64_t seed, uint64_t e0,
                          int64_t count) {
    SampleJob j;
    const int64_t tiles = (net->chunk + kTcTileSamples - 1) / kTcTileSamples;
    j.sq = net->d_sq32;
    j.B = static_cast<__nv_bfloat16 *>(B);
    j.n_out = n;
    j.rows = (size_t)tiles * 256;
    j.plane_stride = j.rows * net->ldK;
    j.seed = seed;
    j.e0 = e0;
    j.count = count;
    j.N = net->N;
    j.ldK = net->ldK;
    j.planesB = net->planesB;
    return j;
}

int launch_sample_bf16(gbs_net *net, uint64_t seed, uint64_t e0, int64_t count) {
    net->pre_valid = false;  // the operands are overwritten
    if (count <= 0) return GBS_OK;
    const int threads = 256;
    const SampleJob job = sample_job_bf16(net, net->d_B, net->d_n, seed, e0, count);
    auto kern = net->planesB == 2 ? k_sample_bf16<true> : k_sample_bf16<false>;
    kern<<<grid_for_warps(net, count, threads), threads, 0, net->stream>>>(job);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace gbs
