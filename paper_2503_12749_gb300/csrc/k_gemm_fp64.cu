// K2 + K3, FP64 path: propagation alpha' = T alpha, beta' = T* beta
// ("Applications to GBS") as a real GEMM of the row-interleaved operand
// A = [Re T_i.; Im T_i.] (2M x N) with B = [alpha_e, beta_e] (N x 2E), fused with
// the occupation epilogue
//   n'_i = alpha'_i beta'_i = (a_r + i a_i)(b_r - i b_i)
//        = (a_r b_r + a_i b_i) + i (a_i b_r - a_r b_i),
//   a = (Re T alpha, Im T alpha)_i, b = (Re T beta, Im T beta)_i,
// summed over the tile's output modes.  alpha', beta' never leave registers;
// the kernel writes one partial n_S per (mode tile, trajectory) and, on
// request (moments and marginals), every n'_i.
//
// Tile: 64 output modes x 32 trajectories per 256-thread block; each thread
// owns 4 modes x 2 trajectories (32 accumulators).  R is the arithmetic of
// the contraction: double (GBS_FP64, bound by the FP64 FMA rate) or float
// (GBS_FP32: T and the samples rounded to FP32 as they are staged, FP32
// products accumulated in FP32 along the N input modes); the occupation
// epilogue and everything after it is FP64 in both.
#include "gbs_internal.cuh"

#include <algorithm>
#include <climits>
#include <vector>

namespace gbs {
namespace {

constexpr int TM = kFp64TileModes;    // 64 modes -> 128 A rows
constexpr int TS = kFp64TileSamples;  // 32 trajectories -> 64 B rows
constexpr int KT = 16;                // K per smem stage

__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }

template <typename R>
__global__ void __launch_bounds__(256) k_gemm_fp64(const double *__restrict__ T64,
                                                   const double *__restrict__ B, int N, int M,
                                                   int64_t count, int64_t ld_part,
                                                   double2 *__restrict__ nS_part, OccOut64 occ) {
    __shared__ R As[KT][2 * TM + 1];
    __shared__ R Bs[KT][2 * TS + 1];
    __shared__ double2 red[16][TS];

    const int tid = threadIdx.x;
    const int tx = tid & 15;  // trajectory pair
    const int ty = tid >> 4;  // mode quad
    const int mtile = blockIdx.y;
    const int i0 = mtile * TM;
    const int64_t s0 = (int64_t)blockIdx.x * TS;

    R acc[4][2][2][2];  // [mode][Re/Im row][trajectory][alpha/beta]
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int d = 0; d < 2; ++d) acc[a][b][c][d] = R(0);

    for (int k0 = 0; k0 < N; k0 += KT) {
        // A tile: 128 rows x 16 k (row = 2*mode_local + re/im), 8 per thread
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int idx = tid + 256 * t;
            const int row = idx >> 4;
            const int kk = idx & 15;
            const int i = i0 + (row >> 1);
            const int k = k0 + kk;
            double v = 0.0;
            if (i < M && k < N) v = T64[((size_t)i * 2 + (row & 1)) * N + k];
            As[kk][row] = R(v);
        }
        // B tile: 64 rows x 16 k (row = 2*traj_local + alpha/beta), 4 per thread
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int idx = tid + 256 * t;
            const int row = idx >> 4;
            const int kk = idx & 15;
            const int64_t s = s0 + (row >> 1);
            const int k = k0 + kk;
            double v = 0.0;
            if (s < count && k < N) v = B[((size_t)s * 2 + (row & 1)) * N + k];
            Bs[kk][row] = R(v);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            R a[8], b[4];
#pragma unroll
            for (int t = 0; t < 8; ++t) a[t] = As[kk][ty * 8 + t];
#pragma unroll
            for (int t = 0; t < 4; ++t) b[t] = Bs[kk][tx * 4 + t];
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int ri = 0; ri < 2; ++ri)
#pragma unroll
                    for (int s = 0; s < 2; ++s)
#pragma unroll
                        for (int ab = 0; ab < 2; ++ab)
                            acc[m][ri][s][ab] = fma_r(a[2 * m + ri], b[2 * s + ab], acc[m][ri][s][ab]);
        }
        __syncthreads();
    }

    // occupation epilogue: sum of n'_i over this thread's 4 modes (and, on
    // request, each n'_i itself)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        double re = 0.0, im = 0.0;
        const int64_t traj = s0 + tx * 2 + s;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const double ar = (double)acc[m][0][s][0], ai = (double)acc[m][1][s][0];
            const double br = (double)acc[m][0][s][1], bi = (double)acc[m][1][s][1];
            const double ore = ar * br + ai * bi;
            const double oim = ai * br - ar * bi;
            if (occ.p && traj < count) {
                double *dst = occ.p + (size_t)(i0 + ty * 4 + m) * occ.ld + traj;
                dst[0] = ore;
                dst[occ.plane] = oim;
            }
            re += ore;
            im += oim;
        }
        red[ty][tx * 2 + s] = make_double2(re, im);
    }
    __syncthreads();
    if (tid < TS) {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            re += red[t][tid].x;
            im += red[t][tid].y;
        }
        const int64_t s = s0 + tid;
        if (s < count) nS_part[(size_t)mtile * ld_part + s] = make_double2(re, im);
    }
}

// FP64 FMA throughput probe: kChains independent accumulators per thread,
// `iters` steps; the sums are stored so that nothing is eliminated.
// kOuter: each step is an outer-product update acc[a][b] += x[a] y[b] (the
// register pattern of a GEMM's inner loop); otherwise every chain steps
// acc = acc m + c with the same m and c (operands shared by consecutive
// instructions).
template <int kChains, bool kOuter>
__global__ void __launch_bounds__(256) k_dfma_rate(double *__restrict__ out, int iters) {
    constexpr int kA = kChains / 4;
    double x[kA], y[4], acc[kChains];
#pragma unroll
    for (int a = 0; a < kA; ++a) x[a] = 1.0 + 1e-3 * a + 1e-9 * threadIdx.x;
#pragma unroll
    for (int b = 0; b < 4; ++b) y[b] = 1e-7 * (b + 1);
#pragma unroll
    for (int q = 0; q < kChains; ++q) acc[q] = kOuter ? 0.0 : 1e-3 * q + 1e-9 * threadIdx.x;
    const double m = 0.999999 + 1e-12 * threadIdx.x, c = 1e-7;
#pragma unroll 2
    for (int i = 0; i < iters; ++i) {
        if (kOuter) {
#pragma unroll
            for (int a = 0; a < kA; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a * 4 + b] = fma(x[a], y[b], acc[a * 4 + b]);
        } else {
#pragma unroll
            for (int q = 0; q < kChains; ++q) acc[q] = fma(acc[q], m, c);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += acc[q];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int kChains>
void launch_dfma_rate(bool outer, int blocks, int threads, cudaStream_t st, double *out,
                      int iters) {
    if (outer)
        k_dfma_rate<kChains, true><<<blocks, threads, 0, st>>>(out, iters);
    else
        k_dfma_rate<kChains, false><<<blocks, threads, 0, st>>>(out, iters);
}

}  // namespace

int launch_gemm_fp64(gbs_net *net, int64_t count, OccOut64 occ) {
    if (count <= 0) return GBS_OK;
    if (occ.p && occ.ld < count) return set_error(GBS_EINVAL, "occupation ld < count");
    const int64_t sblocks = (count + TS - 1) / TS;
    if (sblocks > 0x7fffffff) return set_error(GBS_EINVAL, "chunk too large");
    dim3 grid((unsigned)sblocks, (unsigned)net->mtiles);
    if (net->precision == GBS_FP32)
        k_gemm_fp64<float><<<grid, 256, 0, net->stream>>>(
            net->d_T64, static_cast<const double *>(net->d_B), net->N, net->M, count, net->chunk,
            net->d_nS_part, occ);
    else
        k_gemm_fp64<double><<<grid, 256, 0, net->stream>>>(
            net->d_T64, static_cast<const double *>(net->d_B), net->N, net->M, count, net->chunk,
            net->d_nS_part, occ);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace gbs

using namespace gbs;

extern "C" int gbs_measure_fp64_rate(void *stream, double *tflops) {
    if (!tflops) return set_error(GBS_EINVAL, "tflops is NULL");
    *tflops = 0.0;
    int dev = 0, sms = 0;
    GBS_CUDA_TRY(cudaGetDevice(&dev));
    GBS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int threads = 256, iters = 1 << 12, max_blocks = 8 * sms;
    double *out = nullptr;
    GBS_CUDA_TRY(cudaMallocAsync(&out, sizeof(double) * max_blocks * threads, st));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int rc = GBS_OK;
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess)
        rc = set_error(GBS_ECUDA, "event creation failed");
    double best = 0.0;
    // configurations: (operand pattern, accumulators per thread, blocks per
    // SM); each timed with CUDA events on `stream` over 3 launches after a
    // warm-up launch; the best rate over all of them
    const int cfg[8][3] = {{1, 8, 4}, {1, 16, 4}, {1, 16, 8}, {1, 32, 2},
                           {0, 8, 4}, {0, 8, 8}, {0, 16, 4}, {0, 16, 8}};
    for (int c = 0; c < 8 && rc == GBS_OK; ++c) {
        const bool outer = cfg[c][0] != 0;
        const int chains = cfg[c][1], blocks = cfg[c][2] * sms;
        for (int rep = 0; rep < 4 && rc == GBS_OK; ++rep) {
            cudaEventRecord(ev[0], st);
            if (chains == 8)
                launch_dfma_rate<8>(outer, blocks, threads, st, out, iters);
            else if (chains == 16)
                launch_dfma_rate<16>(outer, blocks, threads, st, out, iters);
            else
                launch_dfma_rate<32>(outer, blocks, threads, st, out, iters);
            cudaEventRecord(ev[1], st);
            float ms = 0.0f;
            if (cudaEventSynchronize(ev[1]) != cudaSuccess ||
                cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) {
                rc = set_error(GBS_ECUDA, "FP64 rate probe failed: %s",
                               cudaGetErrorString(cudaGetLastError()));
                break;
            }
            const double fmas = (double)chains * iters * threads * blocks;
            const double rate = ms > 0.0f ? 2.0 * fmas / (ms * 1e-3) / 1e12 : 0.0;
            if (rep > 0 && rate > best) best = rate;  // rep 0 warms up
        }
    }
    if (rc == GBS_OK) *tflops = best;
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    cudaFreeAsync(out, st);
    cudaStreamSynchronize(st);
    return rc;
}
