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
// owns 4 modes x 2 trajectories (32 FP64 accumulators).  This path is bound
// by the FP64 FMA rate.
#include "gbs_internal.cuh"

#include <algorithm>
#include <climits>
#include <vector>

namespace gbs {
namespace {

constexpr int TM = kFp64TileModes;    // 64 modes -> 128 A rows
constexpr int TS = kFp64TileSamples;  // 32 trajectories -> 64 B rows
constexpr int KT = 16;                // K per smem stage

__global__ void __launch_bounds__(256) k_gemm_fp64(const double *__restrict__ T64,
                                                   const double *__restrict__ B, int N, int M,
                                                   int64_t count, int64_t ld_part,
                                                   double2 *__restrict__ nS_part, OccOut64 occ) {
    __shared__ double As[KT][2 * TM + 1];
    __shared__ double Bs[KT][2 * TS + 1];
    __shared__ double2 red[16][TS];

    const int tid = threadIdx.x;
    const int tx = tid & 15;  // trajectory pair
    const int ty = tid >> 4;  // mode quad
    const int mtile = blockIdx.y;
    const int i0 = mtile * TM;
    const int64_t s0 = (int64_t)blockIdx.x * TS;

    double acc[4][2][2][2];  // [mode][Re/Im row][trajectory][alpha/beta]
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int d = 0; d < 2; ++d) acc[a][b][c][d] = 0.0;

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
            As[kk][row] = v;
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
            Bs[kk][row] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            double a[8], b[4];
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
                            acc[m][ri][s][ab] = fma(a[2 * m + ri], b[2 * s + ab], acc[m][ri][s][ab]);
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
            const double ar = acc[m][0][s][0], ai = acc[m][1][s][0];
            const double br = acc[m][0][s][1], bi = acc[m][1][s][1];
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
// each step an outer-product update acc[a][b] += x[a] y[b] (the register
// pattern of a GEMM's inner loop, distinct operand registers), `iters` steps;
// the sums are stored so that nothing is eliminated.
template <int kChains>
__global__ void __launch_bounds__(256) k_dfma_rate(double *__restrict__ out,
                                                  long long *__restrict__ cycles, int iters) {
    constexpr int kA = kChains / 4;
    const long long c0 = clock64();
    double x[kA], y[4], acc[kChains];
#pragma unroll
    for (int a = 0; a < kA; ++a) x[a] = 1.0 + 1e-3 * a + 1e-9 * threadIdx.x;
#pragma unroll
    for (int b = 0; b < 4; ++b) y[b] = 1e-7 * (b + 1);
#pragma unroll
    for (int q = 0; q < kChains; ++q) acc[q] = 0.0;
#pragma unroll 2
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int a = 0; a < kA; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a * 4 + b] = fma(x[a], y[b], acc[a * 4 + b]);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += acc[q];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t sm;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
        cycles[3 * blockIdx.x] = sm;
        cycles[3 * blockIdx.x + 1] = c0;
        cycles[3 * blockIdx.x + 2] = clock64();
    }
}

}  // namespace

int launch_gemm_fp64(gbs_net *net, int64_t count, OccOut64 occ) {
    if (count <= 0) return GBS_OK;
    if (occ.p && occ.ld < count) return set_error(GBS_EINVAL, "occupation ld < count");
    const int64_t sblocks = (count + TS - 1) / TS;
    if (sblocks > 0x7fffffff) return set_error(GBS_EINVAL, "chunk too large");
    dim3 grid((unsigned)sblocks, (unsigned)net->mtiles);
    k_gemm_fp64<<<grid, 256, 0, net->stream>>>(net->d_T64, static_cast<const double *>(net->d_B),
                                                net->N, net->M, count, net->chunk,
                                                net->d_nS_part, occ);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace gbs

using namespace gbs;

extern "C" int gbs_measure_fp64_rate(void *stream, double *tflops) {
    if (!tflops) return set_error(GBS_EINVAL, "tflops is NULL");
    *tflops = 0.0;
    int dev = 0, sms = 0, khz = 0;
    GBS_CUDA_TRY(cudaGetDevice(&dev));
    GBS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GBS_CUDA_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int threads = 256, iters = 1 << 13, max_blocks = 8 * sms;
    double *out = nullptr;
    long long *cyc = nullptr;
    GBS_CUDA_TRY(cudaMallocAsync(&out, sizeof(double) * max_blocks * threads, st));
    GBS_CUDA_TRY(cudaMallocAsync(&cyc, sizeof(long long) * 3 * max_blocks, st));
    std::vector<long long> h((size_t)3 * max_blocks);
    int rc = GBS_OK;
    double best = 0.0;
    // configurations: (accumulators per thread, blocks per SM); per launch
    // and SM the FMAs its blocks completed over the cycles of its own clock
    // from the first block's start to the last block's end (clock64 and
    // %smid recorded per block), so the rate does not depend on the clock the
    // probe happened to run at; the mean over SMs, the best over the
    // configurations and 3 launches each after a warm-up launch, at the
    // device's maximum clock
    const int cfg[6][2] = {{8, 4}, {8, 8}, {16, 4}, {16, 8}, {32, 2}, {32, 3}};
    for (int c = 0; c < 6 && rc == GBS_OK; ++c) {
        const int chains = cfg[c][0], per_sm = cfg[c][1], blocks = per_sm * sms;
        for (int rep = 0; rep < 4; ++rep) {
            if (chains == 8)
                k_dfma_rate<8><<<blocks, threads, 0, st>>>(out, cyc, iters);
            else if (chains == 16)
                k_dfma_rate<16><<<blocks, threads, 0, st>>>(out, cyc, iters);
            else
                k_dfma_rate<32><<<blocks, threads, 0, st>>>(out, cyc, iters);
            if (cudaMemcpyAsync(h.data(), cyc, sizeof(long long) * 3 * blocks,
                                cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = set_error(GBS_ECUDA, "FP64 rate probe failed: %s",
                               cudaGetErrorString(cudaGetLastError()));
                break;
            }
            // %smid numbers the physical SMs (not necessarily 0 .. sms - 1)
            constexpr int kMaxSmId = 1024;
            std::vector<long long> lo(kMaxSmId, LLONG_MAX), hi(kMaxSmId, LLONG_MIN);
            std::vector<int> nb(kMaxSmId, 0);
            for (int q = 0; q < blocks; ++q) {
                const long long sm = h[3 * q];
                if (sm < 0 || sm >= kMaxSmId) continue;
                lo[sm] = std::min(lo[sm], h[3 * q + 1]);
                hi[sm] = std::max(hi[sm], h[3 * q + 2]);
                ++nb[sm];
            }
            double sum = 0.0;
            int used = 0;
            for (int q = 0; q < kMaxSmId; ++q)
                if (nb[q] > 0 && hi[q] > lo[q]) {
                    sum += (double)chains * iters * threads * nb[q] / (double)(hi[q] - lo[q]);
                    ++used;
                }
            const double fma_per_clk_sm = used ? sum / used : 0.0;
            const double rate = 2.0 * fma_per_clk_sm * sms * (double)khz * 1e3 / 1e12;
            if (rep > 0 && rate > best) best = rate;  // rep 0 warms up
        }
    }
    if (rc == GBS_OK) *tflops = best;
    cudaFreeAsync(out, st);
    cudaFreeAsync(cyc, st);
    cudaStreamSynchronize(st);
    return rc;
}
