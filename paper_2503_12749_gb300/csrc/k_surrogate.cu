// The surrogate's representation of a network and of its count distribution
// (features, their statistics and standardisation, encoding a distribution
// into the network's output grid and decoding an output back into P(m)).
// Not part of the paper; the distribution it represents is the binned total
// count of Eq. total_counts.  Definitions:
//   mu  = t^2 sum_j sinh^2 r_j,  s^2 = sum_j [t^2 sinh^2 r_j + t^4 sinh^2 r_j cosh 2 r_j]
//   (mean and variance of the total count for T = t U, from the cumulants of
//   the uniform-loss determinant generating function);
//   grid x_i = -8 + 16 (i + 1/2) / 256, output o[p*256 + i] = 100 (f_p(x_i) - phi(x_i)/2),
//   f_p(x) = (s/2) P(mu + s x) on the counts of parity p;
//   interpolation: Catmull-Rom cubic (Catmull & Rom 1974) in Hermite form.
// Every reduction runs in a fixed order, so results do not depend on timing.
#include "gbs_internal.cuh"
#include "gbs_surrogate.h"

#include <cmath>
#include <vector>

namespace gbs {
namespace {

constexpr int kGrid = GBS_SUR_GRID;
constexpr int kRec = GBS_SUR_RECORD;
constexpr int kFeat = GBS_SUR_FEATURES;
constexpr double kXLo = -8.0;
constexpr double kDx = 16.0 / kGrid;
constexpr double kOutScale = 100.0;
constexpr double kInvSqrt2Pi = 0.3989422804014327;  // 1 / sqrt(2 pi)

struct NetIn {
    double t;
    int64_t m_off;
    int64_t r0;
    int N, M, K1, pad;
};

__device__ __forceinline__ double cr(double ym1, double y0, double y1, double y2, double u) {
    const double u2 = u * u, u3 = u2 * u;
    const double h00 = 2.0 * u3 - 3.0 * u2 + 1.0;
    const double h10 = u3 - 2.0 * u2 + u;
    const double h01 = -2.0 * u3 + 3.0 * u2;
    const double h11 = u3 - u2;
    return h00 * y0 + h10 * 0.5 * (y1 - ym1) + h01 * y1 + h11 * 0.5 * (y2 - y0);
}

__device__ __forceinline__ double half_phi(double x) { return 0.5 * kInvSqrt2Pi * exp(-0.5 * x * x); }

template <int kThreadsT>
__device__ __forceinline__ double block_sum(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = kThreadsT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double s = red[0];
    __syncthreads();
    return s;
}

// One block (256 threads) per network.
__global__ void k_sur_features(const NetIn *__restrict__ nets, const double *__restrict__ r,
                               double *__restrict__ rec) {
    __shared__ double red[256];
    const NetIn n = nets[blockIdx.x];
    const double *rj = r + n.r0;
    const double eta = n.t * n.t;
    double s1 = 0.0, s2 = 0.0, s3 = 0.0, lo = INFINITY, hi = -INFINITY;
    for (int j = threadIdx.x; j < n.N; j += blockDim.x) {
        const double x = rj[j];
        const double sh = sinh(x);
        const double sh2 = sh * sh;
        s1 += x;
        s2 += eta * sh2;
        s3 += eta * sh2 + eta * eta * sh2 * cosh(2.0 * x);
        lo = fmin(lo, x);
        hi = fmax(hi, x);
    }
    const double sum_r = block_sum<256>(s1, red);
    const double mu = block_sum<256>(s2, red);
    const double var = block_sum<256>(s3, red);
    // min / max
    red[threadIdx.x] = lo;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    const double rmin = red[0];
    __syncthreads();
    red[threadIdx.x] = hi;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    const double rmax = red[0];
    __syncthreads();
    const double mean = sum_r / (double)n.N;
    double d2 = 0.0;
    for (int j = threadIdx.x; j < n.N; j += blockDim.x) {
        const double d = rj[j] - mean;
        d2 += d * d;
    }
    const double ss = block_sum<256>(d2, red);
    if (threadIdx.x == 0) {
        double *o = rec + (size_t)blockIdx.x * kRec;
        const double s = sqrt(var);
        o[0] = log((double)n.N);
        o[1] = log((double)n.M);
        o[2] = mean;
        o[3] = sqrt(ss / (double)n.N);
        o[4] = rmin;
        o[5] = rmax;
        o[6] = n.t;
        o[7] = log2((double)n.K1);
        o[8] = log(mu);
        o[9] = log(s);
        o[10] = mu;
        o[11] = s;
        o[12] = (double)n.m_off;
        o[13] = (double)n.K1;
    }
}

// One block of 32 x kFeat threads: warp f handles feature f.
__global__ void k_sur_stats(const double *__restrict__ rec, int count, double *__restrict__ stats) {
    const int f = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    double s = 0.0, lo = INFINITY, hi = -INFINITY;
    for (int i = lane; i < count; i += 32) {
        const double x = rec[(size_t)i * kRec + f];
        s += x;
        lo = fmin(lo, x);
        hi = fmax(hi, x);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const double mean = s / (double)count;
    double d2 = 0.0;
    for (int i = lane; i < count; i += 32) {
        const double d = rec[(size_t)i * kRec + f] - mean;
        d2 += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    if (lane == 0) {
        stats[f] = mean;
        stats[kFeat + f] = sqrt(d2 / (double)count);
        stats[2 * kFeat + f] = lo;
        stats[3 * kFeat + f] = hi;
    }
}

__global__ void k_sur_standardize(const double *__restrict__ rec, int count,
                                  const double *__restrict__ stats, float *__restrict__ X,
                                  int *__restrict__ in_domain) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int ok = 1;
    for (int f = 0; f < kFeat; ++f) {
        const double u = rec[(size_t)i * kRec + f];
        const double sd = stats[kFeat + f];
        X[(size_t)i * kFeat + f] = sd > 1e-12 ? (float)((u - stats[f]) / sd) : 0.0f;
        const double lo = stats[2 * kFeat + f], hi = stats[3 * kFeat + f];
        const double pad = 0.02 * (hi - lo);
        if (!(u >= lo - pad && u <= hi + pad)) ok = 0;
    }
    if (in_domain) in_domain[i] = ok;
}

// One block of 2 * kGrid threads per network: output o = p * kGrid + i.
__global__ void k_sur_encode(const double *__restrict__ rec, const double *__restrict__ P,
                             int64_t ldP, float *__restrict__ Y) {
    const double *q = rec + (size_t)blockIdx.x * kRec;
    const double mu = q[10], s = q[11];
    const int64_t m_off = (int64_t)q[12];
    const int64_t K1 = min((int64_t)q[13], ldP);
    const double *Pn = P + (size_t)blockIdx.x * ldP;
    const int p = threadIdx.x / kGrid;
    const int i = threadIdx.x % kGrid;
    const double x = kXLo + kDx * (i + 0.5);
    const double pos = (mu + s * x - p) / 2.0;  // on the lattice m = p + 2 pos
    const double q0 = floor(pos);
    const double u = pos - q0;
    double y[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int64_t m = p + 2 * ((int64_t)q0 + d - 1);
        const int64_t j = m - m_off;
        y[d] = (j >= 0 && j < K1) ? Pn[j] : 0.0;
    }
    const double f = 0.5 * s * cr(y[0], y[1], y[2], y[3], u);
    Y[(size_t)blockIdx.x * 2 * kGrid + threadIdx.x] = (float)(kOutScale * (f - half_phi(x)));
}

// One block (256 threads) per network: P(m) on the window, then renormalised.
__global__ void k_sur_decode(const double *__restrict__ rec, const float *__restrict__ Y,
                             double *__restrict__ P, int64_t ldP) {
    __shared__ double f[2][kGrid];
    __shared__ double red[256];
    const double *q = rec + (size_t)blockIdx.x * kRec;
    const double mu = q[10], s = q[11];
    const int64_t m_off = (int64_t)q[12];
    const int64_t K1 = min((int64_t)q[13], ldP);
    const float *o = Y + (size_t)blockIdx.x * 2 * kGrid;
    for (int k = threadIdx.x; k < 2 * kGrid; k += blockDim.x) {
        const double x = kXLo + kDx * ((k % kGrid) + 0.5);
        f[k / kGrid][k % kGrid] = (double)o[k] / kOutScale + half_phi(x);
    }
    __syncthreads();
    double *Pn = P + (size_t)blockIdx.x * ldP;
    double part = 0.0;
    for (int64_t j = threadIdx.x; j < K1; j += blockDim.x) {
        const int64_t m = m_off + j;
        const int p = (int)(m & 1);
        const double g = ((m - mu) / s - (kXLo + 0.5 * kDx)) / kDx;
        double v = 0.0;
        if (g >= 0.0 && g <= kGrid - 1) {
            const double g0 = floor(g);
            const int i0 = (int)g0;
            const double u = g - g0;
            double y[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const int ii = i0 + d - 1;
                y[d] = (ii >= 0 && ii < kGrid) ? f[p][ii] : 0.0;
            }
            v = 2.0 / s * fmax(cr(y[0], y[1], y[2], y[3], u), 0.0);
        }
        Pn[j] = v;
        part += v;
    }
    const double total = block_sum<256>(part, red);
    if (total > 0.0) {
        const double inv = 1.0 / total;
        for (int64_t j = threadIdx.x; j < K1; j += blockDim.x) Pn[j] *= inv;
    }
}

int check_records(int count, const void *feat) {
    if (count < 1) return set_error(GBS_EINVAL, "count must be >= 1");
    if (count > 2147483647 / 512) return set_error(GBS_EINVAL, "count too large");
    if (!feat) return set_error(GBS_EINVAL, "feature records are NULL");
    return GBS_OK;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" {

int gbs_surrogate_features(int count, const int *N, const int *M, const double *t, const int *K1,
                           const int64_t *m_off, const double *r, const int64_t *r_off, void *stream,
                           double *feat_dev) {
    int rc;
    if ((rc = check_records(count, feat_dev))) return rc;
    if (!N || !M || !t || !K1 || !m_off || !r || !r_off)
        return set_error(GBS_EINVAL, "NULL host array");
    if (r_off[0] != 0) return set_error(GBS_EINVAL, "r_off[0] must be 0");
    std::vector<NetIn> h((size_t)count);
    for (int i = 0; i < count; ++i) {
        if (N[i] < 1 || M[i] < 1 || r_off[i + 1] - r_off[i] != N[i])
            return set_error(GBS_EINVAL, "network %d: N, M >= 1 and r_off[i+1] - r_off[i] = N", i);
        if (K1[i] < 2 || K1[i] > (1 << 24) || (K1[i] & (K1[i] - 1)))
            return set_error(GBS_EINVAL, "network %d: K1 must be a power of two in [2, 2^24]", i);
        if (!(t[i] > 0.0 && t[i] <= 1.0)) return set_error(GBS_EINVAL, "network %d: t outside (0, 1]", i);
        if (m_off[i] < 0) return set_error(GBS_EINVAL, "network %d: m_off < 0", i);
        h[(size_t)i] = NetIn{t[i], m_off[i], r_off[i], N[i], M[i], K1[i], 0};
    }
    const int64_t nr = r_off[count];
    for (int64_t j = 0; j < nr; ++j)
        if (!(std::isfinite(r[j]) && r[j] > 0.0))
            return set_error(GBS_EINVAL, "r[%lld] must be finite and > 0", (long long)j);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    NetIn *d_nets = nullptr;
    double *d_r = nullptr;
    if (cudaMalloc(&d_nets, sizeof(NetIn) * (size_t)count) != cudaSuccess ||
        cudaMalloc(&d_r, sizeof(double) * (size_t)nr) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_nets);
        return set_error(GBS_ENOMEM, "upload buffers for the features");
    }
    rc = GBS_OK;
    if (cudaMemcpyAsync(d_nets, h.data(), sizeof(NetIn) * (size_t)count, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_r, r, sizeof(double) * (size_t)nr, cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = set_error(GBS_ECUDA, "upload of the network parameters failed");
    if (!rc) {
        k_sur_features<<<count, 256, 0, s>>>(d_nets, d_r, feat_dev);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = set_error(GBS_ECUDA, "feature kernel: %s", cudaGetErrorString(e));
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && !rc)
        rc = set_error(GBS_ECUDA, "feature kernel failed");
    cudaFree(d_nets);
    cudaFree(d_r);
    return rc;
}

int gbs_surrogate_feature_stats(int count, const double *feat_dev, void *stream, double *stats_dev) {
    int rc;
    if ((rc = check_records(count, feat_dev))) return rc;
    if (!stats_dev) return set_error(GBS_EINVAL, "stats_dev is NULL");
    k_sur_stats<<<1, 32 * kFeat, 0, static_cast<cudaStream_t>(stream)>>>(feat_dev, count, stats_dev);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int gbs_surrogate_standardize(int count, const double *feat_dev, const double *stats_dev,
                              void *stream, float *X_dev, int *in_domain_dev) {
    int rc;
    if ((rc = check_records(count, feat_dev))) return rc;
    if (!stats_dev || !X_dev) return set_error(GBS_EINVAL, "NULL device array");
    k_sur_standardize<<<(count + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        feat_dev, count, stats_dev, X_dev, in_domain_dev);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int gbs_surrogate_encode(int count, const double *feat_dev, const double *P_dev, int64_t ldP,
                         void *stream, float *Y_dev) {
    int rc;
    if ((rc = check_records(count, feat_dev))) return rc;
    if (!P_dev || !Y_dev || ldP < 1) return set_error(GBS_EINVAL, "NULL device array or ldP < 1");
    k_sur_encode<<<count, 2 * kGrid, 0, static_cast<cudaStream_t>(stream)>>>(feat_dev, P_dev, ldP,
                                                                             Y_dev);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int gbs_surrogate_decode(int count, const double *feat_dev, const float *Y_dev, void *stream,
                         double *P_dev, int64_t ldP) {
    int rc;
    if ((rc = check_records(count, feat_dev))) return rc;
    if (!P_dev || !Y_dev || ldP < 1) return set_error(GBS_EINVAL, "NULL device array or ldP < 1");
    k_sur_decode<<<count, 256, 0, static_cast<cudaStream_t>(stream)>>>(feat_dev, Y_dev, P_dev, ldP);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // extern "C"
