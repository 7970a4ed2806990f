// Probability densities of per-trajectory observables (Appendix A): the
// +P projector G_+(m) = n_S^m e^{-n_S} / m! (Eq. phase_space_projector) and
// the matrix-P projector G_0(m) of the same trajectory,
//   G_0(m) = [e^{-n_S} n_S^m e^{n} + e^{n_S} (-n_S)^m e^{-n}] / (m! 2 cosh n)
// (the coefficient of z^m in cosh(n + (z-1) n_S) / cosh n, written with
// numerator and denominator times e^{-|n|}), binned by their real parts into
// equally spaced bins of [lo, hi) plus an underflow and an overflow bin.
// Counts are integers, so the histogram does not depend on the order in
// which trajectories arrive.
#include "gbs_internal.cuh"

#include <cmath>

namespace gbs {
namespace {

constexpr int kHistThreads = 256;

__global__ void k_histogram(const double *__restrict__ n_in, const double2 *__restrict__ nS_in,
                            int64_t count, HistSpec spec, unsigned long long *__restrict__ out) {
    extern __shared__ unsigned int s_cnt[];  // [2][nm][nbins + 2]
    const int per = spec.nbins + 2;
    const int total = 2 * spec.nm * per;
    for (int q = threadIdx.x; q < total; q += blockDim.x) s_cnt[q] = 0u;
    __syncthreads();
    const double inv_width = (double)spec.nbins / (spec.hi - spec.lo);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double n = n_in[i];
        const double2 s = nS_in[i];
        const double c = n - fabs(n);
        const double den = 1.0 + exp(-2.0 * fabs(n));
        const bool zero = s.x == 0.0 && s.y == 0.0;
        const double lr = 0.5 * log(s.x * s.x + s.y * s.y);  // log |n_S|
        const double la = atan2(s.y, s.x);                   // arg n_S
        for (int q = 0; q < spec.nm; ++q) {
            const int m = spec.m[q];
            double gm, gp;
            if (zero) {
                gp = (m == 0) ? 1.0 : 0.0;
                gm = (m == 0) ? (exp(c) + exp(-2.0 * n + c)) / den : 0.0;
            } else {
                // L = m log n_S - lgamma(m + 1)
                const double Lr = (double)m * lr - lgamma((double)m + 1.0);
                const double Li = (double)m * la;
                gp = exp(Lr - s.x) * cos(Li - s.y);                      // Re e^{L - n_S}
                const double t1 = exp(Lr - s.x + c) * cos(Li - s.y);
                const double t2 = exp(Lr + s.x - 2.0 * n + c) * cos(Li + s.y);
                gm = (t1 + ((m & 1) ? -t2 : t2)) / den;
            }
            const double v[2] = {gm, gp};
#pragma unroll
            for (int est = 0; est < 2; ++est) {
                const double x = (v[est] - spec.lo) * inv_width;
                int b;
                if (!(x >= 0.0))
                    b = 0;  // below lo, and NaN
                else if (x >= (double)spec.nbins)
                    b = per - 1;
                else
                    b = 1 + (int)x;
                atomicAdd(&s_cnt[(est * spec.nm + q) * per + b], 1u);
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < total; q += blockDim.x)
        if (s_cnt[q]) atomicAdd(&out[q], (unsigned long long)s_cnt[q]);
}

}  // namespace

int launch_histogram(gbs_net *net, int64_t count, const HistSpec &spec,
                     unsigned long long *out_dev) {
    if (count <= 0) return GBS_OK;
    const size_t smem = sizeof(unsigned int) * 2 * spec.nm * (spec.nbins + 2);
    int64_t blocks = (count + kHistThreads - 1) / kHistThreads;
    if (blocks > (int64_t)net->sm_count * 4) blocks = (int64_t)net->sm_count * 4;
    k_histogram<<<(int)blocks, kHistThreads, smem, net->stream>>>(net->d_n, net->d_nS, count, spec,
                                                                   out_dev);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace gbs
