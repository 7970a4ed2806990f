// K5: inverse DFT of the sub-ensemble means and the statistics over
// sub-ensembles (Eq. total_counts; sub-ensemble errors, Appendix A):
//   P_r(m) = (1/K1) sum_k <G>_r(z_k) z_k^{-m},   m = m_off + q, q = 0..K1-1,
//          = (1/K1) sum_k [<G>_r(z_k) z_k^{-m_off}] e^{-2 pi i k q / K1},
// a forward DFT of the pre-twiddled means, computed by a radix-2 Stockham
// autosort FFT in FP64 (one butterfly per thread per pass; e.g. Govindaraju
// et al., "High performance discrete Fourier transforms on graphics
// processors", SC'08).  Then P(m) = mean_r Re P_r(m) and
// sigma(m) = std_r(Re P_r(m)) / sqrt(N_R).
#include "gbs_internal.cuh"

namespace gbs {
namespace {

// a[b][k] = acc[b][k] / (count_r K1) * e^{-2 pi i k m_off / K1},  b = est*n_sub + r
__global__ void k_prep(const double2 *__restrict__ acc, const int64_t *__restrict__ counts,
                       int n_sub, int K1, int64_t mo, const double2 *__restrict__ wfft,
                       double2 *__restrict__ out) {
    const int64_t total = (int64_t)2 * n_sub * K1;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % K1);
        const int r = (int)((idx / K1) % n_sub);
        const double scale = 1.0 / ((double)counts[r] * (double)K1);
        const double2 w = wfft[(int)(((int64_t)k * mo) % K1)];
        const double2 a = acc[idx];
        out[idx] = make_double2((a.x * w.x - a.y * w.y) * scale, (a.x * w.y + a.y * w.x) * scale);
    }
}

// One radix-2 Stockham pass of size-K1 forward DFTs over `batch` rows.
__global__ void k_stockham(const double2 *__restrict__ x, double2 *__restrict__ y, int K1,
                           int Ns, int64_t batch, const double2 *__restrict__ wfft) {
    const int h = K1 >> 1;
    const int64_t total = batch * h;
    const int stride_tw = K1 / (2 * Ns);
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / h;
        const int j = (int)(idx - b * h);
        const double2 *xb = x + b * K1;
        double2 *yb = y + b * K1;
        const int kk = j & (Ns - 1);
        const double2 v0 = xb[j];
        const double2 u = xb[j + h];
        const double2 w = wfft[kk * stride_tw];
        const double2 v1 = make_double2(u.x * w.x - u.y * w.y, u.x * w.y + u.y * w.x);
        const int d = (j - kk) * 2 + kk;
        yb[d] = make_double2(v0.x + v1.x, v0.y + v1.y);
        yb[d + Ns] = make_double2(v0.x - v1.x, v0.y - v1.y);
    }
}

// out layout [P_mP | sig_mP | P_pP | sig_pP], each K1 doubles.
__global__ void k_stats(const double2 *__restrict__ Pr, int n_sub, int K1,
                        double *__restrict__ out) {
    const int64_t total = (int64_t)2 * K1;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int est = (int)(idx / K1);
        const int q = (int)(idx % K1);
        const double2 *p = Pr + (size_t)est * n_sub * K1 + q;
        double mean = 0.0;
        for (int r = 0; r < n_sub; ++r) mean += p[(size_t)r * K1].x;
        mean /= (double)n_sub;
        double var = 0.0;
        for (int r = 0; r < n_sub; ++r) {
            const double d = p[(size_t)r * K1].x - mean;
            var += d * d;
        }
        const double sd = n_sub > 1 ? sqrt(var / (double)(n_sub - 1)) : 0.0;
        out[(size_t)(2 * est) * K1 + q] = mean;
        out[(size_t)(2 * est + 1) * K1 + q] = sd / sqrt((double)n_sub);
    }
}

__global__ void k_count_nonfinite(const double2 *__restrict__ acc, int64_t total,
                                  unsigned long long *__restrict__ flag) {
    unsigned long long local = 0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = acc[idx];
        if (!isfinite(a.x) || !isfinite(a.y)) ++local;
    }
    if (local) atomicAdd(flag, local);
}

int blocks_for(gbs_net *net, int64_t work) {
    int64_t b = (work + 255) / 256;
    const int64_t cap = (int64_t)net->sm_count * 8;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

int launch_invert(gbs_net *net, int64_t m_offset, double *out_dev) {
    const int K1 = net->K1;
    const int64_t batch = (int64_t)2 * net->n_sub;
    int64_t mo = m_offset % K1;
    if (mo < 0) mo += K1;
    k_prep<<<blocks_for(net, batch * K1), 256, 0, net->stream>>>(
        net->d_acc, net->d_counts, net->n_sub, K1, mo, net->d_wfft, net->d_fft0);
    GBS_LAUNCH_CHECK();
    double2 *x = net->d_fft0, *y = net->d_fft1;
    for (int Ns = 1; Ns < K1; Ns <<= 1) {
        k_stockham<<<blocks_for(net, batch * (K1 / 2)), 256, 0, net->stream>>>(x, y, K1, Ns, batch,
                                                                                 net->d_wfft);
        GBS_LAUNCH_CHECK();
        double2 *tmp = x;
        x = y;
        y = tmp;
    }
    k_stats<<<blocks_for(net, 2 * (int64_t)K1), 256, 0, net->stream>>>(x, net->n_sub, K1, out_dev);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int launch_fft_rows(const double2 *wfft, int K, int64_t batch, double2 *x, double2 *y,
                    double2 **result, cudaStream_t stream, int sm_count) {
    const int64_t work = batch * (K / 2);
    int64_t b = (work + 255) / 256;
    if (b > (int64_t)sm_count * 8) b = (int64_t)sm_count * 8;
    if (b < 1) b = 1;
    for (int Ns = 1; Ns < K; Ns <<= 1) {
        k_stockham<<<(int)b, 256, 0, stream>>>(x, y, K, Ns, batch, wfft);
        GBS_LAUNCH_CHECK();
        double2 *tmp = x;
        x = y;
        y = tmp;
    }
    *result = x;
    return GBS_OK;
}

int launch_count_nonfinite(gbs_net *net) {
    GBS_CUDA_TRY(cudaMemsetAsync(net->d_flags, 0, sizeof(unsigned long long), net->stream));
    const int64_t total = (int64_t)2 * net->n_sub * net->K1;
    k_count_nonfinite<<<blocks_for(net, total), 256, 0, net->stream>>>(net->d_acc, total,
                                                                        net->d_flags);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace gbs
