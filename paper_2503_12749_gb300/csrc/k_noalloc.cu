// gbs_binned_counts_noalloc: the inverse DFT and sub-ensemble statistics of
// gbs_binned_counts_device for callers that cannot allocate device memory.
//
// The caller passes the sub-ensemble sums, their counts and the output
// buffer; the FFT work buffers and the twiddle table live in one file-scope
// device array of fixed size (kNaWork complex entries per work buffer, K1 <=
// kNaMaxK1), reserved on every GPU that loads this library until the process
// exits.  No call allocates: not the entry point, not its kernels.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device (that device current) looks the address up once with
// cudaGetSymbolAddress and caches it; make that first call before capturing
// any stream.  Every call shares the array and overwrites all of it that it
// reads, so nothing carries over from the previous call; calls whose work
// overlaps on the GPU (different streams, or different host threads on the
// same device without ordering) race on the array.
#include "gbs_internal.cuh"

#include <mutex>

namespace gbs {
namespace {

constexpr int64_t kNaWork = (int64_t)1 << 20;  // complex entries per FFT work buffer
constexpr int kNaMaxK1 = 1 << 16;              // twiddle-table entries
constexpr int kNaMaxDevices = 64;

// [work buffer 0 | work buffer 1 | twiddles e^{-2 pi i k / K1}]
static __device__ __align__(256) double2 g_na_scratch[2 * kNaWork + kNaMaxK1];

std::mutex g_na_mutex;
double2 *g_na_addr[kNaMaxDevices] = {};

__global__ void k_na_twiddle(int K1, double2 *__restrict__ wfft) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K1; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)K1, &s, &c);
        wfft[k] = make_double2(c, -s);
    }
}

// a[b][k] = acc[b][k] / (counts[r] K1) * e^{-2 pi i k m_off / K1}, b = est*n_sub + r
__global__ void k_na_prep(const double2 *__restrict__ acc, const int64_t *__restrict__ counts,
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

// One radix-2 Stockham pass (forward DFT) over all rows.
__global__ void k_na_stockham(const double2 *__restrict__ x, double2 *__restrict__ y, int K1,
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

// out = [P_mP | sig_mP | P_plusP | sig_plusP], each K1 doubles
__global__ void k_na_stats(const double2 *__restrict__ Pr, int n_sub, int K1,
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

int na_blocks(int64_t work) {
    int64_t b = (work + 255) / 256;
    if (b > 4096) b = 4096;
    return b < 1 ? 1 : (int)b;
}

// Device address of the scratch array on the current device (looked up once per device).
int na_scratch(double2 **out) {
    int dev = -1;
    GBS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices)
        return set_error(GBS_ENOTSUP, "device ordinal %d beyond the %d supported", dev,
                         kNaMaxDevices);
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        cudaError_t err = cudaGetSymbolAddress(&p, g_na_scratch);
        if (err != cudaSuccess || !p)
            return set_error(GBS_ECUDA, "cudaGetSymbolAddress(scratch) failed on device %d: %s",
                             dev, cudaGetErrorString(err));
        g_na_addr[dev] = static_cast<double2 *>(p);
    }
    *out = g_na_addr[dev];
    return GBS_OK;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" int gbs_binned_counts_noalloc(const double *acc_dev, const int64_t *counts_dev,
                                         int n_sub, int K1, int64_t m_offset, double *out_dev,
                                         void *stream) {
    if (!acc_dev || !counts_dev || !out_dev)
        return set_error(GBS_EINVAL, "acc_dev, counts_dev and out_dev must be device pointers");
    if (n_sub < 1 || n_sub > 65535) return set_error(GBS_EINVAL, "n_sub must be in [1, 65535]");
    if (K1 < 2 || (K1 & (K1 - 1)) != 0 || K1 > kNaMaxK1)
        return set_error(GBS_EINVAL, "K1 must be a power of two in [2, %d]", kNaMaxK1);
    const int64_t batch = (int64_t)2 * n_sub;
    if (batch * K1 > kNaWork)
        return set_error(GBS_EINVAL,
                         "2 * n_sub * K1 = %lld exceeds the fixed scratch of %lld complex "
                         "entries",
                         (long long)(batch * K1), (long long)kNaWork);
    double2 *base = nullptr;
    int rc;
    if ((rc = na_scratch(&base))) return rc;
    double2 *w0 = base, *w1 = base + kNaWork, *wfft = base + 2 * kNaWork;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t mo = m_offset % K1;
    if (mo < 0) mo += K1;
    k_na_twiddle<<<na_blocks(K1), 256, 0, s>>>(K1, wfft);
    GBS_LAUNCH_CHECK();
    k_na_prep<<<na_blocks(batch * K1), 256, 0, s>>>(reinterpret_cast<const double2 *>(acc_dev),
                                                   counts_dev, n_sub, K1, mo, wfft, w0);
    GBS_LAUNCH_CHECK();
    double2 *x = w0, *y = w1;
    for (int Ns = 1; Ns < K1; Ns <<= 1) {
        k_na_stockham<<<na_blocks(batch * (K1 / 2)), 256, 0, s>>>(x, y, K1, Ns, batch, wfft);
        GBS_LAUNCH_CHECK();
        double2 *t = x;
        x = y;
        y = t;
    }
    k_na_stats<<<na_blocks(2 * (int64_t)K1), 256, 0, s>>>(x, n_sub, K1, out_dev);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}
