// Normally-ordered photon-count moments and single-mode count marginals
// ("Photon-counting observables") from the per-mode occupations
// n'_j = alpha'_j beta'_j that the propagation GEMM writes for a chunk.
//
// Per trajectory (n = sum_k alpha_k beta_k, M = 2 parity case, T_0 = tanh n):
//   moments (Eq. moment):   matrix-P (n'_j)^m tanh(n)^(m mod 2),  +P (n'_j)^m;
//   marginals (Eq. projection_op with S = {j}, per trajectory Eq.
//   c-number-variable with n_S = n'_j):
//     matrix-P  (n'^c / c!) [cosh or sinh](n - n') / cosh n   (c even / odd),
//     +P        (n'^c / c!) e^{-n'}.
// With s = sign n, a = |n|, x = s n', L = -log(1 + e^{-2a}):
//   cosh(n - n') / cosh n = e^{-x + L} + e^{x - 2a + L},
//   sinh(n - n') / cosh n = s (e^{-x + L} - e^{x - 2a + L}),
// so no exponential overflows for any n.  Even orders of the matrix-P
// moments equal the +P ones trajectory by trajectory and are not summed
// twice.
//
// Work split: one CTA per output mode j (grid-stride), 256 threads.  A
// trajectory e belongs to sub-ensemble e mod N_R.  With N_R <= 128 the CTA
// runs K = floor(256 / N_R) replicas of every sub-ensemble: thread
// t = k N_R + r takes the k-th, (k + K)-th, ... trajectories of
// sub-ensemble r in the chunk, so that at each step the CTA reads K N_R
// consecutive trajectories (coalesced).  With N_R > 128 each thread takes
// whole sub-ensembles r = t, t + 256, ... in turn.  Values are summed in
// registers over runs of 32 trajectories (FP32 for BF16 networks, FP64 for
// FP64 networks) and the runs in FP64 in shared memory; the replicas are
// combined in a fixed order and added to the FP64 sub-ensemble sums
// acc[r][j][q], so a run is bitwise reproducible for a fixed chunking.
// FP32 arithmetic is used only while |Re n'| <= 40 and |n'| <= 40 (every
// product then stays below 2^100); other trajectories take the FP64 route.
#include "gbs_internal.cuh"

namespace gbs {
namespace {

constexpr int kMomThreads = 256;
constexpr int kRun = 32;

template <typename Real>
struct __align__(4 * sizeof(Real)) TrajPar {
    Real w;   // tanh n
    Real s;   // sign n (+1 at n = 0)
    Real L;   // -log(1 + e^{-2|n|})
    Real L2;  // L - 2|n|
};

template <int MM, int CM>
struct MomLayout {
    // q in [0, MM): +P Re n'^m (m = q + 1)
    // q in [MM, MM + MM/2): matrix-P tanh(n) Re n'^m, odd m = 2 (q - MM) + 1
    // q in [B0, B0 + CM + 1): matrix-P marginal, c = q - B0
    // q in [B1, B1 + CM + 1): +P marginal, c = q - B1
    static constexpr int B0 = MM + MM / 2;
    static constexpr int B1 = B0 + CM + 1;
    static constexpr int Q = B1 + CM + 1;
};

__device__ __forceinline__ void sin_cos(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void sin_cos(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }

// The contributions of one (mode, trajectory) element; add(q, value).
template <typename A, int MM, int CM, typename Add>
__device__ __forceinline__ void element(A re, A im, A w, A s, A L, A L2, Add &&add) {
    using Lay = MomLayout<MM, CM>;
    // moments
    A pr = re, pi = im;
    add(0, pr);
    add(MM, w * pr);
#pragma unroll
    for (int m = 2; m <= MM; ++m) {
        const A tr = pr * re - pi * im;
        pi = pr * im + pi * re;
        pr = tr;
        add(m - 1, pr);
        if (m & 1) add(MM + (m - 1) / 2, w * pr);
    }
    // marginals
    A sn, cs;
    sin_cos(im, &sn, &cs);
    const A eA = exp_(L - s * re);
    const A eB = exp_(s * re + L2);
    const A eP = exp_(-re);
    const A t1r = eA * cs, t1i = -s * (eA * sn);  // e^{-x + L}
    const A t2r = eB * cs, t2i = s * (eB * sn);   // e^{x - 2a + L}
    const A fer = t1r + t2r, fei = t1i + t2i;
    const A f_or = s * (t1r - t2r), f_oi = s * (t1i - t2i);
    const A ppr = eP * cs, ppi = -(eP * sn);
    A wr = A(1), wi = A(0);  // n'^c / c!
#pragma unroll
    for (int c = 0; c <= CM; ++c) {
        if (c > 0) {
            const A ic = A(1) / A(c);
            const A xr = (wr * re - wi * im) * ic;
            wi = (wr * im + wi * re) * ic;
            wr = xr;
        }
        const A fr = (c & 1) ? f_or : fer;
        const A fi = (c & 1) ? f_oi : fei;
        add(Lay::B0 + c, wr * fr - wi * fi);
        add(Lay::B1 + c, wr * ppr - wi * ppi);
    }
}

template <typename Real>
__global__ void k_moment_prep(const double *__restrict__ n, int64_t count,
                              TrajPar<Real> *__restrict__ par) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = n[i];
        const double a = fabs(x);
        const double L = -log1p(exp(-2.0 * a));
        TrajPar<Real> p;
        p.w = (Real)tanh(x);
        p.s = x < 0.0 ? Real(-1) : Real(1);
        p.L = (Real)L;
        p.L2 = (Real)(L - 2.0 * a);
        par[i] = p;
    }
}

template <typename Real, int MM, int CM>
__global__ void __launch_bounds__(kMomThreads)
    k_moments(const Real *__restrict__ occ, int64_t occ_plane, int64_t ld_occ,
              const TrajPar<Real> *__restrict__ par, int64_t count, int e0mod, int n_sub, int M,
              double *__restrict__ acc) {
    using Lay = MomLayout<MM, CM>;
    constexpr int Q = Lay::Q;
    extern __shared__ double sacc[];  // [Q][kMomThreads]
    const int t = threadIdx.x;
    const int K = n_sub <= kMomThreads / 2 ? kMomThreads / n_sub : 1;
    const int nslots = K * n_sub;
    const int64_t step = (int64_t)K * n_sub;
    for (int j = blockIdx.x; j < M; j += gridDim.x) {
        const Real *ore = occ + (size_t)j * ld_occ;
        const Real *oim = ore + occ_plane;
        for (int slot0 = 0; slot0 < nslots; slot0 += kMomThreads) {
            const int slot = slot0 + t;
            const bool active = slot < nslots;
            const int r = slot % n_sub;
            const int k = slot / n_sub;
#pragma unroll
            for (int q = 0; q < Q; ++q) sacc[q * kMomThreads + t] = 0.0;
            if (active) {
                const int64_t off = (int64_t)((r - e0mod + n_sub) % n_sub) + (int64_t)k * n_sub;
                Real part[Q];
#pragma unroll
                for (int q = 0; q < Q; ++q) part[q] = Real(0);
                int np = 0;
                auto add_part = [&](int q, Real v) { part[q] += v; };
                auto add_smem = [&](int q, double v) { sacc[q * kMomThreads + t] += v; };
                for (int64_t i = off; i < count; i += step) {
                    const Real re = ore[i], im = oim[i];
                    const TrajPar<Real> p = par[i];
                    bool fast = true;
                    if (sizeof(Real) == 4) fast = fabs((float)re) <= 40.0f && re * re + im * im <= Real(1600);
                    if (fast) {
                        element<Real, MM, CM>(re, im, p.w, p.s, p.L, p.L2, add_part);
                    } else {
                        element<double, MM, CM>((double)re, (double)im, (double)p.w, (double)p.s,
                                                (double)p.L, (double)p.L2, add_smem);
                    }
                    if (++np == kRun) {
#pragma unroll
                        for (int q = 0; q < Q; ++q) {
                            sacc[q * kMomThreads + t] += (double)part[q];
                            part[q] = Real(0);
                        }
                        np = 0;
                    }
                }
#pragma unroll
                for (int q = 0; q < Q; ++q) sacc[q * kMomThreads + t] += (double)part[q];
            }
            __syncthreads();
            if (K > 1) {
                // replicas k = 0..K-1 of sub-ensemble t, in order
                if (t < n_sub) {
                    double *dst = acc + ((size_t)t * M + j) * Q;
                    for (int q = 0; q < Q; ++q) {
                        double v = 0.0;
                        for (int kk = 0; kk < K; ++kk) v += sacc[q * kMomThreads + kk * n_sub + t];
                        dst[q] += v;
                    }
                }
            } else if (active) {
                double *dst = acc + ((size_t)r * M + j) * Q;
                for (int q = 0; q < Q; ++q) dst[q] += sacc[q * kMomThreads + t];
            }
            __syncthreads();
        }
    }
}

// mean over sub-ensembles of acc[r][j][q] / cnt[r] and its error; outputs
// [2][M][mmax] moments and [2][M][cmax + 1] marginals (matrix-P first).
template <int MM, int CM>
__global__ void k_moment_stats(const double *__restrict__ acc, const int64_t *__restrict__ cnt,
                               int n_sub, int M, int mmax, int cmax, double *__restrict__ mom,
                               double *__restrict__ smom, double *__restrict__ marg,
                               double *__restrict__ smarg) {
    using Lay = MomLayout<MM, CM>;
    constexpr int Q = Lay::Q;
    const int per_mode = 2 * mmax + 2 * (cmax + 1);
    const int64_t total = (int64_t)M * per_mode;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(id / per_mode);
        int o = (int)(id % per_mode);
        int q;
        double *out_m, *out_s;
        size_t idx;
        if (o < 2 * mmax) {
            const int est = o / mmax, m = o % mmax + 1;
            q = (est == 0 && (m & 1)) ? MM + (m - 1) / 2 : m - 1;
            out_m = mom;
            out_s = smom;
            idx = ((size_t)est * M + j) * mmax + (m - 1);
        } else {
            o -= 2 * mmax;
            const int est = o / (cmax + 1), c = o % (cmax + 1);
            q = (est == 0 ? Lay::B0 : Lay::B1) + c;
            out_m = marg;
            out_s = smarg;
            idx = ((size_t)est * M + j) * (cmax + 1) + c;
        }
        double mean = 0.0;
        for (int r = 0; r < n_sub; ++r) mean += acc[((size_t)r * M + j) * Q + q] / (double)cnt[r];
        mean /= (double)n_sub;
        double var = 0.0;
        for (int r = 0; r < n_sub; ++r) {
            const double d = acc[((size_t)r * M + j) * Q + q] / (double)cnt[r] - mean;
            var += d * d;
        }
        out_m[idx] = mean;
        out_s[idx] = n_sub > 1 ? sqrt(var / (double)(n_sub - 1)) / sqrt((double)n_sub) : 0.0;
    }
}

template <typename Real, int MM, int CM>
int launch_t(const MomentSpec &sp, const void *occ, int64_t occ_plane, int64_t ld_occ,
             const void *par, int64_t count, uint64_t e0, double *acc, cudaStream_t stream,
             int sm_count) {
    constexpr int Q = MomLayout<MM, CM>::Q;
    const size_t smem = (size_t)Q * kMomThreads * sizeof(double);
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        GBS_CUDA_TRY(cudaFuncSetAttribute(k_moments<Real, MM, CM>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set[dev] = true;
    }
    const int grid = std::min(sp.M, sm_count * 8);
    k_moments<Real, MM, CM><<<grid, kMomThreads, smem, stream>>>(
        static_cast<const Real *>(occ), occ_plane, ld_occ, static_cast<const TrajPar<Real> *>(par),
        count, (int)(e0 % (uint64_t)sp.n_sub), sp.n_sub, sp.M, acc);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace

size_t moment_par_bytes(bool fp64) { return fp64 ? sizeof(TrajPar<double>) : sizeof(TrajPar<float>); }

int moment_quantities(int mmax, int cmax) {
    const int MM = mmax <= 4 ? 4 : 8, CM = cmax <= 7 ? 7 : 15;
    return MM + MM / 2 + 2 * (CM + 1);
}

int launch_moment_prep(const double *n, int64_t count, bool fp64, void *par, cudaStream_t stream,
                       int sm_count) {
    if (count <= 0) return GBS_OK;
    const int grid = (int)std::min<int64_t>((count + 255) / 256, (int64_t)sm_count * 8);
    if (fp64)
        k_moment_prep<double><<<grid, 256, 0, stream>>>(n, count, static_cast<TrajPar<double> *>(par));
    else
        k_moment_prep<float><<<grid, 256, 0, stream>>>(n, count, static_cast<TrajPar<float> *>(par));
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int launch_moments(const MomentSpec &sp, bool fp64, const void *occ, int64_t occ_plane,
                   int64_t ld_occ, const void *par, int64_t count, uint64_t e0, double *acc,
                   cudaStream_t stream, int sm_count) {
    if (count <= 0) return GBS_OK;
    const bool m8 = sp.mmax > 4, c15 = sp.cmax > 7;
#define GBS_MOM_CASE(R, A, B)                                                                     \
    return launch_t<R, A, B>(sp, occ, occ_plane, ld_occ, par, count, e0, acc, stream, sm_count)
    if (fp64) {
        if (!m8 && !c15) GBS_MOM_CASE(double, 4, 7);
        if (!m8) GBS_MOM_CASE(double, 4, 15);
        if (!c15) GBS_MOM_CASE(double, 8, 7);
        GBS_MOM_CASE(double, 8, 15);
    }
    if (!m8 && !c15) GBS_MOM_CASE(float, 4, 7);
    if (!m8) GBS_MOM_CASE(float, 4, 15);
    if (!c15) GBS_MOM_CASE(float, 8, 7);
    GBS_MOM_CASE(float, 8, 15);
#undef GBS_MOM_CASE
}

int launch_moment_stats(const MomentSpec &sp, const double *acc, const int64_t *cnt, double *out,
                        cudaStream_t stream, int sm_count) {
    const size_t nm = (size_t)2 * sp.M * sp.mmax, nc = (size_t)2 * sp.M * (sp.cmax + 1);
    double *mom = out, *smom = out + nm, *marg = out + 2 * nm, *smarg = out + 2 * nm + nc;
    const int64_t total = (int64_t)sp.M * (2 * sp.mmax + 2 * (sp.cmax + 1));
    const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count * 8);
    const bool m8 = sp.mmax > 4, c15 = sp.cmax > 7;
    if (!m8 && !c15)
        k_moment_stats<4, 7><<<grid, 256, 0, stream>>>(acc, cnt, sp.n_sub, sp.M, sp.mmax, sp.cmax, mom, smom, marg, smarg);
    else if (!m8)
        k_moment_stats<4, 15><<<grid, 256, 0, stream>>>(acc, cnt, sp.n_sub, sp.M, sp.mmax, sp.cmax, mom, smom, marg, smarg);
    else if (!c15)
        k_moment_stats<8, 7><<<grid, 256, 0, stream>>>(acc, cnt, sp.n_sub, sp.M, sp.mmax, sp.cmax, mom, smom, marg, smarg);
    else
        k_moment_stats<8, 15><<<grid, 256, 0, stream>>>(acc, cnt, sp.n_sub, sp.M, sp.mmax, sp.cmax, mom, smom, marg, smarg);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace gbs
