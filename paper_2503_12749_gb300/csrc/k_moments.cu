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
// Work split: one CTA per (output mode j, trajectory segment).  A
// trajectory e belongs to sub-ensemble e mod N_R.  With N_R <= 128 the CTA
// runs K = floor(256 / N_R) replicas of every sub-ensemble: thread
// t = k N_R + r takes the k-th, (k + K)-th, ... trajectories of
// sub-ensemble r, so that the CTA's threads cover K N_R consecutive
// trajectories at a time; the CTA has K N_R threads rounded up to whole
// warps.  With N_R > 128 each thread takes whole sub-ensembles r = t,
// t + 256, ... in turn (one pass over the segment per 256).  A mode's
// occupations of a trajectory range are contiguous, so the CTA streams its
// segment in tiles of 4 KB per plane (Re n', Im n' and the per-trajectory
// parameters) with bulk asynchronous copies into a 3-stage shared-memory
// ring (one thread issues, an mbarrier per stage, every wait bounded), and
// the threads evaluate their trajectories of a tile out of shared memory.
// Values are summed in registers over runs of 64 trajectories (FP32 for
// BF16 networks, FP64 for FP64 networks) and the runs in FP64 in shared
// memory; the replicas are combined in a fixed order.  The tiles of a chunk
// are cut into S segments (S chosen so that the M S CTAs fill the GPU's
// waves evenly); segment sums go to a scratch array and are added to the
// FP64 sub-ensemble sums acc[r][j][q] in segment order, so a run is bitwise
// reproducible for a fixed chunking.
//
// On the FP32 route the exponentials come from one SFU exp and one
// reciprocal, and the sine and cosine from the SFU after a Cody-Waite
// reduction (relative errors below 3e-6 at |Re n'| = 40, a few 1e-7 near 1;
// the FP32 occupations carry 2^-14 of their amplitude scale):
// with e^{L - 2a} = e^{-2a} / (1 + e^{-2a}) and e^{L} = 1 - e^{L - 2a} per
// trajectory, e^{-x + L} and e^{x - 2a + L} are e^{-Re n'} or e^{Re n'} times
// those, and the marginals' 1/c! is applied to the summed values.  The route
// is taken only while |Re n'| <= B and |n'| <= B, B = 40 for c <= 7 and 20
// for c <= 15 (every unscaled product then stays below 2^95); other
// trajectories take an FP64 route that evaluates the exponents in log form
// from n itself.
#include "gbs_internal.cuh"
#include "tc_ptx.cuh"
#include "dfloat.cuh"

#include <algorithm>
#include <cmath>

namespace gbs {
namespace {

constexpr int kMaxThreads = 256;
constexpr int kRun = 128;
constexpr int kMaxSeg = 4;

// Per-trajectory parameters.  FP32 route: (tanh n, e^{L - 2a}), from which
// sign n = sign(tanh n) and e^{L} = 1 - e^{L - 2a} (8 bytes, re-read for
// every mode from L2); FP64 route (FP64 networks): (tanh n, sign n, L, L - 2a).
template <typename Real>
struct TrajPar;
template <>
struct __align__(8) TrajPar<float> {
    float w;
    float l2;
};
template <>
struct __align__(32) TrajPar<double> {
    double w;
    double s;
    double l1;
    double l2;
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

// FP32 route (|x| <= 40): Cody-Waite reduction by 2 pi with a two-part
// constant (C1 = 6.28125 has 9 significant bits, so k C1 is exact for the
// |k| <= 7 used here), then the SFU sine and cosine on [-pi, pi] (absolute
// error about 2^-21).
__device__ __forceinline__ void sin_cos(float x, float *s, float *c) {
    const float k = rintf(x * 0.159154943091895336f);
    float r = fmaf(-k, 6.28125f, x);
    r = fmaf(-k, 1.93530717958647692e-3f, r);
    __sincosf(r, s, c);
}
__device__ __forceinline__ void sin_cos(double x, double *s, double *c) { sincos(x, s, c); }

// The contributions of one (mode, trajectory) element, given n' = re + i im,
// w = tanh n, s = sign n and the three exponentials
//   eA = e^{-s Re n' + L},  eB = e^{s Re n' + L - 2a},  eP = e^{-Re n'};
// add(q, value).  kFact = false leaves out the marginals' 1/c! (the caller
// applies it to the summed values).
template <typename A, int MM, int CM, bool kFact, typename Add>
__device__ __forceinline__ void element(A re, A im, A w, A s, A eA, A eB, A eP, Add &&add) {
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
    // marginals: e^{-x + L} (cos, -s sin), e^{x - 2a + L} (cos, s sin) of Im n'
    A sn, cs;
    sin_cos(im, &sn, &cs);
    const A t1r = eA * cs, t1i = -s * (eA * sn);
    const A t2r = eB * cs, t2i = s * (eB * sn);
    const A fer = t1r + t2r, fei = t1i + t2i;
    const A f_or = s * (t1r - t2r), f_oi = s * (t1i - t2i);
    const A ppr = eP * cs, ppi = -(eP * sn);
    A wr = A(1), wi = A(0);  // n'^c (/ c!)
#pragma unroll
    for (int c = 0; c <= CM; ++c) {
        if (c > 0) {
            A xr = wr * re - wi * im;
            A xi = wr * im + wi * re;
            if (kFact) {
                const A ic = A(1) / A(c);
                xr *= ic;
                xi *= ic;
            }
            wr = xr;
            wi = xi;
        }
        const A fr = (c & 1) ? f_or : fer;
        const A fi = (c & 1) ? f_oi : fei;
        add(Lay::B0 + c, wr * fr - wi * fi);
        add(Lay::B1 + c, wr * ppr - wi * ppi);
    }
}

// The FP32 route's element with its sums in pairs on the packed FP32x2
// instructions: pair k < KM holds the moment quantities q = 2k, 2k + 1
// (+P Re n'^m for q < MM; matrix-P tanh(n) Re n'^m of odd m above), pair
// KM + c the matrix-P and +P marginal terms of count c (q = B0 + c, B1 + c);
// marginal factors unscaled (1/c! applied to the sums).
template <int MM, int CM>
__device__ __forceinline__ void element_f2(float re, float im, float w, float s, float eA, float eB,
                                           float eP, float2 (&pp)[MomLayout<MM, CM>::Q / 2]) {
    constexpr int KM = (MM + MM / 2) / 2;
    // moments: Re n'^m, m = 1..MM
    float prs[MM];
    float pr = re, pi = im;
    prs[0] = re;
#pragma unroll
    for (int m = 2; m <= MM; ++m) {
        const float tr = pr * re - pi * im;
        pi = pr * im + pi * re;
        pr = tr;
        prs[m - 1] = pr;
    }
#pragma unroll
    for (int k = 0; k < MM / 2; ++k) pp[k] = f2_add(pp[k], f2(prs[2 * k], prs[2 * k + 1]));
#pragma unroll
    for (int k = 0; k < MM / 4; ++k)
        pp[MM / 2 + k] = f2_fma(f2(w, w), f2(prs[4 * k], prs[4 * k + 2]), pp[MM / 2 + k]);
    // marginals: e^{-x + L} (cos, -s sin), e^{x - 2a + L} (cos, s sin) of Im n'
    float sn, cs;
    sin_cos(im, &sn, &cs);
    const float t1r = eA * cs, t1i = -s * (eA * sn);
    const float t2r = eB * cs, t2i = s * (eB * sn);
    const float fer = t1r + t2r, fei = t1i + t2i;
    const float f_or = s * (t1r - t2r), f_oi = s * (t1i - t2i);
    const float ppr = eP * cs, ppi = -(eP * sn);
    float wr = 1.0f, wi = 0.0f;  // n'^c, unscaled
#pragma unroll
    for (int c = 0; c <= CM; ++c) {
        if (c > 0) {
            const float xr = wr * re - wi * im;
            wi = wr * im + wi * re;
            wr = xr;
        }
        const float fr = (c & 1) ? f_or : fer;
        const float fi = (c & 1) ? f_oi : fei;
        pp[KM + c] = f2_fma(f2(wr, wr), f2(fr, ppr), f2_fma(f2(-wi, -wi), f2(fi, ppi), pp[KM + c]));
    }
}

// FP64 route from n itself (log form of the exponents).
template <int MM, int CM, bool kFact, typename Add>
__device__ __forceinline__ void element_log(double re, double im, double n, Add &&add) {
    const double a = fabs(n);
    const double L = -log1p(exp(-2.0 * a));
    const double s = n < 0.0 ? -1.0 : 1.0;
    element<double, MM, CM, kFact>(re, im, tanh(n), s, exp(L - s * re),
                                   exp(s * re + L - 2.0 * a), exp(-re), add);
}

template <typename Real>
__global__ void k_moment_prep(const double *__restrict__ n, int64_t count,
                              TrajPar<Real> *__restrict__ par) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = n[i];
        const double a = fabs(x);
        const double q = exp(-2.0 * a);
        TrajPar<Real> p;
        if constexpr (sizeof(Real) == sizeof(float)) {
            p.w = (float)tanh(x);
            p.l2 = (float)(q / (1.0 + q));
        } else {
            const double L = -log1p(q);
            p.w = tanh(x);
            p.s = x < 0.0 ? -1.0 : 1.0;
            p.l1 = L;
            p.l2 = L - 2.0 * a;
        }
        par[i] = p;
    }
}

// Shared-memory layout of k_moments: the FP64 run sums [Q][T], then kStages
// stages of one tile (Re n', Im n', per-trajectory parameters), then the
// stages' mbarriers.
template <typename Real>
struct MomTile {
    static constexpr int TT = 4096 / (int)sizeof(Real);  // trajectories per tile (at most)
    static constexpr int kStages = 2;
    // a tile's copies start at the 16-byte boundary at or below its first
    // trajectory: room for the shift
    static constexpr int kAlignOcc = 16 / (int)sizeof(Real);
    static constexpr int kAlignPar =
        sizeof(TrajPar<Real>) >= 16 ? 1 : 16 / (int)sizeof(TrajPar<Real>);
    static constexpr size_t kOccBytes = ((size_t)(TT + kAlignOcc) * sizeof(Real) + 15) / 16 * 16;
    static constexpr size_t kParBytes =
        ((size_t)(TT + kAlignPar) * sizeof(TrajPar<Real>) + 15) / 16 * 16;
    static constexpr size_t kStageBytes = 2 * kOccBytes + kParBytes;
};

template <typename Real, int MM>
size_t mom_smem_bytes(int Q, int T) {
    return (size_t)Q * T * sizeof(double) + MomTile<Real>::kStages * MomTile<Real>::kStageBytes +
           MomTile<Real>::kStages * sizeof(uint64_t);
}

// One bulk copy global -> shared completing on an mbarrier (both addresses
// 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
        : "memory");
}

template <typename Real, int MM, int CM>
__global__ void __launch_bounds__(kMaxThreads)
    k_moments(const Real *__restrict__ occ, int64_t occ_plane, int64_t ld_occ,
              const TrajPar<Real> *__restrict__ par, const double *__restrict__ nvals,
              int64_t count, int e0mod, int n_sub, int M, int K, int64_t L, int tiles_per_seg,
              double *__restrict__ out, int accumulate, unsigned long long *err_ptr) {
    using Lay = MomLayout<MM, CM>;
    using Tl = MomTile<Real>;
    constexpr int Q = Lay::Q;
    constexpr int NS = Tl::kStages;
    // FP32 route bound on |Re n'| and |n'|: every unscaled n'^c e^{|Re n'|}
    // (c <= CM), and a run of kRun of them, stays below 2^101
    constexpr float kFastBound = CM <= 7 ? 40.0f : 20.0f;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int j = blockIdx.x;
    const int seg = blockIdx.y;
    double *sacc = reinterpret_cast<double *>(smem_raw);  // [Q][T]
    uint8_t *stage_base = smem_raw + (size_t)Q * T * sizeof(double);
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage_base + NS * Tl::kStageBytes);
    auto st_re = [&](int sidx) {
        return reinterpret_cast<Real *>(stage_base + sidx * Tl::kStageBytes);
    };
    auto st_im = [&](int sidx) {
        return reinterpret_cast<Real *>(stage_base + sidx * Tl::kStageBytes + Tl::kOccBytes);
    };
    auto st_par = [&](int sidx) {
        return reinterpret_cast<TrajPar<Real> *>(stage_base + sidx * Tl::kStageBytes +
                                                 2 * Tl::kOccBytes);
    };
    volatile unsigned long long *err = err_ptr;

    const int nslots = K * n_sub;
    const int64_t step = (int64_t)K * n_sub;
    const Real *ore = occ + (size_t)j * ld_occ;
    const Real *oim = ore + occ_plane;
    double *dst_base = out + (accumulate ? 0 : (size_t)seg * n_sub * M * Q);
    const int64_t ntiles_all = (count + L - 1) / L;
    const int64_t tile0 = (int64_t)seg * tiles_per_seg;
    const int nt = (int)std::max<int64_t>(0, std::min<int64_t>(tiles_per_seg, ntiles_all - tile0));

    if (t == 0) {
        for (int q = 0; q < NS; ++q) ptx::mbar_init(ptx::smem_u32(&bars[q]), 1);
        ptx::fence_barrier_init();
    }
    __syncthreads();

    // tile g (g-th of the segment) = trajectories [a, b), a = (tile0 + g) L,
    // into stage sidx; the copies start at the 16-byte boundaries a_o <= a
    // (occupations) and a_p <= a (parameters)
    auto issue = [&](int g, int sidx) {
        const int64_t a = (tile0 + g) * L;
        const int64_t b = std::min<int64_t>(a + L, count);
        const int64_t a_o = a - a % Tl::kAlignOcc, a_p = a - a % Tl::kAlignPar;
        const uint32_t b_occ = (uint32_t)((((b - a_o) * (int64_t)sizeof(Real)) + 15) / 16 * 16);
        const uint32_t b_par =
            (uint32_t)((((b - a_p) * (int64_t)sizeof(TrajPar<Real>)) + 15) / 16 * 16);
        const uint32_t bar = ptx::smem_u32(&bars[sidx]);
        ptx::mbar_arrive_expect_tx(bar, 2 * b_occ + b_par);
        bulk_copy(ptx::smem_u32(st_re(sidx)), ore + a_o, b_occ, bar);
        bulk_copy(ptx::smem_u32(st_im(sidx)), oim + a_o, b_occ, bar);
        bulk_copy(ptx::smem_u32(st_par(sidx)), par + a_p, b_par, bar);
    };

    int64_t gtile = 0;  // tiles issued so far by this CTA (stage g % NS, phase (g / NS) & 1)
    bool ok = true;
    for (int slot0 = 0; slot0 < nslots; slot0 += T) {
        const int slot = slot0 + t;
        const bool active = slot < nslots;
        const int r = slot % n_sub;
        const int k = slot / n_sub;
        const int64_t off = (int64_t)((r - e0mod + n_sub) % n_sub) + (int64_t)k * n_sub;
#pragma unroll
        for (int q = 0; q < Q; ++q) sacc[q * T + t] = 0.0;
        // FP64 route: per-quantity sums; FP32 route: sums in pairs (element_f2)
        Real part[Q];
        float2 pp[Q / 2];
#pragma unroll
        for (int q = 0; q < Q; ++q) part[q] = Real(0);
#pragma unroll
        for (int k = 0; k < Q / 2; ++k) pp[k] = f2(0.0f, 0.0f);
        int np = 0;
        auto add_part = [&](int q, Real v) { part[q] += v; };
        auto add_smem = [&](int q, double v) { sacc[q * T + t] += v; };
        auto flush = [&]() {
            if constexpr (sizeof(Real) == sizeof(float)) {
                constexpr int KM = (MM + MM / 2) / 2;
#pragma unroll
                for (int k = 0; k < Q / 2; ++k) {
                    const int q0 = k < KM ? 2 * k : Lay::B0 + (k - KM);
                    const int q1 = k < KM ? 2 * k + 1 : Lay::B1 + (k - KM);
                    sacc[q0 * T + t] += (double)pp[k].x;
                    sacc[q1 * T + t] += (double)pp[k].y;
                    pp[k] = f2(0.0f, 0.0f);
                }
            } else {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    sacc[q * T + t] += (double)part[q];
                    part[q] = Real(0);
                }
            }
        };
        const int64_t g0 = gtile;
        if (t == 0)
            for (int g = 0; g < NS - 1 && g < nt; ++g) issue(g, (int)((g0 + g) % NS));
        for (int lt = 0; lt < nt; ++lt) {
            const int64_t gi = g0 + lt;
            const int sidx = (int)(gi % NS);
            // the stage of tile lt + NS - 1 was last read for tile lt - 1,
            // released by the barrier that ended that iteration
            if (t == 0 && lt + NS - 1 < nt) issue(lt + NS - 1, (int)((gi + NS - 1) % NS));
            const bool landed = ptx::mbar_wait(ptx::smem_u32(&bars[sidx]), (uint32_t)((gi / NS) & 1), err);
            ok = ok && landed;
            if (landed && active) {
                const int64_t a = (tile0 + lt) * L;
                const int64_t b = std::min<int64_t>(a + L, count);
                const Real *sre = st_re(sidx) + a % Tl::kAlignOcc;
                const Real *sim = st_im(sidx) + a % Tl::kAlignOcc;
                const TrajPar<Real> *spar = st_par(sidx) + a % Tl::kAlignPar;
                for (int64_t i = a + ((off - a % step) % step + step) % step; i < b; i += step) {
                    const int u = (int)(i - a);
                    const Real c_re = sre[u], c_im = sim[u];
                    const TrajPar<Real> c_p = spar[u];
                    if constexpr (sizeof(Real) == sizeof(float)) {
                        if (fabsf(c_re) <= kFastBound &&
                            c_re * c_re + c_im * c_im <= kFastBound * kFastBound) {
                            const float eP = __expf(-c_re);
                            const float iP = __frcp_rn(eP);
                            const bool neg = c_p.w < 0.0f;
                            const float sg = neg ? -1.0f : 1.0f;
                            const float eL = 1.0f - c_p.l2;
                            element_f2<MM, CM>(c_re, c_im, c_p.w, sg, (neg ? iP : eP) * eL,
                                               (neg ? eP : iP) * c_p.l2, eP, pp);
                        } else {
                            element_log<MM, CM, false>((double)c_re, (double)c_im, nvals[i],
                                                       add_smem);
                        }
                    } else {
                        element<Real, MM, CM, true>(c_re, c_im, c_p.w, c_p.s,
                                                    exp(c_p.l1 - c_p.s * c_re),
                                                    exp(c_p.s * c_re + c_p.l2), exp(-c_re),
                                                    add_part);
                    }
                    if (++np == kRun) {
                        flush();
                        np = 0;
                    }
                }
            }
            __syncthreads();
        }
        gtile = g0 + nt;
        if (active) flush();
        __syncthreads();
        if (K > 1) {
            // replicas k = 0..K-1 of sub-ensemble t, in order
            if (t < n_sub) {
                double *dst = dst_base + ((size_t)t * M + j) * Q;
                for (int q = 0; q < Q; ++q) {
                    double v = 0.0;
                    for (int kk = 0; kk < K; ++kk) v += sacc[q * T + kk * n_sub + t];
                    dst[q] = accumulate ? dst[q] + v : v;
                }
            }
        } else if (active) {
            double *dst = dst_base + ((size_t)r * M + j) * Q;
            for (int q = 0; q < Q; ++q)
                dst[q] = accumulate ? dst[q] + sacc[q * T + t] : sacc[q * T + t];
        }
        __syncthreads();
    }
    // after a timed-out wait, copies of this CTA may still be in flight: wait
    // (again bounded, ignoring the flag) for the last phase of every stage
    if (!ok && t == 0) {
        for (int q = 0; q < NS && q < gtile; ++q) {
            const int64_t last = gtile - 1 - ((gtile - 1 - q) % NS);  // last tile in stage q
            const uint32_t bar = ptx::smem_u32(&bars[last % NS]);
            const uint64_t t0 = ptx::globaltimer();
            while (!ptx::mbar_try_wait(bar, (uint32_t)((last / NS) & 1)))
                if (ptx::globaltimer() - t0 > 1000000000ull) break;
        }
    }
}

// acc[idx] += sum over segments s = 0..S-1 (in order) of part[s][idx].
__global__ void k_moment_combine(const double *__restrict__ part, int S, int64_t total,
                                 double *__restrict__ acc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int s = 0; s < S; ++s) v += part[(size_t)s * total + i];
        acc[i] += v;
    }
}

// mean over sub-ensembles of acc[r][j][q] / cnt[r] and its error; outputs
// [2][M][mmax] moments and [2][M][cmax + 1] marginals (matrix-P first).
template <int MM, int CM>
__global__ void k_moment_stats(const double *__restrict__ acc, const int64_t *__restrict__ cnt,
                               int n_sub, int M, int mmax, int cmax, int unscaled,
                               double *__restrict__ mom, double *__restrict__ smom,
                               double *__restrict__ marg, double *__restrict__ smarg) {
    using Lay = MomLayout<MM, CM>;
    constexpr int Q = Lay::Q;
    const int per_mode = 2 * mmax + 2 * (cmax + 1);
    const int64_t total = (int64_t)M * per_mode;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(id / per_mode);
        int o = (int)(id % per_mode);
        int q;
        double *out_m, *out_s, scale = 1.0;
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
            if (unscaled)
                for (int d = 2; d <= c; ++d) scale /= (double)d;  // 1 / c!
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
        out_m[idx] = scale * mean;
        out_s[idx] = n_sub > 1 ? scale * sqrt(var / (double)(n_sub - 1)) / sqrt((double)n_sub) : 0.0;
    }
}

// CTA shape for n_sub: replicas K and threads.
void cta_shape(int n_sub, int *K, int *threads) {
    if (n_sub <= kMaxThreads / 2) {
        *K = kMaxThreads / n_sub;
        *threads = ((*K * n_sub + 31) / 32) * 32;
    } else {
        *K = 1;
        *threads = std::min(kMaxThreads, ((n_sub + 31) / 32) * 32);
    }
}

template <typename Real, int MM, int CM>
int launch_t(const MomentSpec &sp, const void *occ, int64_t occ_plane, int64_t ld_occ,
             const void *par, const double *nvals, int64_t count, uint64_t e0, double *acc,
             double *scratch, int max_seg, unsigned long long *err, cudaStream_t stream,
             int sm_count, int *nlaunch) {
    constexpr int Q = MomLayout<MM, CM>::Q;
    constexpr int TT = MomTile<Real>::TT;
    int K, T;
    cta_shape(sp.n_sub, &K, &T);
    const size_t smem = mom_smem_bytes<Real, MM>(Q, T);
    static bool attr_set[64] = {};
    int dev = 0;
    GBS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(GBS_ECUDA, "device index out of range");
    if (!attr_set[dev]) {
        GBS_CUDA_TRY(cudaFuncSetAttribute(k_moments<Real, MM, CM>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)mom_smem_bytes<Real, MM>(Q, kMaxThreads)));
        attr_set[dev] = true;
    }
    int nb = 0;
    GBS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_moments<Real, MM, CM>, T, smem));
    nb = std::max(nb, 1);
    // tiles of whole rows of K N_R trajectories (every thread then has the
    // same number per tile), at most TT; rows longer than TT are cut
    const int64_t step = (int64_t)K * sp.n_sub;
    const int64_t L = step <= TT ? (TT / step) * step : (int64_t)TT;
    // segments: the S in 1..max_seg whose M S CTAs fill their last wave best
    // (a larger S must gain more than 1 %), each segment >= 4 tiles
    const int64_t ntiles = (count + L - 1) / L;
    const int64_t conc = (int64_t)nb * sm_count;
    int S = 1;
    double best = -1.0;
    for (int s = 1; s <= max_seg; ++s) {
        if (s > 1 && ntiles / s < 4) break;
        const double waves = (double)((int64_t)sp.M * s) / (double)conc;
        const double eff = waves / std::ceil(waves);
        if (eff > best + 0.01) {
            best = eff;
            S = s;
        }
    }
    const int tps = (int)((ntiles + S - 1) / S);
    dim3 grid((unsigned)sp.M, (unsigned)S);
    double *dst = S > 1 ? scratch : acc;
    k_moments<Real, MM, CM><<<grid, T, smem, stream>>>(
        static_cast<const Real *>(occ), occ_plane, ld_occ, static_cast<const TrajPar<Real> *>(par),
        nvals, count, (int)(e0 % (uint64_t)sp.n_sub), sp.n_sub, sp.M, K, L, tps, dst,
        S > 1 ? 0 : 1, err);
    GBS_LAUNCH_CHECK();
    if (nlaunch) *nlaunch = S > 1 ? 2 : 1;
    if (S > 1) {
        const int64_t total = (int64_t)sp.n_sub * sp.M * Q;
        const int g = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count * 8);
        k_moment_combine<<<g, 256, 0, stream>>>(scratch, S, total, acc);
        GBS_LAUNCH_CHECK();
    }
    return GBS_OK;
}

}  // namespace

size_t moment_par_bytes(bool fp64) { return fp64 ? sizeof(TrajPar<double>) : sizeof(TrajPar<float>); }

int moment_quantities(int mmax, int cmax) {
    const int MM = mmax <= 4 ? 4 : 8, CM = cmax <= 7 ? 7 : 15;
    return MM + MM / 2 + 2 * (CM + 1);
}

int moment_max_segments(int n_sub, int M, int mmax, int cmax) {
    // scratch of S [n_sub][M][Q] sums kept below 1 GiB
    const double per = (double)n_sub * M * moment_quantities(mmax, cmax) * sizeof(double);
    int s = kMaxSeg;
    while (s > 1 && per * s > (double)(1u << 30)) --s;
    return s;
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
                   int64_t ld_occ, const void *par, const double *nvals, int64_t count,
                   uint64_t e0, double *acc, double *scratch, int max_seg,
                   unsigned long long *err, cudaStream_t stream, int sm_count, int *nlaunch) {
    if (nlaunch) *nlaunch = 0;
    if (count <= 0) return GBS_OK;
    if (sp.M < 1 || sp.n_sub < 1) return set_error(GBS_EINVAL, "bad moment sizes");
    if (max_seg < 1 || (max_seg > 1 && !scratch)) max_seg = 1;
    const bool m8 = sp.mmax > 4, c15 = sp.cmax > 7;
#define GBS_MOM_CASE(R, A, B)                                                                    \
    return launch_t<R, A, B>(sp, occ, occ_plane, ld_occ, par, nvals, count, e0, acc, scratch,   \
                             max_seg, err, stream, sm_count, nlaunch)
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

int launch_moment_stats(const MomentSpec &sp, bool fp64, const double *acc, const int64_t *cnt,
                        double *out, cudaStream_t stream, int sm_count) {
    const int unscaled = fp64 ? 0 : 1;  // FP32 route sums leave out 1/c!
    const size_t nm = (size_t)2 * sp.M * sp.mmax, nc = (size_t)2 * sp.M * (sp.cmax + 1);
    double *mom = out, *smom = out + nm, *marg = out + 2 * nm, *smarg = out + 2 * nm + nc;
    const int64_t total = (int64_t)sp.M * (2 * sp.mmax + 2 * (sp.cmax + 1));
    const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count * 8);
    const bool m8 = sp.mmax > 4, c15 = sp.cmax > 7;
    if (!m8 && !c15)
        k_moment_stats<4, 7><<<grid, 256, 0, stream>>>(acc, cnt, sp.n_sub, sp.M, sp.mmax, sp.cmax, unscaled,
                                                       mom, smom, marg, smarg);
    else if (!m8)
        k_moment_stats<4, 15><<<grid, 256, 0, stream>>>(acc, cnt, sp.n_sub, sp.M, sp.mmax, sp.cmax, unscaled,
                                                        mom, smom, marg, smarg);
    else if (!c15)
        k_moment_stats<8, 7><<<grid, 256, 0, stream>>>(acc, cnt, sp.n_sub, sp.M, sp.mmax, sp.cmax, unscaled,
                                                       mom, smom, marg, smarg);
    else
        k_moment_stats<8, 15><<<grid, 256, 0, stream>>>(acc, cnt, sp.n_sub, sp.M, sp.mmax, sp.cmax, unscaled,
                                                        mom, smom, marg, smarg);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace gbs
