// Internal declarations of the GB300 matrix-P library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <string>
#include <vector>

#include "gbs.h"

namespace gbs {

// ---------------------------------------------------------------------------
// Error reporting (thread-local message, see gbs_last_error)
// ---------------------------------------------------------------------------
int set_error(int code, const char *fmt, ...);
const char *error_message();

#define GBS_CUDA_TRY(call)                                                             \
    do {                                                                               \
        cudaError_t err__ = (call);                                                    \
        if (err__ != cudaSuccess)                                                      \
            return ::gbs::set_error(GBS_ECUDA, "%s failed: %s (%s:%d)", #call,         \
                                    cudaGetErrorString(err__), __FILE__, __LINE__);    \
    } while (0)

#define GBS_LAUNCH_CHECK()                                                             \
    do {                                                                               \
        cudaError_t err__ = cudaGetLastError();                                        \
        if (err__ != cudaSuccess)                                                      \
            return ::gbs::set_error(GBS_ECUDA, "kernel launch failed: %s (%s:%d)",     \
                                    cudaGetErrorString(err__), __FILE__, __LINE__);    \
    } while (0)

// ---------------------------------------------------------------------------
// Constants
// ---------------------------------------------------------------------------
// Terms of a generating function whose log-magnitude is below -60 ln 2
// (|term| < 2^-60) are not evaluated by the FP64 kernels; the double-float
// kernel, whose own rounding of terms of order one is 2^-46, skips those
// below 2^-47 (each skipped term moves every P(m) by less than 2^-47 / K1).
constexpr double kSkipLog = 41.58883083359672;    // 60 * ln 2
constexpr double kSkipLogDf = 32.57791748631743;  // 47 * ln 2
constexpr int kFp64TileModes = 64;              // output modes per FP64 GEMM tile
constexpr int kFp64TileSamples = 32;            // samples per FP64 GEMM tile
constexpr int kTcTileModes = 64;                // output modes per tcgen05 tile (128 A rows)
constexpr int kTcTileSamples = 128;             // samples per tcgen05 tile (256 B rows)
constexpr int kTcBlockK = 64;                   // K elements per pipeline stage (128 B of bf16)

// Per-sample windows of the generating-function evaluation, in units of k:
// w1 = half-width around theta = 0 (both estimators' e^{(z-1) n_S} term),
// w2 = half-width around theta = pi (matrix-P's e^{-(z-1) n_S - 2n} term),
// -1 = empty, >= K1/2 = whole circle.
struct Window {
    int w1;
    int w2;
};

// Binned estimator (2..kMaxBins output bins): per dimension the half-width
// in k of the e^{L} term's window around 0 (w1) and of the e^{-L} term's
// window around pi (w2); -1 = empty.
constexpr int kMaxBins = 4;
struct WindowD {
    int w1[kMaxBins];
    int w2[kMaxBins];
};

// ---------------------------------------------------------------------------
// The network object behind gbs_net_t
// ---------------------------------------------------------------------------
struct TcPlan;  // tcgen05 GEMM plan (tensor maps, tiling), defined in k_gemm_tc.cu

// Operand description of one network for the (grouped) tcgen05 GEMM, kept in
// device memory so that one launch can serve many networks.
struct __align__(128) GemmNetDesc {
    CUtensorMap mapA[3];     // A planes [K/32][rows][32], box 32 x 128 x 1
    CUtensorMap mapB[2][3];  // B planes, box 32 x 256 x 1 (one CTA per tile) / 32 x 128 x 1 (CTA pairs)
    int KB;                  // 32-wide K blocks
    int mtiles;              // 64-mode tiles
    int stiles;              // 128-trajectory tiles (grouped launches)
    int pad;
    int64_t count;           // trajectories (grouped launches)
    int64_t ld_part;         // leading dimension of nS_part
    double2 *nS_part;        // [mtiles][ld_part] per-tile n_S partials
    unsigned int *wave_sync; // wave-alignment counter (single-network launches), or null
};

// Optional per-mode occupation output of the propagation GEMMs: n'_i of
// trajectory s at p[i * ld + s] (real parts) and p[plane + i * ld + s]
// (imaginary parts), i < mtiles * 64 (the padding modes of the last tile
// included), s < ld.  p == nullptr: not written.
struct OccOut {
    float *p = nullptr;
    int64_t ld = 0;
    int64_t plane = 0;
};
struct OccOut64 {
    double *p = nullptr;
    int64_t ld = 0;
    int64_t plane = 0;
};

// One chunk's work for the BF16 sampler (sampler_dev.cuh): trajectories
// e0 .. e0 + count - 1 into the sample operand at B (planesB planes of
// plane_stride elements, rows rows each, K-blocked with ldK) and n_out[count].
// count == 0: nothing to sample.
struct SampleJob {
    const float2 *sq = nullptr;  // [N] (sqrt(s+/2), sqrt(s-/2))
    __nv_bfloat16 *B = nullptr;
    double *n_out = nullptr;
    size_t plane_stride = 0, rows = 0;
    uint64_t seed = 0, e0 = 0;
    int64_t count = 0;
    int N = 0, ldK = 0, planesB = 0;
};

// The sampler work of a sampling GEMM: one job (n == 0: `one`), or n jobs in
// device memory whose trajectories are taken as one list (job j owns list
// positions prefix[j] .. prefix[j + 1] - 1).
struct SampleJobs {
    const SampleJob *jobs = nullptr;
    const int64_t *prefix = nullptr;  // [n + 1]
    int n = 0;
    SampleJob one;
};

// CUDA-event timing of kernel phases (gbs_profile_*).
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<cudaEvent_t> marks[GBS_NPHASES];  // start, stop, start, stop, ...
    int64_t launches[GBS_NPHASES] = {};
};

// The SIMT precisions (GBS_FP64, GBS_FP32) share the FP64 sampler, network
// operand, generating functions and inversion; only the GEMM's arithmetic
// differs.  The BF16 split precisions run the tcgen05 path.
inline bool simt_precision(int precision) {
    return precision == GBS_FP64 || precision == GBS_FP32;
}

}  // namespace gbs

struct gbs_net {
    int N = 0, M = 0, precision = 0;
    cudaStream_t stream = nullptr;
    int device = 0, sm_count = 0;

    // per-mode sampler coefficients: (sqrt(s+/2), sqrt(s-/2)), s+- = sinh r e^{+-r}
    double2 *d_sq64 = nullptr;
    float2 *d_sq32 = nullptr;

    // FP64 network operand: [M][2][N], row (i,0) = Re T_i., (i,1) = Im T_i.
    double *d_T64 = nullptr;

    // BF16 split operands (GBS_BF16X3 / X6): planes of A = [Re T; Im T] rows
    // interleaved per mode, K-blocked: [planes][ldK / 32][rowsA][32] bf16,
    // ldK = N rounded up to a multiple of 32 (the sample operand likewise)
    __nv_bfloat16 *d_A = nullptr;
    int planesA = 0, planesB = 0, rowsA = 0, ldK = 0;
    gbs::TcPlan *tc = nullptr;

    // chunk workspace
    int64_t chunk = 0;
    void *d_B = nullptr;  // sample operand
    size_t B_bytes = 0;
    double *d_n = nullptr;          // [chunk]
    // second sample operand and n[] (BF16X3): the GEMM of one chunk fills
    // them with the next chunk's samples; swapped with d_B, d_n per chunk
    void *d_B_alt = nullptr;
    double *d_n_alt = nullptr;
    int fuse_sampler = 1;           // gbs_set_sampler_fusion: 0 off, 1 automatic, 2 always
    // samples drawn ahead by the last GEMM of a folded gbs_sample into the
    // second operand: trajectories pre_e0 .. pre_e0 + pre_count - 1 of seed
    // pre_seed (valid until anything else samples into this network)
    bool pre_valid = false;
    uint64_t pre_seed = 0, pre_e0 = 0;
    int64_t pre_count = 0;
    void *pre_buf = nullptr;        // the operand (d_B or d_B_alt) holding them
    // the last gbs_sample call's seed and first + E: a call that continues it
    // (same seed, first = that end) draws ahead for the call after it
    bool have_last = false;
    uint64_t last_seed = 0, last_end = 0;
    double2 *d_nS_part = nullptr;   // [mtiles][chunk]
    int mtiles = 0;
    double2 *d_nS = nullptr;        // [chunk]
    gbs::Window *d_win = nullptr;   // [chunk]
    void *d_gfrec = nullptr;        // [chunk] generating-function records (BF16 paths)
    int *d_wmax = nullptr;          // [2]: union of the chunk's windows (max w1, max w2)

    // estimator state
    int n_sub = 0, K1 = 0;
    bool est_fixed = false;
    double2 *d_acc = nullptr;       // [2][n_sub][K1]
    int64_t *d_counts = nullptr;    // [n_sub]
    std::vector<int64_t> counts;    // host mirror, updated per call
    double2 *d_tw = nullptr;        // [K1]: (cos theta_k - 1, sin theta_k)
    double2 *d_fft0 = nullptr, *d_fft1 = nullptr;  // [2][n_sub][K1]
    double2 *d_wfft = nullptr;      // [K1]: e^{-2 pi i k / K1}
    double *d_out = nullptr;        // [4][K1]
    unsigned long long *d_flags = nullptr;  // [4]: non-finite count, timeout flag, ...
    // bound of every pipeline wait in this network's GEMM launches
    // (gbs_set_wait_limit; the default gives up after 2 s)
    uint64_t wait_ns = 2000000000ull;

    gbs::Profiler prof;

    // Output bins (gbs_make_network_binned, 2..kMaxBins): the output modes
    // of each bin are stored as consecutive rows, each bin padded with zero
    // rows to whole 64-mode tiles; bin b is tiles [bin_tiles[b], bin_tiles[b+1]).
    int nbins = 1;
    int bin_tiles[gbs::kMaxBins + 1] = {};
    int M_user = 0;  // output modes as given (M includes the padding rows)
    // binned estimator state (gbs_sample_nd)
    double2 *d_nS2 = nullptr;       // [chunk][nbins]: n_Sb
    gbs::WindowD *d_win2 = nullptr; // [chunk]
    int *d_wmax2 = nullptr;         // [2 kMaxBins]: union of the chunk's windows (w1, then w2)
    bool est2_fixed = false;
    int n_sub2 = 0;
    int Kd[gbs::kMaxBins] = {};     // points per dimension
    int64_t grid2 = 0;              // prod Kd
    double2 *d_acc2 = nullptr;      // [2][n_sub2][grid2]
    int64_t *d_counts2 = nullptr;   // [n_sub2]
    std::vector<int64_t> counts2;
    double2 *d_tw2 = nullptr;       // [sum Kd]: (cos theta - 1, sin theta) of each dimension
    double2 *d_wf2 = nullptr;       // [sum Kd]: e^{-i theta}
    double2 *d_f2a = nullptr, *d_f2b = nullptr;  // [2][n_sub2][grid2] FFT work
    double *d_out2 = nullptr;       // [4][grid2]
    int64_t *d_mo2 = nullptr;       // [kMaxBins] DFT window offsets
    void *d_sep2 = nullptr;         // [chunk] per-trajectory constants (BF16 networks)
};

namespace gbs {

// ---------------------------------------------------------------------------
// Kernel launchers (each returns a GBS status)
// ---------------------------------------------------------------------------
// Stream-ordered device memory from the default pool (kept between
// networks); freed with pool_free_raw on the same stream.
int pool_alloc(void **p, size_t bytes, cudaStream_t stream, const char *what);
void pool_free_raw(void *p, cudaStream_t stream);

// Sampler: writes the sample operand for trajectories e0..e0+count-1 and n[].
int launch_sample_fp64(gbs_net *net, uint64_t seed, uint64_t e0, int64_t count);
int launch_sample_bf16(gbs_net *net, uint64_t seed, uint64_t e0, int64_t count);
// The BF16 sampler's job for trajectories e0..e0+count-1 into (B, n).
SampleJob sample_job_bf16(gbs_net *net, void *B, double *n, uint64_t seed, uint64_t e0,
                          int64_t count);

// Propagation GEMM with the fused occupation epilogue -> nS_part[mtiles][chunk].
int launch_gemm_fp64(gbs_net *net, int64_t count, OccOut64 occ = OccOut64());
int tc_plan_create(gbs_net *net);
void tc_plan_destroy(gbs_net *net);
int launch_gemm_tc(gbs_net *net, int64_t count, OccOut occ = OccOut());
// 3-product GEMM of the chunk in (d_B, d_n) whose spare warps run `job`
// (the next chunk, into d_B_alt, d_n_alt); needs tc_sampling_ready().
int launch_gemm_tc_sampling(gbs_net *net, int64_t count, const SampleJob &job,
                            OccOut occ = OccOut());
// Trajectories per chunk of a gbs_sample call (and of a batch round) over E
// trajectories: the fewest chunks of at most net->chunk (a multiple of the
// tile), the even split rounded up to whole 128-trajectory tiles, so that
// no chunk but the last ends in a partly filled trajectory tile.
inline int64_t chunk_step(const gbs_net *net, int64_t E) {
    if (E <= net->chunk) return E > 0 ? E : net->chunk;
    const int64_t nch = (E + net->chunk - 1) / net->chunk;
    const int64_t even = (E + nch - 1) / nch;
    const int64_t tiled = (even + kTcTileSamples - 1) / kTcTileSamples * kTcTileSamples;
    return tiled < net->chunk ? tiled : net->chunk;
}

// Output modes from which a network's sampling pays off inside its GEMM:
// the 6 sampler warps per SM draw a chunk of N-mode trajectories in about
// 1.6 ms x N / 1000 while the GEMM takes about 1.8 ms x N M / 10^6 (both
// measured at N = M = 1000, 131072 trajectories), so below M ~ 860 the
// sampler would become the launch's tail.
constexpr int kFoldMinModes = 900;
// gbs_set_sampler_fusion's setting: 0 never, 1 from kFoldMinModes output
// modes, 2 whenever the network can.
inline bool fold_wanted(const gbs_net *net) {
    return net->fuse_sampler == 2 || (net->fuse_sampler == 1 && net->M >= kFoldMinModes);
}
// Whether this network can run the sampling GEMM: 3 products, the kernel's
// register split verified, the second operand allocated (allocates it when
// `allocate`).
bool tc_sampling_ready(gbs_net *net, bool allocate);
// Swap (d_B, d_n, tensor maps) with their second copies.
void tc_swap_sample_buffers(gbs_net *net);
// GEMM configuration: pair = 1 (one CTA per tile) or 2 (CTA pairs,
// cta_group::2), band = mode-tile groups per band of the tile order (0: plain
// order), keep = 1: a band's A tiles loaded with the evict-last L2 policy;
// pair 0 returns to the autotuner.
struct GemmCfg {
    int pair = 0;
    int band = 0;
    int keep = 0;
};
int tc_set_config(gbs_net *net, const GemmCfg &cfg);
GemmCfg tc_get_config(gbs_net *net);
// Whether the autotuner also times CTA pairs (process-wide; clears its cache).
void tc_set_pair_autotune(bool on);
bool tc_pair_autotune();

int tc_products(gbs_net *net);
int tc_fill_desc(gbs_net *net, GemmNetDesc *out, bool alt = false);  // alt: the second operand's maps
// One launch over the tiles of many networks (d_tiles: {net, mode-tile group,
// trajectory tile} per entry; NULL = closed-form tiles of d_nets[0] with
// count0 trajectories in bands of `band` groups); wait_ns bounds every
// pipeline wait of the kernel.  shallow = 1 runs the operand ring one stage
// shallower than the deepest that fits (a batch autotuner candidate; the
// results are bitwise the same).
int launch_gemm_grouped(cudaStream_t stream, int sm_count, int P, int pair, int band, int keep_a,
                        uint64_t wait_ns, const GemmNetDesc *d_nets, const int4 *d_tiles,
                        int ntiles, int64_t count0, unsigned long long *err,
                        OccOut occ = OccOut(), int shallow = 0);
// The same launch (3 products, listed tiles) whose spare warps run `jobs`.
int launch_gemm_grouped_sampling(cudaStream_t stream, int sm_count, int pair, uint64_t wait_ns,
                                 const GemmNetDesc *d_nets, const int4 *d_tiles, int ntiles,
                                 unsigned long long *err, const SampleJobs &jobs,
                                 int shallow = 0);
// Stages of the GEMM's operand ring for (products, pair, shallow).
int tc_ring_stages(int P, int pair, int shallow);
// Whether the sampling GEMM variants with the shallower ring can run.
bool tc_shallow_sampling_ok();

// Finalise n_S (fixed-order sum of tile partials) and the evaluation windows.
int launch_finalize(gbs_net *net, int64_t count);

// Generating functions, summed per sub-ensemble into d_acc.
int launch_gf(gbs_net *net, uint64_t e0, int64_t count);
// Bytes per trajectory of the records the finalize kernel writes for the
// double-float generating functions (d_gfrec).
size_t gf_record_bytes();

// Twiddle tables for K1 points.
int launch_tables(gbs_net *net);

// Inverse DFT + statistics into out_dev[4][K1].
int launch_invert(gbs_net *net, int64_t m_offset, double *out_dev);

// Non-finite count of the accumulators into d_flags[0].
int launch_count_nonfinite(gbs_net *net);

// Forward DFTs of length K (a power of two) over `batch` contiguous rows of
// x (radix-2 Stockham passes alternating between x and y); *result is the
// buffer holding the output.
int launch_fft_rows(const double2 *wfft, int K, int64_t batch, double2 *x, double2 *y,
                    double2 **result, cudaStream_t stream, int sm_count);

// Histograms of per-trajectory projectors (k_hist.cu, Appendix A).
constexpr int kHistMaxM = 16;
constexpr int kHistMaxBins = 4096;
struct HistSpec {
    int m[kHistMaxM];
    int nm;
    int nbins;
    double lo, hi;
};
// Adds the chunk's trajectories (d_n, d_nS) to out_dev[2][nm][nbins + 2]
// (matrix-P first; bin 0 = below lo, nbins + 1 = at or above hi).
int launch_histogram(gbs_net *net, int64_t count, const HistSpec &spec,
                     unsigned long long *out_dev);

// Moments and single-mode marginals (k_moments.cu).
struct MomentSpec {
    int M, n_sub, mmax, cmax;
};
// Bytes per trajectory of the per-trajectory parameters; quantities summed
// per (sub-ensemble, mode) for (mmax, cmax).
size_t moment_par_bytes(bool fp64);
int moment_quantities(int mmax, int cmax);
// Per-trajectory parameters (tanh n, sign n, logs) of the chunk from n[].
int launch_moment_prep(const double *n, int64_t count, bool fp64, void *par, cudaStream_t stream,
                       int sm_count);
// Segments of a chunk whose scratch sums (max_seg [n_sub][M][Q] doubles) stay
// below 1 GiB.
int moment_max_segments(int n_sub, int M, int mmax, int cmax);
// Adds the chunk's trajectories (first global index e0; n[] their input
// totals) to acc[n_sub][M][Q], through scratch[max_seg][n_sub][M][Q] when
// the chunk is cut into segments; a bounded wait that gives up raises *err;
// *nlaunch = kernels launched.
int launch_moments(const MomentSpec &sp, bool fp64, const void *occ, int64_t occ_plane,
                   int64_t ld_occ, const void *par, const double *n, int64_t count, uint64_t e0,
                   double *acc, double *scratch, int max_seg, unsigned long long *err,
                   cudaStream_t stream, int sm_count, int *nlaunch);
// Means and errors over sub-ensembles into out = [mom, sig_mom, marg, sig_marg]
// (the sums of BF16 networks hold the marginals without their 1/c!).
int launch_moment_stats(const MomentSpec &sp, bool fp64, const double *acc, const int64_t *cnt,
                        double *out, cudaStream_t stream, int sm_count);

// Binned estimator (k_bin2d.cu): finalize (per-bin n_S and windows),
// generating functions on the K_1 x .. x K_d grid, and the d-dimensional
// inversion into out_dev[4][grid2] (*launches: kernels launched).
int launch_finalize2d(gbs_net *net, int64_t count);
int launch_gf2d(gbs_net *net, uint64_t e0, int64_t count);
size_t sep2_bytes_per_trajectory();
int launch_tables2d(gbs_net *net);
int launch_invert2d(gbs_net *net, const int64_t *m_off, double *out_dev, int *launches);

// Fix (or check) a network's estimator shape, allocating its sums on first use.
int fix_estimator(gbs_net *net, int n_sub, int K1);
// Host mirror of the sub-ensemble sizes after trajectories first..first+E-1.
void count_samples(gbs_net *net, uint64_t first, int64_t E);

// Phase timing: bracket the launches of one phase (no-ops when disabled).
void prof_mark(gbs_net *net, int phase, int launches_if_stop, bool start);

// Tensor map of a row-major BF16 array (rows x inner elements, row pitch
// row_bytes) read in boxes of box_inner x box_rows with the 64-byte swizzle
// (box_inner = 32 elements = one 64-byte row).  Out-of-range box rows read as
// zeros.
int encode_2d(CUtensorMap *map, void *base, uint64_t inner, uint64_t rows, uint64_t row_bytes,
              uint32_t box_inner, uint32_t box_rows);

// Device properties helper.
bool device_has_tcgen05(int device);

}  // namespace gbs
