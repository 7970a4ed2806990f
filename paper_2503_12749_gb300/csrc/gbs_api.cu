// C ABI of the GB300 matrix-P library (declared in include/gbs.h).
//
// Orchestration of the ensemble loop of the matrix phase-space method for
// Gaussian boson sampling: per chunk of trajectories
//   K1 sampler -> K2/K3 propagation GEMM + occupation epilogue -> finalize
//   -> K4 generating functions summed per sub-ensemble,
// and on request K5 (inverse DFT + statistics).  Every device buffer is
// owned by the network object; all work runs on the network's stream.
#include "gbs_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

namespace gbs {

static thread_local char g_err[1024] = "";

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

const char *error_message() { return g_err; }

bool device_has_tcgen05(int device) {
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess)
        return false;
    if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess)
        return false;
    return major == 10 && minor == 3;  // this library is built for sm_103a only
}

void prof_mark(gbs_net *net, int phase, int launches_if_stop, bool start) {
    Profiler &pr = net->prof;
    if (!pr.on) return;
    cudaEvent_t ev;
    if (!pr.pool.empty()) {
        ev = pr.pool.back();
        pr.pool.pop_back();
    } else if (cudaEventCreate(&ev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(ev, net->stream);
    pr.marks[phase].push_back(ev);
    if (!start) pr.launches[phase] += launches_if_stop;
}

// Stream-ordered allocations from the device's default memory pool, for
// every buffer a network owns (the chunk workspace alone is about 1 GiB at
// N = 1000): the pool keeps the memory when a network is freed (release
// threshold raised once per device for this process), so creating and
// freeing networks in a loop neither goes back to the driver for every
// network nor synchronises the device as cudaFree does.  Allocated and freed
// on the network's stream; plain cudaMalloc / cudaFree on a device without
// memory pools.
namespace {
// per device: 0 not yet known, -1 plain cudaMalloc (no memory pools), 1 pool
int g_pool_state[64] = {};
std::mutex g_pool_mu;

bool pool_supported() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (g_pool_state[dev] == 0) {
        int ok = 0;
        cudaMemPool_t pool;
        if (cudaDeviceGetAttribute(&ok, cudaDevAttrMemoryPoolsSupported, dev) == cudaSuccess && ok &&
            cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            g_pool_state[dev] = 1;
        } else {
            g_pool_state[dev] = -1;
        }
        cudaGetLastError();
    }
    return g_pool_state[dev] == 1;
}
}  // namespace

int pool_alloc(void **p, size_t bytes, cudaStream_t stream, const char *what) {
    *p = nullptr;
    if (bytes == 0) return GBS_OK;
    // without stream-ordered pools on this device: plain allocations
    const bool pool = pool_supported();
    const cudaError_t err = pool ? cudaMallocAsync(p, bytes, stream) : cudaMalloc(p, bytes);
    if (err != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(err == cudaErrorMemoryAllocation ? GBS_ENOMEM : GBS_ECUDA,
                         "%s(%s, %zu bytes) failed: %s", pool ? "cudaMallocAsync" : "cudaMalloc",
                         what, bytes, cudaGetErrorString(err));
    }
    return GBS_OK;
}

void pool_free_raw(void *p, cudaStream_t stream) {
    if (!p) return;
    if (pool_supported())
        cudaFreeAsync(p, stream);
    else
        cudaFree(p);
}

namespace {

void prof_clear(gbs_net *net) {
    Profiler &pr = net->prof;
    for (int ph = 0; ph < GBS_NPHASES; ++ph) {
        for (cudaEvent_t e : pr.marks[ph]) pr.pool.push_back(e);
        pr.marks[ph].clear();
        pr.launches[ph] = 0;
    }
}

void prof_destroy(gbs_net *net) {
    prof_clear(net);
    for (cudaEvent_t e : net->prof.pool) cudaEventDestroy(e);
    net->prof.pool.clear();
}

template <typename T>
int pool_alloc_n(T **p, size_t count, cudaStream_t stream, const char *what) {
    return pool_alloc(reinterpret_cast<void **>(p), count * sizeof(T), stream, what);
}

template <typename T>
void pool_free(T *&p, cudaStream_t stream) {
    pool_free_raw(p, stream);
    p = nullptr;
}

// A network's own buffers, stream-ordered on its stream (used there, or on
// streams forked from it after the allocation).
template <typename T>
int net_alloc(gbs_net *net, T **p, size_t count, const char *what) {
    return pool_alloc_n(p, count, net->stream, what);
}
template <typename T>
void net_free(gbs_net *net, T *&p) {
    pool_free(p, net->stream);
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int64_t pick_chunk(const gbs_net *net) {
    // trajectories per chunk: sample operand <= 1 GiB, multiple of 128, in [128, 2^17]
    size_t per_traj;
    if (simt_precision(net->precision))
        per_traj = (size_t)16 * net->N;
    else
        per_traj = (size_t)4 * net->planesB * net->ldK;
    int64_t c = (int64_t)((size_t)1 << 30) / (int64_t)per_traj;
    c = std::min<int64_t>(c, (int64_t)1 << 17);
    c = (c / 128) * 128;
    return std::max<int64_t>(c, 128);
}

void release_estimator(gbs_net *net) {
    net_free(net, net->d_acc);
    net_free(net, net->d_counts);
    net_free(net, net->d_tw);
    net_free(net, net->d_wfft);
    net_free(net, net->d_fft0);
    net_free(net, net->d_fft1);
    net_free(net, net->d_out);
    net->counts.clear();
    net->est_fixed = false;
    net->n_sub = 0;
    net->K1 = 0;
    net_free(net, net->d_acc2);
    net_free(net, net->d_counts2);
    net_free(net, net->d_tw2);
    net_free(net, net->d_wf2);
    net_free(net, net->d_f2a);
    net_free(net, net->d_f2b);
    net_free(net, net->d_out2);
    net_free(net, net->d_mo2);
    pool_free(net->d_sep2, net->stream);
    net->counts2.clear();
    net->est2_fixed = false;
    net->n_sub2 = 0;
    net->grid2 = 0;
    for (int b = 0; b < kMaxBins; ++b) net->Kd[b] = 0;
}

void release_all(gbs_net *net) {
    release_estimator(net);
    prof_destroy(net);
    if (net->tc) tc_plan_destroy(net);
    net_free(net, net->d_sq64);
    net_free(net, net->d_sq32);
    net_free(net, net->d_T64);
    net_free(net, net->d_A);
    pool_free(net->d_B, net->stream);
    pool_free(net->d_B_alt, net->stream);
    pool_free(net->d_n_alt, net->stream);
    pool_free(net->d_n, net->stream);
    pool_free(net->d_nS_part, net->stream);
    pool_free(net->d_nS, net->stream);
    pool_free(net->d_win, net->stream);
    pool_free(net->d_gfrec, net->stream);
    net_free(net, net->d_wmax);
    net_free(net, net->d_flags);
    net_free(net, net->d_nS2);
    net_free(net, net->d_win2);
    net_free(net, net->d_wmax2);
}

// Sampler + propagation + finalize for one chunk of `count` trajectories.
int run_chunk_front(gbs_net *net, uint64_t seed, uint64_t e0, int64_t count) {
    int rc;
    const bool fp64 = simt_precision(net->precision);
    prof_mark(net, GBS_PHASE_SAMPLE, 0, true);
    rc = fp64 ? launch_sample_fp64(net, seed, e0, count) : launch_sample_bf16(net, seed, e0, count);
    if (rc) return rc;
    prof_mark(net, GBS_PHASE_SAMPLE, 1, false);
    prof_mark(net, GBS_PHASE_GEMM, 0, true);
    rc = fp64 ? launch_gemm_fp64(net, count) : launch_gemm_tc(net, count);
    if (rc) return rc;
    prof_mark(net, GBS_PHASE_GEMM, 1, false);
    prof_mark(net, GBS_PHASE_FINALIZE, 0, true);
    if ((rc = launch_finalize(net, count))) return rc;
    prof_mark(net, GBS_PHASE_FINALIZE, 1, false);
    return GBS_OK;
}

// A chunk loop with the sampler folded into the GEMM (BF16X3): the first
// chunk is sampled alone; the GEMM of chunk i also samples chunk i + 1 into
// the second operand (gemm(count, job); job.count == 0 for the last chunk),
// after(e0, count) launches what consumes chunk i, and the two operands swap
// roles after every chunk (back to their original roles at the end, so that
// the other entry points always find the first operand current).  The
// samples, and so every sum, are bitwise those of the plain chunk loop.
//
// With `ahead` (gbs_sample, chunks of chunk_step): the last chunk's GEMM also
// draws the chunk a following call on the same seed from first + E would
// start with (into the second operand, recorded in net->pre_*), and a
// call that finds its own first chunk drawn that way starts from it instead
// of sampling it again.
template <typename Gemm, typename After>
int pipelined_chunks(gbs_net *net, uint64_t seed, uint64_t first, int64_t E, int64_t step,
                     Gemm gemm, After after, bool ahead = false) {
    int rc = GBS_OK, swaps = 0;
    if (ahead) {
        // not inside a stream capture: the host's record of what was drawn
        // ahead would not follow the graph's launches
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(net->stream, &cs) != cudaSuccess ||
            cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            ahead = false;
            net->pre_valid = false;
        }
    }
    const int64_t c0 = std::min<int64_t>(step, E);
    const bool reuse = ahead && net->pre_valid && net->pre_seed == seed && net->pre_e0 == first &&
                       net->pre_count >= c0 &&
                       (net->pre_buf == net->d_B || net->pre_buf == net->d_B_alt);
    if (reuse) {
        if (net->pre_buf == net->d_B_alt) {  // the drawn-ahead chunk becomes current
            tc_swap_sample_buffers(net);
            ++swaps;
        }
    } else {
        prof_mark(net, GBS_PHASE_SAMPLE, 0, true);
        rc = launch_sample_bf16(net, seed, first, c0);
        prof_mark(net, GBS_PHASE_SAMPLE, 1, false);
    }
    net->pre_valid = false;
    for (int64_t done = 0; rc == GBS_OK && done < E; done += step) {
        const int64_t c = std::min<int64_t>(step, E - done);
        const uint64_t e0 = first + (uint64_t)done;
        const int64_t next = std::min<int64_t>(step, E - done - c);
        SampleJob job;
        if (next > 0) {
            job = sample_job_bf16(net, net->d_B_alt, net->d_n_alt, seed, e0 + (uint64_t)c, next);
        } else if (ahead) {
            // the last chunk: draw the next call's first chunk
            job = sample_job_bf16(net, net->d_B_alt, net->d_n_alt, seed, e0 + (uint64_t)c, step);
        }
        prof_mark(net, GBS_PHASE_GEMM, 0, true);
        if ((rc = gemm(c, job))) break;
        prof_mark(net, GBS_PHASE_GEMM, 1, false);
        if ((rc = after(e0, c))) break;
        void *drawn_into = net->d_B_alt;
        tc_swap_sample_buffers(net);
        ++swaps;
        if (next == 0 && ahead) {
            net->pre_valid = true;
            net->pre_seed = seed;
            net->pre_e0 = e0 + (uint64_t)c;
            net->pre_count = step;
            net->pre_buf = drawn_into;
        }
    }
    if (swaps & 1) tc_swap_sample_buffers(net);
    if (rc) net->pre_valid = false;
    return rc;
}

// Whether a chunk loop of E trajectories in steps of `step` folds the sampler.
bool fold_sampler(gbs_net *net, int64_t E, int64_t step) {
    return E > step && net->precision == GBS_BF16X3 && fold_wanted(net) &&
           tc_sampling_ready(net, true);
}

int sample_chunks_pipelined(gbs_net *net, uint64_t seed, uint64_t first, int64_t E) {
    auto gemm = [&](int64_t c, const SampleJob &job) {
        return job.count ? launch_gemm_tc_sampling(net, c, job) : launch_gemm_tc(net, c);
    };
    auto after = [&](uint64_t e0, int64_t c) {
        int rc;
        prof_mark(net, GBS_PHASE_FINALIZE, 0, true);
        if ((rc = launch_finalize(net, c))) return rc;
        prof_mark(net, GBS_PHASE_FINALIZE, 1, false);
        prof_mark(net, GBS_PHASE_GF, 0, true);
        if ((rc = launch_gf(net, e0, c))) return rc;
        prof_mark(net, GBS_PHASE_GF, 1, false);
        return GBS_OK;
    };
    // draw ahead only within a stream of consecutive calls: this call
    // continues the previous one, so the next probably continues this one
    const bool ahead = net->have_last && net->last_seed == seed && net->last_end == first;
    return pipelined_chunks(net, seed, first, E, chunk_step(net, E), gemm, after, ahead);
}

// T (device, M x N complex, (re, im) interleaved, row-major) -> [M][2][N] FP64.
__global__ void k_t64_from_dev(const double *__restrict__ T, int N, int M, double *__restrict__ out,
                               unsigned long long *nonfinite) {
    const int64_t total = (int64_t)M * N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / N, j = q % N;
        const double re = T[2 * q], im = T[2 * q + 1];
        if (!isfinite(re) || !isfinite(im)) atomicAdd(nonfinite, 1ull);
        out[(i * 2 + 0) * N + j] = re;
        out[(i * 2 + 1) * N + j] = im;
    }
}

// T (device) -> BF16 planes of A = [Re T_i.; Im T_i.] (rows interleaved per
// mode, K-blocked: element (row, j) at ((j / 32) * rows + row) * 32 + j % 32),
// T rounded to FP32 and split T = T0 + T1 + T2.
__global__ void k_split_from_dev(const double *__restrict__ T, int N, int M, int rows,
                                 __nv_bfloat16 *__restrict__ A, size_t plane,
                                 unsigned long long *nonfinite) {
    const int64_t total = (int64_t)M * N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / N, j = q % N;
        for (int c = 0; c < 2; ++c) {
            const double v = T[2 * q + c];
            if (!isfinite(v)) atomicAdd(nonfinite, 1ull);
            const float x = __double2float_rn(v);
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
            const float r1 = x - __bfloat162float(h0);
            const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
            const float r2 = r1 - __bfloat162float(h1);
            const size_t o = ((size_t)(j >> 5) * rows + (size_t)(2 * i + c)) * 32 + (j & 31);
            A[o] = h0;
            A[plane + o] = h1;
            A[2 * plane + o] = __float2bfloat16_rn(r2);
        }
    }
}

// Sampler + propagation + two-bin finalize for one chunk.
int run_chunk_front2d(gbs_net *net, uint64_t seed, uint64_t e0, int64_t count) {
    int rc;
    const bool fp64 = simt_precision(net->precision);
    prof_mark(net, GBS_PHASE_SAMPLE, 0, true);
    rc = fp64 ? launch_sample_fp64(net, seed, e0, count) : launch_sample_bf16(net, seed, e0, count);
    if (rc) return rc;
    prof_mark(net, GBS_PHASE_SAMPLE, 1, false);
    prof_mark(net, GBS_PHASE_GEMM, 0, true);
    rc = fp64 ? launch_gemm_fp64(net, count) : launch_gemm_tc(net, count);
    if (rc) return rc;
    prof_mark(net, GBS_PHASE_GEMM, 1, false);
    prof_mark(net, GBS_PHASE_FINALIZE, 0, true);
    if ((rc = launch_finalize2d(net, count))) return rc;
    prof_mark(net, GBS_PHASE_FINALIZE, 1, false);
    return GBS_OK;
}

int fix_estimator2d(gbs_net *net, int n_sub, const int *K) {
    const int d = net->nbins;
    if (net->est2_fixed) {
        bool same = n_sub == net->n_sub2;
        for (int b = 0; b < d; ++b) same = same && K[b] == net->Kd[b];
        if (!same)
            return set_error(GBS_EINVAL,
                             "n_sub and the grid differ from the values fixed by the first call "
                             "(n_sub %d); call gbs_reset first",
                             net->n_sub2);
        return GBS_OK;
    }
    if (n_sub < 1 || n_sub > 65535) return set_error(GBS_EINVAL, "n_sub must be in [1, 65535]");
    int64_t grid = 1;
    int tot = 0;
    for (int b = 0; b < d; ++b) {
        if (!is_pow2(K[b]) || K[b] < 2 || K[b] > (1 << 20))
            return set_error(GBS_EINVAL, "K[%d] = %d: grid sizes must be powers of two >= 2", b, K[b]);
        grid *= K[b];
        tot += K[b];
        if (grid > (1 << 22)) return set_error(GBS_EINVAL, "the grid must have at most 2^22 points");
    }
    net->n_sub2 = n_sub;
    for (int b = 0; b < kMaxBins; ++b) net->Kd[b] = b < d ? K[b] : 0;
    net->grid2 = grid;
    const size_t accn = (size_t)2 * n_sub * grid;
    int rc;
    if ((rc = net_alloc(net, &net->d_acc2, accn, "acc2")) ||
        (rc = net_alloc(net, &net->d_counts2, (size_t)n_sub, "counts2")) ||
        (rc = net_alloc(net, &net->d_tw2, (size_t)tot, "tw2")) ||
        (rc = net_alloc(net, &net->d_wf2, (size_t)tot, "wf2")) ||
        (rc = net_alloc(net, &net->d_f2a, accn, "fft2a")) ||
        (rc = net_alloc(net, &net->d_f2b, accn, "fft2b")) ||
        (rc = net_alloc(net, &net->d_out2, (size_t)4 * grid, "out2")) ||
        (rc = net_alloc(net, &net->d_mo2, (size_t)kMaxBins, "window offsets")))
        return rc;
    if (!simt_precision(net->precision)) {
        if ((rc = pool_alloc(&net->d_sep2, (size_t)net->chunk * sep2_bytes_per_trajectory(),
                             net->stream, "sep2")))
            return rc;
    }
    GBS_CUDA_TRY(cudaMemsetAsync(net->d_acc2, 0, accn * sizeof(double2), net->stream));
    GBS_CUDA_TRY(cudaMemsetAsync(net->d_counts2, 0, (size_t)n_sub * sizeof(int64_t), net->stream));
    if ((rc = launch_tables2d(net))) return rc;
    net->counts2.assign((size_t)n_sub, 0);
    net->est2_fixed = true;
    return GBS_OK;
}

int validate_net(gbs_net *net) {
    if (!net) return set_error(GBS_EINVAL, "null network");
    return GBS_OK;
}

}  // namespace

int fix_estimator(gbs_net *net, int n_sub, int K1) {
    if (net->est_fixed) {
        if (n_sub != net->n_sub || K1 != net->K1)
            return set_error(GBS_EINVAL,
                             "n_sub/K1 (%d, %d) differ from the values fixed by the first call "
                             "(%d, %d); call gbs_reset first",
                             n_sub, K1, net->n_sub, net->K1);
        return GBS_OK;
    }
    if (n_sub < 1 || n_sub > 65535) return set_error(GBS_EINVAL, "n_sub must be in [1, 65535]");
    if (!is_pow2(K1) || K1 < 2 || K1 > (1 << 20))
        return set_error(GBS_EINVAL, "K1 must be a power of two in [2, 2^20]");
    net->n_sub = n_sub;
    net->K1 = K1;
    const size_t accn = (size_t)2 * n_sub * K1;
    int rc;
    if ((rc = net_alloc(net, &net->d_acc, accn, "acc")) ||
        (rc = net_alloc(net, &net->d_counts, (size_t)n_sub, "counts")) ||
        (rc = net_alloc(net, &net->d_tw, (size_t)K1, "tw")) ||
        (rc = net_alloc(net, &net->d_wfft, (size_t)K1, "wfft")) ||
        (rc = net_alloc(net, &net->d_fft0, accn, "fft0")) ||
        (rc = net_alloc(net, &net->d_fft1, accn, "fft1")) ||
        (rc = net_alloc(net, &net->d_out, (size_t)4 * K1, "out"))) {
        release_estimator(net);
        return rc;
    }
    GBS_CUDA_TRY(cudaMemsetAsync(net->d_acc, 0, accn * sizeof(double2), net->stream));
    GBS_CUDA_TRY(cudaMemsetAsync(net->d_counts, 0, (size_t)n_sub * sizeof(int64_t), net->stream));
    if ((rc = launch_tables(net))) {
        release_estimator(net);
        return rc;
    }
    net->counts.assign((size_t)n_sub, 0);
    net->est_fixed = true;
    return GBS_OK;
}

void count_samples(gbs_net *net, uint64_t first_sample, int64_t E) {
    const uint64_t ns = (uint64_t)net->n_sub;
    const uint64_t full = (uint64_t)E / ns, rem = (uint64_t)E % ns;
    const uint64_t start = first_sample % ns;
    for (uint64_t q = 0; q < ns; ++q) net->counts[q] += (int64_t)full;
    for (uint64_t q = 0; q < rem; ++q) net->counts[(start + q) % ns] += 1;
}

}  // namespace gbs

using namespace gbs;

extern "C" {

const char *gbs_last_error(void) { return error_message(); }

}  // extern "C"

namespace gbs {
namespace {

// Counts the non-finite entries found by one of the T conversion kernels.
int finish_device_T(gbs_net *net, unsigned long long *d_bad) {
    GBS_LAUNCH_CHECK();
    unsigned long long bad = 0;
    GBS_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, net->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(net->stream));
    if (bad) return set_error(GBS_EINVAL, "T has %llu non-finite entries", bad);
    return GBS_OK;
}

// Shared by gbs_make_network (T in host memory) and gbs_make_network_device.
int make_network(int N, int M, const double *T, bool T_device, const double *r, int precision,
                 void *stream, gbs_net_t *out) {
    if (!out) return set_error(GBS_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 1 || M < 1 || N > 65536 || M > 65536)
        return set_error(GBS_EINVAL, "N and M must be in [1, 65536] (got %d, %d)", N, M);
    if (!T || !r) return set_error(GBS_EINVAL, "T and r must be non-NULL pointers");
    if (precision != GBS_FP64 && precision != GBS_FP32 && precision != GBS_BF16X3 &&
        precision != GBS_BF16X6)
        return set_error(GBS_EINVAL, "unknown precision %d", precision);
    for (int j = 0; j < N; ++j)
        if (!std::isfinite(r[j]) || r[j] < 0.0)
            return set_error(GBS_EINVAL, "r[%d] = %g: squeezing must be finite and >= 0", j, r[j]);
    if (!T_device) {
        // T in page-locked host memory that the device can address (both
        // ends of the array in such an allocation, at a consistent device
        // address): the conversion kernels read it there directly, one pass
        // over the host link, with no staging buffer.  The call synchronises
        // before it returns, so T is not read afterwards.
        const size_t count = (size_t)2 * M * N;
        cudaPointerAttributes a0{}, a1{};
        if (cudaPointerGetAttributes(&a0, T) == cudaSuccess &&
            cudaPointerGetAttributes(&a1, T + (count - 1)) == cudaSuccess &&
            a0.type == cudaMemoryTypeHost && a1.type == cudaMemoryTypeHost && a0.devicePointer &&
            a1.devicePointer &&
            static_cast<const double *>(a1.devicePointer) -
                    static_cast<const double *>(a0.devicePointer) ==
                (ptrdiff_t)(count - 1))
            return make_network(N, M, static_cast<const double *>(a0.devicePointer), true, r,
                                precision, stream, out);
        cudaGetLastError();  // pageable memory: not an error
        // other host memory: upload it as given and build the operand layout
        // (and check for non-finite entries) on the GPU, as for device T
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        double *tmp = nullptr;
        int rc0;
        if ((rc0 = pool_alloc_n(&tmp, (size_t)2 * M * N, st, "T upload"))) return rc0;
        if (cudaMemcpyAsync(tmp, T, sizeof(double) * 2 * (size_t)M * N, cudaMemcpyHostToDevice,
                            st) != cudaSuccess) {
            cudaGetLastError();
            pool_free(tmp, st);
            return set_error(GBS_ECUDA, "upload of T failed");
        }
        rc0 = make_network(N, M, tmp, true, r, precision, stream, out);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            if (!rc0) rc0 = set_error(GBS_ECUDA, "network set-up failed");
        }
        pool_free(tmp, st);
        return rc0;
    }

    gbs_net *net = new (std::nothrow) gbs_net();
    if (!net) return set_error(GBS_ENOMEM, "host allocation failed");
    net->N = N;
    net->M = M;
    net->precision = precision;
    net->stream = static_cast<cudaStream_t>(stream);
    int rc = GBS_OK;
    auto fail = [&](int code) {
        release_all(net);
        delete net;
        return code;
    };
    if (cudaGetDevice(&net->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&net->sm_count, cudaDevAttrMultiProcessorCount, net->device) !=
            cudaSuccess) {
        cudaGetLastError();
        return fail(set_error(GBS_ECUDA, "no usable CUDA device"));
    }
    if (!device_has_tcgen05(net->device))
        return fail(set_error(GBS_ENOTSUP, "this library is built for sm_103a (GB300) only"));
    net->mtiles = (M + kFp64TileModes - 1) / kFp64TileModes;

    // sampler coefficients sqrt(s+-/2), s+- = sinh r e^{+-r}
    std::vector<double2> sq64(N);
    std::vector<float2> sq32(N);
    for (int j = 0; j < N; ++j) {
        const double sp = std::sinh(r[j]) * std::exp(r[j]);
        const double sm = std::sinh(r[j]) * std::exp(-r[j]);
        sq64[j] = make_double2(std::sqrt(0.5 * sp), std::sqrt(0.5 * sm));
        sq32[j] = make_float2((float)sq64[j].x, (float)sq64[j].y);
    }
    if ((rc = net_alloc(net, &net->d_sq64, (size_t)N, "sq64")) ||
        (rc = net_alloc(net, &net->d_sq32, (size_t)N, "sq32")))
        return fail(rc);
    if (cudaMemcpyAsync(net->d_sq64, sq64.data(), sizeof(double2) * N, cudaMemcpyHostToDevice,
                        net->stream) != cudaSuccess ||
        cudaMemcpyAsync(net->d_sq32, sq32.data(), sizeof(float2) * N, cudaMemcpyHostToDevice,
                        net->stream) != cudaSuccess ||
        cudaStreamSynchronize(net->stream) != cudaSuccess)  // the host vectors go out of scope
        return fail(set_error(GBS_ECUDA, "upload of sampler coefficients failed"));

    unsigned long long *d_bad = nullptr;
    if (T_device) {
        if ((rc = net_alloc(net, &d_bad, (size_t)1, "T check"))) return fail(rc);
        if (cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), net->stream) != cudaSuccess) {
            net_free(net, d_bad);
            return fail(set_error(GBS_ECUDA, "memset failed"));
        }
    }
    const int conv_blocks =
        (int)std::min<int64_t>(((int64_t)M * N + 255) / 256, (int64_t)net->sm_count * 16);
    if (simt_precision(precision) && T_device) {
        if ((rc = net_alloc(net, &net->d_T64, (size_t)M * 2 * N, "T64"))) {
            net_free(net, d_bad);
            return fail(rc);
        }
        k_t64_from_dev<<<conv_blocks, 256, 0, net->stream>>>(T, N, M, net->d_T64, d_bad);
        rc = finish_device_T(net, d_bad);
        net_free(net, d_bad);
        if (rc) return fail(rc);
    } else {
        // A = [Re T_i.; Im T_i.] rows interleaved per output mode, T rounded to
        // FP32 and split into BF16 planes T = T0 + T1 + T2, each plane
        // K-blocked [ldK / 32][rowsA][32] so that a 32-wide K block of
        // consecutive rows is one contiguous run of memory.
        net->planesA = 3;
        net->planesB = (precision == GBS_BF16X3) ? 2 : 3;
        net->ldK = (N + 31) / 32 * 32;  // K padded to whole 32-wide blocks
        net->rowsA = 2 * M;
        const size_t plane = (size_t)net->rowsA * net->ldK;
        if (T_device) {
            if ((rc = net_alloc(net, &net->d_A, (size_t)net->planesA * plane, "A planes"))) {
                net_free(net, d_bad);
                return fail(rc);
            }
            if (cudaMemsetAsync(net->d_A, 0, (size_t)net->planesA * plane * sizeof(__nv_bfloat16),
                                net->stream) != cudaSuccess) {
                net_free(net, d_bad);
                return fail(set_error(GBS_ECUDA, "memset of T planes failed"));
            }
            k_split_from_dev<<<conv_blocks, 256, 0, net->stream>>>(T, N, M, net->rowsA, net->d_A,
                                                                  plane, d_bad);
            rc = finish_device_T(net, d_bad);
            net_free(net, d_bad);
            if (rc) return fail(rc);
        }
    }
    // chunk workspace
    net->chunk = pick_chunk(net);
    if (simt_precision(precision)) {
        net->B_bytes = (size_t)net->chunk * 2 * N * sizeof(double);
    } else {
        const int64_t tiles = (net->chunk + kTcTileSamples - 1) / kTcTileSamples;
        net->B_bytes = (size_t)net->planesB * tiles * 256 * net->ldK * sizeof(__nv_bfloat16);
    }
    // the chunk workspace from the stream-ordered pool; the sampler writes
    // every element the GEMM reads for valid trajectories (K padding
    // included), so nothing needs clearing
    if ((rc = pool_alloc(&net->d_B, net->B_bytes, net->stream, "sample operand")) ||
        (rc = pool_alloc_n(&net->d_n, (size_t)net->chunk, net->stream, "n")) ||
        (rc = pool_alloc_n(&net->d_nS_part, (size_t)net->chunk * net->mtiles, net->stream, "nS_part")) ||
        (rc = pool_alloc_n(&net->d_nS, (size_t)net->chunk, net->stream, "nS")) ||
        (rc = pool_alloc_n(&net->d_win, (size_t)net->chunk, net->stream, "windows")) ||
        (rc = net_alloc(net, &net->d_wmax, (size_t)2, "window union")) ||
        (rc = net_alloc(net, &net->d_flags, (size_t)4, "flags")))
        return fail(rc);
    if (cudaMemsetAsync(net->d_flags, 0, 4 * sizeof(unsigned long long), net->stream) != cudaSuccess)
        return fail(set_error(GBS_ECUDA, "memset of flags failed"));
    if (!simt_precision(precision)) {
        if ((rc = pool_alloc(&net->d_gfrec, (size_t)net->chunk * gf_record_bytes(), net->stream,
                             "generating-function records")))
            return fail(rc);
        if ((rc = tc_plan_create(net))) return fail(rc);
    }
    *out = net;
    return GBS_OK;
}

}  // namespace
}  // namespace gbs

extern "C" {

int gbs_make_network(int N, int M, const double *T, const double *r, int precision, void *stream,
                     gbs_net_t *out) {
    return make_network(N, M, T, false, r, precision, stream, out);
}

int gbs_make_network_device(int N, int M, const double *T_dev, const double *r, int precision,
                            void *stream, gbs_net_t *out) {
    return make_network(N, M, T_dev, true, r, precision, stream, out);
}

int gbs_make_network_binned(int N, int M, const double *T, const double *r, const int *bin,
                            int precision, void *stream, gbs_net_t *out) {
    if (!out) return set_error(GBS_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 1 || M < 2 || N > 65536 || M > 65536)
        return set_error(GBS_EINVAL, "N in [1, 65536] and M in [2, 65536] required");
    if (!T || !r || !bin) return set_error(GBS_EINVAL, "T, r and bin must be non-NULL host pointers");
    int Mb[kMaxBins] = {0, 0, 0, 0};
    int d = 0;
    for (int i = 0; i < M; ++i) {
        if (bin[i] < 0 || bin[i] >= kMaxBins)
            return set_error(GBS_EINVAL, "bin[%d] = %d: must be in [0, %d]", i, bin[i], kMaxBins - 1);
        ++Mb[bin[i]];
        d = std::max(d, bin[i] + 1);
    }
    if (d < 2) return set_error(GBS_EINVAL, "need at least two bins");
    for (int b = 0; b < d; ++b)
        if (!Mb[b]) return set_error(GBS_EINVAL, "bin %d has no output mode", b);
    // each bin's rows, then zero rows to a whole tile
    int tiles[kMaxBins + 1] = {0, 0, 0, 0, 0};
    for (int b = 0; b < d; ++b) tiles[b + 1] = tiles[b] + (Mb[b] + kFp64TileModes - 1) / kFp64TileModes;
    for (int b = d; b < kMaxBins; ++b) tiles[b + 1] = tiles[b];
    const int Mp = tiles[d] * kFp64TileModes;
    if (Mp > 65536) return set_error(GBS_EINVAL, "padded output modes exceed 65536");
    std::vector<double> Tp((size_t)2 * Mp * N, 0.0);
    int next[kMaxBins];
    for (int b = 0; b < kMaxBins; ++b) next[b] = tiles[b] * kFp64TileModes;
    for (int i = 0; i < M; ++i) {
        const int row = next[bin[i]]++;
        std::copy(T + (size_t)2 * i * N, T + (size_t)2 * (i + 1) * N, Tp.begin() + (size_t)2 * row * N);
    }
    gbs_net_t net = nullptr;
    int rc = make_network(N, Mp, Tp.data(), false, r, precision, stream, &net);
    if (rc) return rc;
    net->nbins = d;
    for (int b = 0; b <= kMaxBins; ++b) net->bin_tiles[b] = tiles[b];
    net->M_user = M;
    if ((rc = net_alloc(net, &net->d_nS2, (size_t)d * net->chunk, "nS per bin")) ||
        (rc = net_alloc(net, &net->d_win2, (size_t)net->chunk, "windows per bin")) ||
        (rc = net_alloc(net, &net->d_wmax2, (size_t)2 * kMaxBins, "window union per bin"))) {
        gbs_free_network(net);
        return rc;
    }
    *out = net;
    return GBS_OK;
}

int gbs_sample(gbs_net_t net, uint64_t seed, uint64_t first_sample, int64_t E, int n_sub, int K1) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (E < 0) return set_error(GBS_EINVAL, "E must be >= 0");
    if (first_sample + (uint64_t)E < first_sample)
        return set_error(GBS_EINVAL, "sample index range overflows 64 bits");
    if ((rc = fix_estimator(net, n_sub, K1))) return rc;
    if (fold_sampler(net, E, net->chunk)) {
        if ((rc = sample_chunks_pipelined(net, seed, first_sample, E))) return rc;
    } else {
        const int64_t step = chunk_step(net, E);
        for (int64_t done = 0; done < E; done += step) {
            const int64_t c = std::min<int64_t>(step, E - done);
            const uint64_t e0 = first_sample + (uint64_t)done;
            if ((rc = run_chunk_front(net, seed, e0, c))) return rc;
            prof_mark(net, GBS_PHASE_GF, 0, true);
            if ((rc = launch_gf(net, e0, c))) return rc;
            prof_mark(net, GBS_PHASE_GF, 1, false);
        }
    }
    count_samples(net, first_sample, E);
    net->have_last = true;
    net->last_seed = seed;
    net->last_end = first_sample + (uint64_t)E;
    return GBS_OK;
}

int gbs_binned_counts_device(gbs_net_t net, int64_t m_offset, double *out_dev) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (!out_dev) return set_error(GBS_EINVAL, "out_dev is NULL");
    if (!net->est_fixed) return set_error(GBS_EINVAL, "no samples drawn yet");
    for (int q = 0; q < net->n_sub; ++q)
        if (net->counts[q] <= 0)
            return set_error(GBS_EINVAL, "sub-ensemble %d has no trajectories", q);
    int log2k = 0;
    while ((1 << log2k) < net->K1) ++log2k;
    prof_mark(net, GBS_PHASE_INVERT, 0, true);
    if ((rc = launch_invert(net, m_offset, out_dev))) return rc;
    prof_mark(net, GBS_PHASE_INVERT, 2 + log2k, false);
    return GBS_OK;
}

int gbs_check_finite(gbs_net_t net, int64_t *count) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (count) *count = 0;
    // a GEMM launch that gave up waiting on its pipeline since the last check
    unsigned long long timed_out = 0;
    GBS_CUDA_TRY(cudaMemcpyAsync(&timed_out, net->d_flags + 1, sizeof(timed_out),
                                 cudaMemcpyDeviceToHost, net->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(net->stream));
    if (timed_out) {
        GBS_CUDA_TRY(cudaMemsetAsync(net->d_flags + 1, 0, sizeof(unsigned long long), net->stream));
        GBS_CUDA_TRY(cudaStreamSynchronize(net->stream));
        return set_error(GBS_ETIMEOUT, "a GEMM kernel gave up waiting on its pipeline; the sums "
                                       "since the last check are not meaningful");
    }
    if (!net->est_fixed) return GBS_OK;
    prof_mark(net, GBS_PHASE_INVERT, 0, true);
    if ((rc = launch_count_nonfinite(net))) return rc;
    prof_mark(net, GBS_PHASE_INVERT, 1, false);
    unsigned long long h = 0;
    GBS_CUDA_TRY(cudaMemcpyAsync(&h, net->d_flags, sizeof(h), cudaMemcpyDeviceToHost, net->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(net->stream));
    if (count) *count = (int64_t)h;
    if (h) return set_error(GBS_ENONFINITE, "%llu non-finite generating-function sums", h);
    return GBS_OK;
}

int gbs_binned_counts(gbs_net_t net, int64_t m_offset, double *P_mP, double *sig_mP,
                      double *P_plusP, double *sig_plusP) {
    int rc;
    if ((rc = gbs_binned_counts_device(net, m_offset, net ? net->d_out : nullptr))) return rc;
    int64_t bad = 0;
    if ((rc = gbs_check_finite(net, &bad))) return rc;
    double *dst[4] = {P_mP, sig_mP, P_plusP, sig_plusP};
    for (int q = 0; q < 4; ++q)
        if (dst[q])
            GBS_CUDA_TRY(cudaMemcpyAsync(dst[q], net->d_out + (size_t)q * net->K1,
                                         sizeof(double) * net->K1, cudaMemcpyDeviceToHost,
                                         net->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(net->stream));
    return GBS_OK;
}

int gbs_debug_samples(gbs_net_t net, uint64_t seed, uint64_t e0, int64_t count, double *n,
                      double *nS) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (count < 0 || !n || !nS) return set_error(GBS_EINVAL, "bad count or NULL output");
    const int saved_K1 = net->K1;
    if (net->K1 == 0) net->K1 = 2;  // finalize computes windows for some K1; unused here
    for (int64_t done = 0; done < count; done += net->chunk) {
        const int64_t c = std::min<int64_t>(net->chunk, count - done);
        if ((rc = run_chunk_front(net, seed, e0 + (uint64_t)done, c))) {
            net->K1 = saved_K1;
            return rc;
        }
        cudaError_t e1 = cudaMemcpyAsync(n + done, net->d_n, sizeof(double) * c,
                                         cudaMemcpyDeviceToHost, net->stream);
        cudaError_t e2 = cudaMemcpyAsync(nS + 2 * done, net->d_nS, sizeof(double2) * c,
                                         cudaMemcpyDeviceToHost, net->stream);
        cudaError_t e3 = cudaStreamSynchronize(net->stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            net->K1 = saved_K1;
            return set_error(GBS_ECUDA, "debug copy failed: %s",
                             cudaGetErrorString(e3 != cudaSuccess ? e3 : (e2 != cudaSuccess ? e2 : e1)));
        }
    }
    net->K1 = saved_K1;
    return GBS_OK;
}

int gbs_debug_windows(gbs_net_t net, uint64_t seed, uint64_t e0, int64_t count, int *w) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (count < 0 || !w) return set_error(GBS_EINVAL, "bad count or NULL output");
    if (!net->est_fixed) return set_error(GBS_EINVAL, "K1 not fixed yet (call gbs_sample first)");
    static_assert(sizeof(Window) == 2 * sizeof(int), "window layout");
    for (int64_t done = 0; done < count; done += net->chunk) {
        const int64_t c = std::min<int64_t>(net->chunk, count - done);
        if ((rc = run_chunk_front(net, seed, e0 + (uint64_t)done, c))) return rc;
        cudaError_t e1 = cudaMemcpyAsync(w + 2 * done, net->d_win, sizeof(Window) * c,
                                         cudaMemcpyDeviceToHost, net->stream);
        cudaError_t e2 = cudaStreamSynchronize(net->stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess)
            return set_error(GBS_ECUDA, "debug copy failed: %s",
                             cudaGetErrorString(e2 != cudaSuccess ? e2 : e1));
    }
    return GBS_OK;
}

int gbs_histogram(gbs_net_t net, uint64_t seed, uint64_t first_sample, int64_t E, const int *m,
                  int nm, double lo, double hi, int nbins, int64_t *counts) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (E < 0 || !m || !counts) return set_error(GBS_EINVAL, "bad E or NULL m/counts");
    if (nm < 1 || nm > kHistMaxM) return set_error(GBS_EINVAL, "nm must be in [1, %d]", kHistMaxM);
    if (nbins < 1 || nbins > kHistMaxBins)
        return set_error(GBS_EINVAL, "nbins must be in [1, %d]", kHistMaxBins);
    if (!(std::isfinite(lo) && std::isfinite(hi) && hi > lo))
        return set_error(GBS_EINVAL, "need finite lo < hi");
    if ((size_t)2 * nm * (nbins + 2) * sizeof(unsigned int) > 48 * 1024)
        return set_error(GBS_EINVAL, "2 * nm * (nbins + 2) must be <= 12288 (shared-memory counts)");
    HistSpec spec = {};
    for (int q = 0; q < nm; ++q) {
        if (m[q] < 0 || m[q] > 100000) return set_error(GBS_EINVAL, "m[%d] out of range", q);
        spec.m[q] = m[q];
    }
    spec.nm = nm;
    spec.nbins = nbins;
    spec.lo = lo;
    spec.hi = hi;
    const size_t total = (size_t)2 * nm * (nbins + 2);
    unsigned long long *d_cnt = nullptr;
    if ((rc = net_alloc(net, &d_cnt, total, "histogram"))) return rc;
    if (cudaMemsetAsync(d_cnt, 0, total * sizeof(unsigned long long), net->stream) != cudaSuccess)
        rc = set_error(GBS_ECUDA, "memset of the histogram failed");
    const int saved_K1 = net->K1;
    if (net->K1 == 0) net->K1 = 2;  // finalize computes windows for some K1; unused here
    for (int64_t done = 0; !rc && done < E; done += net->chunk) {
        const int64_t c = std::min<int64_t>(net->chunk, E - done);
        rc = run_chunk_front(net, seed, first_sample + (uint64_t)done, c);
        if (!rc) rc = launch_histogram(net, c, spec, d_cnt);
    }
    net->K1 = saved_K1;
    if (!rc) {
        std::vector<unsigned long long> h(total);
        if (cudaMemcpyAsync(h.data(), d_cnt, total * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, net->stream) != cudaSuccess ||
            cudaStreamSynchronize(net->stream) != cudaSuccess)
            rc = set_error(GBS_ECUDA, "histogram copy failed");
        else
            for (size_t q = 0; q < total; ++q) counts[q] = (int64_t)h[q];
    }
    net_free(net, d_cnt);
    return rc;
}

namespace {

// Sampler and propagation GEMM of one chunk with the per-mode occupations
// written to occ (FP32 planes for the BF16 paths, FP64 for the FP64 path).
int run_chunk_occ(gbs_net *net, uint64_t seed, uint64_t e0, int64_t count, void *occ,
                  int64_t ld_occ) {
    int rc;
    const bool fp64 = simt_precision(net->precision);
    const int64_t plane = (int64_t)net->mtiles * 64 * ld_occ;
    prof_mark(net, GBS_PHASE_SAMPLE, 0, true);
    rc = fp64 ? launch_sample_fp64(net, seed, e0, count) : launch_sample_bf16(net, seed, e0, count);
    if (rc) return rc;
    prof_mark(net, GBS_PHASE_SAMPLE, 1, false);
    prof_mark(net, GBS_PHASE_GEMM, 0, true);
    if (fp64) {
        OccOut64 o;
        o.p = static_cast<double *>(occ);
        o.ld = ld_occ;
        o.plane = plane;
        rc = launch_gemm_fp64(net, count, o);
    } else {
        OccOut o;
        o.p = static_cast<float *>(occ);
        o.ld = ld_occ;
        o.plane = plane;
        rc = launch_gemm_tc(net, count, o);
    }
    if (rc) return rc;
    prof_mark(net, GBS_PHASE_GEMM, 1, false);
    return GBS_OK;
}

// Trajectories per occupation chunk: <= the network's chunk, a multiple of
// 128, occupation planes <= 2 GiB.
int64_t occ_chunk(const gbs_net *net, int64_t E) {
    const size_t elt = simt_precision(net->precision) ? sizeof(double) : sizeof(float);
    const size_t per_traj = (size_t)2 * net->mtiles * 64 * elt;
    int64_t c = (int64_t)(((size_t)1 << 31) / per_traj);
    c = std::min<int64_t>(c, net->chunk);
    c = std::min<int64_t>(c, ((E + 127) / 128) * 128);
    c = (c / 128) * 128;
    return std::max<int64_t>(c, 128);
}

}  // namespace

int gbs_debug_occupations(gbs_net_t net, uint64_t seed, uint64_t e0, int64_t count, double *occ) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (count < 0 || !occ) return set_error(GBS_EINVAL, "bad count or NULL output");
    if (net->nbins != 1) return set_error(GBS_EINVAL, "occupations of a binned network are not exposed");
    if (count == 0) return GBS_OK;
    const bool fp64 = simt_precision(net->precision);
    const int64_t ld = occ_chunk(net, count);
    const int64_t plane = (int64_t)net->mtiles * 64 * ld;
    void *d_occ = nullptr;
    if (fp64) rc = net_alloc(net, reinterpret_cast<double **>(&d_occ), (size_t)2 * plane, "occupations");
    else rc = net_alloc(net, reinterpret_cast<float **>(&d_occ), (size_t)2 * plane, "occupations");
    if (rc) return rc;
    const size_t elt = fp64 ? sizeof(double) : sizeof(float);
    std::vector<uint8_t> h((size_t)2 * plane * elt);
    for (int64_t done = 0; !rc && done < count; done += ld) {
        const int64_t c = std::min<int64_t>(ld, count - done);
        rc = run_chunk_occ(net, seed, e0 + (uint64_t)done, c, d_occ, ld);
        if (rc) break;
        if (cudaMemcpyAsync(h.data(), d_occ, h.size(), cudaMemcpyDeviceToHost, net->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(net->stream) != cudaSuccess) {
            rc = set_error(GBS_ECUDA, "occupation copy failed");
            break;
        }
        for (int j = 0; j < net->M; ++j)
            for (int64_t i = 0; i < c; ++i) {
                const size_t a = (size_t)j * ld + i, b = (size_t)plane + a;
                double re, im;
                if (fp64) {
                    re = reinterpret_cast<const double *>(h.data())[a];
                    im = reinterpret_cast<const double *>(h.data())[b];
                } else {
                    re = reinterpret_cast<const float *>(h.data())[a];
                    im = reinterpret_cast<const float *>(h.data())[b];
                }
                occ[2 * ((size_t)j * count + done + i)] = re;
                occ[2 * ((size_t)j * count + done + i) + 1] = im;
            }
    }
    net_free(net, d_occ);
    return rc;
}

int gbs_moments(gbs_net_t net, uint64_t seed, uint64_t first_sample, int64_t E, int n_sub,
                int mmax, int cmax, double *mom, double *sig_mom, double *marg, double *sig_marg) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (net->nbins != 1) return set_error(GBS_EINVAL, "moments need an unbinned network");
    if (mmax < 1 || mmax > 8) return set_error(GBS_EINVAL, "mmax must be in [1, 8]");
    if (cmax < 0 || cmax > 15) return set_error(GBS_EINVAL, "cmax must be in [0, 15]");
    if (n_sub < 1 || n_sub > 65535) return set_error(GBS_EINVAL, "n_sub must be in [1, 65535]");
    if (E < n_sub) return set_error(GBS_EINVAL, "E must be >= n_sub (no empty sub-ensemble)");
    const bool fp64 = simt_precision(net->precision);
    MomentSpec sp;
    sp.M = net->M;
    sp.n_sub = n_sub;
    sp.mmax = mmax;
    sp.cmax = cmax;
    const int Q = moment_quantities(mmax, cmax);
    const int64_t ld = occ_chunk(net, E);
    const int64_t plane = (int64_t)net->mtiles * 64 * ld;
    const size_t nm = (size_t)2 * net->M * mmax, nc = (size_t)2 * net->M * (cmax + 1);
    void *d_occ = nullptr;
    uint8_t *d_par = nullptr;
    double *d_acc = nullptr, *d_out = nullptr, *d_scr = nullptr;
    const int max_seg = moment_max_segments(n_sub, net->M, mmax, cmax);
    int64_t *d_cnt = nullptr;
    if (fp64) rc = net_alloc(net, reinterpret_cast<double **>(&d_occ), (size_t)2 * plane, "occupations");
    else rc = net_alloc(net, reinterpret_cast<float **>(&d_occ), (size_t)2 * plane, "occupations");
    if (!rc) rc = net_alloc(net, &d_par, (size_t)ld * moment_par_bytes(fp64), "trajectory parameters");
    if (!rc) rc = net_alloc(net, &d_acc, (size_t)n_sub * net->M * Q, "moment sums");
    if (!rc && max_seg > 1)
        rc = net_alloc(net, &d_scr, (size_t)max_seg * n_sub * net->M * Q, "moment segment sums");
    if (!rc) rc = net_alloc(net, &d_cnt, (size_t)n_sub, "sub-ensemble sizes");
    if (!rc) rc = net_alloc(net, &d_out, 2 * nm + 2 * nc, "moment outputs");
    if (!rc && cudaMemsetAsync(d_acc, 0, sizeof(double) * n_sub * net->M * Q, net->stream) != cudaSuccess)
        rc = set_error(GBS_ECUDA, "memset of the moment sums failed");
    std::vector<int64_t> cnt((size_t)n_sub, E / n_sub);
    for (int64_t q = 0; q < E % n_sub; ++q) cnt[(size_t)((first_sample + (uint64_t)q) % (uint64_t)n_sub)] += 1;
    if (!rc && cudaMemcpyAsync(d_cnt, cnt.data(), sizeof(int64_t) * n_sub, cudaMemcpyHostToDevice,
                               net->stream) != cudaSuccess)
        rc = set_error(GBS_ECUDA, "copy of the sub-ensemble sizes failed");
    auto consume = [&](uint64_t e0, int64_t c) {
        int r, nl = 0;
        prof_mark(net, GBS_PHASE_MOMENTS, 0, true);
        if ((r = launch_moment_prep(net->d_n, c, fp64, d_par, net->stream, net->sm_count))) return r;
        if ((r = launch_moments(sp, fp64, d_occ, plane, ld, d_par, net->d_n, c, e0, d_acc, d_scr,
                                max_seg, net->d_flags + 1, net->stream, net->sm_count, &nl)))
            return r;
        prof_mark(net, GBS_PHASE_MOMENTS, 1 + nl, false);
        return GBS_OK;
    };
    if (!rc && fold_sampler(net, E, ld)) {
        OccOut o;
        o.p = static_cast<float *>(d_occ);
        o.ld = ld;
        o.plane = plane;
        auto gemm = [&](int64_t c, const SampleJob &job) {
            return job.count ? launch_gemm_tc_sampling(net, c, job, o) : launch_gemm_tc(net, c, o);
        };
        rc = pipelined_chunks(net, seed, first_sample, E, ld, gemm, consume);
    } else {
        for (int64_t done = 0; !rc && done < E; done += ld) {
            const int64_t c = std::min<int64_t>(ld, E - done);
            const uint64_t e0 = first_sample + (uint64_t)done;
            rc = run_chunk_occ(net, seed, e0, c, d_occ, ld);
            if (!rc) rc = consume(e0, c);
        }
    }
    if (!rc) {
        prof_mark(net, GBS_PHASE_MOMENTS, 0, true);
        rc = launch_moment_stats(sp, fp64, d_acc, d_cnt, d_out, net->stream, net->sm_count);
        if (!rc) prof_mark(net, GBS_PHASE_MOMENTS, 1, false);
    }
    if (!rc) {
        std::vector<double> h(2 * nm + 2 * nc);
        unsigned long long timed_out = 0;
        if (cudaMemcpyAsync(h.data(), d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                            net->stream) != cudaSuccess ||
            cudaMemcpyAsync(&timed_out, net->d_flags + 1, sizeof(timed_out), cudaMemcpyDeviceToHost,
                            net->stream) != cudaSuccess ||
            cudaStreamSynchronize(net->stream) != cudaSuccess)
            rc = set_error(GBS_ECUDA, "moment copy failed");
        else if (timed_out) {
            cudaMemsetAsync(net->d_flags + 1, 0, sizeof(unsigned long long), net->stream);
            cudaStreamSynchronize(net->stream);
            rc = set_error(GBS_ETIMEOUT, "a GEMM or moments kernel gave up waiting on its pipeline");
        } else {
            if (mom) std::memcpy(mom, h.data(), sizeof(double) * nm);
            if (sig_mom) std::memcpy(sig_mom, h.data() + nm, sizeof(double) * nm);
            if (marg) std::memcpy(marg, h.data() + 2 * nm, sizeof(double) * nc);
            if (sig_marg) std::memcpy(sig_marg, h.data() + 2 * nm + nc, sizeof(double) * nc);
        }
    }
    net_free(net, d_occ);
    net_free(net, d_par);
    net_free(net, d_acc);
    net_free(net, d_scr);
    net_free(net, d_cnt);
    net_free(net, d_out);
    return rc;
}

int gbs_get_accumulators(gbs_net_t net, int *n_sub, int *K1, double *acc, int64_t *counts) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (n_sub) *n_sub = net->n_sub;
    if (K1) *K1 = net->K1;
    if (!net->est_fixed) return GBS_OK;
    if (acc)
        GBS_CUDA_TRY(cudaMemcpyAsync(acc, net->d_acc, sizeof(double2) * 2 * net->n_sub * net->K1,
                                     cudaMemcpyDeviceToHost, net->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(net->stream));
    if (counts) std::memcpy(counts, net->counts.data(), sizeof(int64_t) * net->n_sub);
    return GBS_OK;
}

int gbs_set_accumulators(gbs_net_t net, int n_sub, int K1, const double *acc,
                         const int64_t *counts) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (!acc || !counts) return set_error(GBS_EINVAL, "acc and counts must be non-NULL");
    for (int q = 0; q < n_sub; ++q)
        if (counts[q] < 0) return set_error(GBS_EINVAL, "negative count");
    if ((rc = fix_estimator(net, n_sub, K1))) return rc;
    GBS_CUDA_TRY(cudaMemcpyAsync(net->d_acc, acc, sizeof(double2) * 2 * n_sub * K1,
                                 cudaMemcpyHostToDevice, net->stream));
    GBS_CUDA_TRY(cudaMemcpyAsync(net->d_counts, counts, sizeof(int64_t) * n_sub,
                                 cudaMemcpyHostToDevice, net->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(net->stream));
    std::memcpy(net->counts.data(), counts, sizeof(int64_t) * n_sub);
    return GBS_OK;
}

int gbs_sample_nd(gbs_net_t net, uint64_t seed, uint64_t first_sample, int64_t E, int n_sub,
                  const int *K) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (net->nbins < 2) return set_error(GBS_EINVAL, "the network has no output bins (gbs_make_network_binned)");
    if (!K) return set_error(GBS_EINVAL, "K is NULL");
    if (E < 0) return set_error(GBS_EINVAL, "E must be >= 0");
    if (first_sample + (uint64_t)E < first_sample)
        return set_error(GBS_EINVAL, "sample index range overflows 64 bits");
    if ((rc = fix_estimator2d(net, n_sub, K))) return rc;
    if (fold_sampler(net, E, net->chunk)) {
        auto gemm = [&](int64_t c, const SampleJob &job) {
            return job.count ? launch_gemm_tc_sampling(net, c, job) : launch_gemm_tc(net, c);
        };
        auto after = [&](uint64_t e0, int64_t c) {
            int r;
            prof_mark(net, GBS_PHASE_FINALIZE, 0, true);
            if ((r = launch_finalize2d(net, c))) return r;
            prof_mark(net, GBS_PHASE_FINALIZE, 1, false);
            prof_mark(net, GBS_PHASE_GF, 0, true);
            if ((r = launch_gf2d(net, e0, c))) return r;
            prof_mark(net, GBS_PHASE_GF, 2, false);
            return GBS_OK;
        };
        if ((rc = pipelined_chunks(net, seed, first_sample, E, net->chunk, gemm, after))) return rc;
    } else {
        for (int64_t done = 0; done < E; done += net->chunk) {
            const int64_t c = std::min<int64_t>(net->chunk, E - done);
            const uint64_t e0 = first_sample + (uint64_t)done;
            if ((rc = run_chunk_front2d(net, seed, e0, c))) return rc;
            prof_mark(net, GBS_PHASE_GF, 0, true);
            if ((rc = launch_gf2d(net, e0, c))) return rc;
            prof_mark(net, GBS_PHASE_GF, simt_precision(net->precision) ? 1 : 2, false);
        }
    }
    const uint64_t ns = (uint64_t)net->n_sub2;
    const uint64_t full = (uint64_t)E / ns, rem = (uint64_t)E % ns;
    const uint64_t start = first_sample % ns;
    for (uint64_t q = 0; q < ns; ++q) net->counts2[q] += (int64_t)full;
    for (uint64_t q = 0; q < rem; ++q) net->counts2[(start + q) % ns] += 1;
    return GBS_OK;
}

int gbs_binned_counts_nd(gbs_net_t net, const int64_t *m_offset, double *P_mP, double *sig_mP,
                         double *P_plusP, double *sig_plusP) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (!net->est2_fixed) return set_error(GBS_EINVAL, "no binned samples drawn yet");
    if (!m_offset) return set_error(GBS_EINVAL, "m_offset is NULL");
    for (int q = 0; q < net->n_sub2; ++q)
        if (net->counts2[q] <= 0)
            return set_error(GBS_EINVAL, "sub-ensemble %d has no trajectories", q);
    int nl = 0;
    prof_mark(net, GBS_PHASE_INVERT, 0, true);
    if ((rc = launch_invert2d(net, m_offset, net->d_out2, &nl))) return rc;
    prof_mark(net, GBS_PHASE_INVERT, nl, false);  // prep, FFT passes, rotations, stats
    const size_t grid = (size_t)net->grid2;
    double *dst[4] = {P_mP, sig_mP, P_plusP, sig_plusP};
    for (int q = 0; q < 4; ++q)
        if (dst[q])
            GBS_CUDA_TRY(cudaMemcpyAsync(dst[q], net->d_out2 + q * grid, sizeof(double) * grid,
                                         cudaMemcpyDeviceToHost, net->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(net->stream));
    return GBS_OK;
}

int gbs_sample_2d(gbs_net_t net, uint64_t seed, uint64_t first_sample, int64_t E, int n_sub,
                  int K1, int K2) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (net->nbins != 2) return set_error(GBS_EINVAL, "the network does not have two output bins");
    const int K[2] = {K1, K2};
    return gbs_sample_nd(net, seed, first_sample, E, n_sub, K);
}

int gbs_binned_counts_2d(gbs_net_t net, int64_t m1_offset, int64_t m2_offset, double *P_mP,
                         double *sig_mP, double *P_plusP, double *sig_plusP) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (net->nbins != 2) return set_error(GBS_EINVAL, "the network does not have two output bins");
    const int64_t mo[2] = {m1_offset, m2_offset};
    return gbs_binned_counts_nd(net, mo, P_mP, sig_mP, P_plusP, sig_plusP);
}

int gbs_reset(gbs_net_t net) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    GBS_CUDA_TRY(cudaStreamSynchronize(net->stream));
    release_estimator(net);
    return GBS_OK;
}

int gbs_network_info(gbs_net_t net, int *N, int *M, int *precision, int64_t *chunk) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (N) *N = net->N;
    if (M) *M = net->M;
    if (precision) *precision = net->precision;
    if (chunk) *chunk = net->chunk;
    return GBS_OK;
}

int gbs_set_gemm_config(gbs_net_t net, int pair, int band, int keep_a) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (simt_precision(net->precision))
        return set_error(GBS_EINVAL, "the FP64 and FP32 paths have no tcgen05 GEMM");
    GemmCfg c;
    c.pair = pair;
    c.band = band;
    c.keep = keep_a;
    return tc_set_config(net, c);
}

int gbs_set_pair_autotune(int enable) {
    tc_set_pair_autotune(enable != 0);
    return GBS_OK;
}

int gbs_set_wait_limit(gbs_net_t net, uint64_t limit_ns) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    net->wait_ns = limit_ns;
    return GBS_OK;
}

int gbs_set_sampler_fusion(gbs_net_t net, int mode) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (mode < 0 || mode > 2) return set_error(GBS_EINVAL, "mode must be 0, 1 or 2");
    net->fuse_sampler = mode;
    return GBS_OK;
}

int gbs_sampler_fusion(gbs_net_t net, int *active) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (!active) return set_error(GBS_EINVAL, "active is NULL");
    *active = (fold_wanted(net) && tc_sampling_ready(net, false)) ? 1 : 0;
    return GBS_OK;
}

int gbs_gemm_config(gbs_net_t net, int *pair, int *band, int *keep_a) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    if (!pair || !band || !keep_a) return set_error(GBS_EINVAL, "NULL argument");
    const GemmCfg c = tc_get_config(net);
    *pair = c.pair;
    *band = c.band;
    *keep_a = c.keep;
    return GBS_OK;
}

int gbs_profile_enable(gbs_net_t net, int enable) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    GBS_CUDA_TRY(cudaStreamSynchronize(net->stream));
    prof_clear(net);
    net->prof.on = enable != 0;
    return GBS_OK;
}

int gbs_profile_read(gbs_net_t net, double *ms, int64_t *launches) {
    int rc;
    if ((rc = validate_net(net))) return rc;
    GBS_CUDA_TRY(cudaStreamSynchronize(net->stream));
    for (int ph = 0; ph < GBS_NPHASES; ++ph) {
        double tot = 0.0;
        const std::vector<cudaEvent_t> &m = net->prof.marks[ph];
        for (size_t q = 0; q + 1 < m.size(); q += 2) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, m[q], m[q + 1]) == cudaSuccess) tot += t;
            else cudaGetLastError();
        }
        if (ms) ms[ph] = tot;
        if (launches) launches[ph] = net->prof.launches[ph];
    }
    prof_clear(net);
    return GBS_OK;
}

void gbs_free_network(gbs_net_t net) {
    if (!net) return;
    cudaStreamSynchronize(net->stream);
    release_all(net);
    delete net;
}

}  // extern "C"
