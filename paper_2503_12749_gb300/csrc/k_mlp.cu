// The surrogate's multilayer perceptron on the tcgen05 tensor cores:
// forward (GEMM + bias + silu), backward (data and weight GEMMs with the
// silu derivative fused), loss, bias gradients and Adam (Kingma & Ba 2015,
// Algorithm 1).  Not part of the paper: it learns the distribution the
// matrix-P ensemble computes.
//
// Every product is C = A B^T with both operands K-major BF16 in global
// memory, loaded by TMA in 32-wide K boxes (64-byte swizzle) into a 4-stage
// shared-memory ring, multiplied by one thread with tcgen05.mma M=128 N=256
// K=16 into a 256-column TMEM accumulator, and read back by four epilogue
// warps with tcgen05.ld.  Weights enter as one BF16 plane (their rounding
// of the FP32 master copy); activations and gradients as two planes hi + lo
// (hi = bf16(x), lo = bf16(x - hi)), so each product of an activation plane
// pair with the weights gives ~16 significant bits:
//   forward          Y_l    = H_{l-1} W_l^T            A = H (2 planes), B = W (1)
//   backward, data   dH_{l-1} = dY_l W_l               A = dY (2), B = W^T (1)
//   backward, weight dW_l   = dY_l^T H_{l-1}           A = dY^T (2), B = H^T (2)
// The forward and backward epilogues write their results both row-major
// (the next layer's A operand) and transposed (the weight GEMM's operands),
// and the Adam kernel writes W and W^T, so that no operand needs a transpose
// inside a GEMM.  The weight GEMM splits its K (the batch) over blockIdx.z;
// the Adam kernel sums the split partials in a fixed order, so a training
// step is deterministic.
#include "gbs_internal.cuh"
#include "gbs_surrogate.h"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

namespace gbs {
namespace {

constexpr int kBM = 128;   // rows of A per tile (TMEM lanes)
constexpr int kBN = 256;   // rows of B per tile (TMEM columns)
constexpr int kStages = 4;
constexpr int kAPlane = kBM * 64;  // bytes of one A plane per 32-wide K block
constexpr int kBPlane = kBN * 64;
constexpr int kStageBytes = 2 * kAPlane + 2 * kBPlane;
constexpr int kSmem = 1024 + kStages * kStageBytes + 256;
constexpr int kThreads = 192;  // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr uint32_t kIdesc = ptx::idesc_bf16_f32(kBM, kBN);
constexpr int kMaxLayers = 8;
constexpr int kInPad = 32;     // input features padded to one K block
constexpr int kMaxSplit = 8;

enum Epi { kEpiHidden = 0, kEpiOut = 1, kEpiBwd = 2, kEpiGrad = 3 };

struct MlpGemm {
    CUtensorMap a[2];  // A planes [rows][K], box 32 x 128
    CUtensorMap b[2];  // B planes [rows][K], box 32 x 256
    int na, nb;        // planes of A and B (products: every pair with ia + ib <= 1)
    int kb_total;      // 32-wide K blocks
    int kb_split;      // K blocks per blockIdx.z
    int mode;
    int rows_valid;    // A rows that carry data (batch rows); others are written as 0
    int cols_valid;    // B rows (output columns) written by kEpiGrad
    const float *bias;             // [N] (kEpiHidden, kEpiOut)
    const float *aux;              // pre-activations [M][ld_aux] (kEpiBwd)
    int ld_aux;
    float *out;                    // FP32 result [M][ld_out] (+ z * split_stride)
    int ld_out;
    int64_t split_stride;
    __nv_bfloat16 *hi, *lo;        // row-major planes [M][ld_bf]
    int ld_bf;
    __nv_bfloat16 *thi, *tlo;      // transposed planes [N][ld_t]
    int ld_t;
    unsigned long long *err;
};

__device__ __forceinline__ float silu_f(float y) { return y / (1.0f + expf(-y)); }

__device__ __forceinline__ float silu_grad_f(float y) {
    const float s = 1.0f / (1.0f + expf(-y));
    return s * (1.0f + y * (1.0f - s));
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &h, __nv_bfloat16 &l) {
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(x - __bfloat162float(h));
}

// Stores of 32 consecutive values of one row: FP32 and two BF16 planes.
__device__ __forceinline__ void store_row_f32(float *dst, const float (&v)[32]) {
    float4 *d = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__device__ __forceinline__ void store_row_planes(__nv_bfloat16 *hi, __nv_bfloat16 *lo,
                                                 const float (&v)[32]) {
    __align__(16) __nv_bfloat16 h[32];
    __align__(16) __nv_bfloat16 l[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) split_bf16(v[i], h[i], l[i]);
    uint4 *dh = reinterpret_cast<uint4 *>(hi);
    uint4 *dl = reinterpret_cast<uint4 *>(lo);
    const uint4 *sh = reinterpret_cast<const uint4 *>(h);
    const uint4 *sl = reinterpret_cast<const uint4 *>(l);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        dh[q] = sh[q];
        dl[q] = sl[q];
    }
}

// Column c0 + i of this thread's row goes to row (c0 + i) of the transposed
// planes; the 32 lanes of a warp hold 32 consecutive rows, so each store
// instruction writes 64 contiguous bytes.
__device__ __forceinline__ void store_col_planes(__nv_bfloat16 *thi, __nv_bfloat16 *tlo, int ld_t,
                                                 int col0, int row, const float (&v)[32]) {
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        __nv_bfloat16 h, l;
        split_bf16(v[i], h, l);
        thi[(size_t)(col0 + i) * ld_t + row] = h;
        tlo[(size_t)(col0 + i) * ld_t + row] = l;
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_mlp_gemm(const __grid_constant__ MlpGemm p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    auto a_tile = [&](int s, int q) { return smem + s * kStageBytes + q * kAPlane; };
    auto b_tile = [&](int s, int q) { return smem + s * kStageBytes + 2 * kAPlane + q * kBPlane; };
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    uint64_t *full = bars;
    uint64_t *empty = bars + kStages;
    uint64_t *tfull = bars + 2 * kStages;
    uint64_t *drain = tfull + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    volatile unsigned long long *err = p.err;
    const int kb0 = blockIdx.z * p.kb_split;
    const int nkb = min(p.kb_total, kb0 + p.kb_split) - kb0;  // >= 1 (host)
    const int m0 = blockIdx.x * kBM;
    const int n0 = blockIdx.y * kBN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(ptx::smem_u32(&full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&empty[s]), 1);
        }
        ptx::mbar_init(ptx::smem_u32(tfull), 1);
        ptx::mbar_init(ptx::smem_u32(drain), 1);
        ptx::fence_barrier_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(tmem_slot), 256);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------------ TMA producer
            for (int q = 0; q < p.na; ++q) ptx::prefetch_tmap(&p.a[q]);
            for (int q = 0; q < p.nb; ++q) ptx::prefetch_tmap(&p.b[q]);
            const uint32_t bytes = (uint32_t)(p.na * kAPlane + p.nb * kBPlane);
            int stage = 0;
            uint32_t phase = 0, used = 0, last_phase = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                if (!ptx::mbar_wait(ptx::smem_u32(&empty[stage]), phase ^ 1u, err)) break;
                const uint32_t fb = ptx::smem_u32(&full[stage]);
                ptx::mbar_arrive_expect_tx(fb, bytes);
                const int kx = (kb0 + kb) * 32;
                for (int q = 0; q < p.na; ++q)
                    ptx::tma_load_2d(ptx::smem_u32(a_tile(stage, q)), &p.a[q], fb, kx, m0);
                for (int q = 0; q < p.nb; ++q)
                    ptx::tma_load_2d(ptx::smem_u32(b_tile(stage, q)), &p.b[q], fb, kx, n0);
                used |= 1u << stage;
                last_phase = (last_phase & ~(1u << stage)) | (phase << stage);
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            // every load issued here has landed before the CTA may exit
            for (int s = 0; s < kStages; ++s)
                if (used & (1u << s))
                    ptx::mbar_wait(ptx::smem_u32(&full[s]), (last_phase >> s) & 1u, err,
                                   200000000ull);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------------ MMA issuer
            // products with ia + ib <= 1, the main product A0 B0 last
            int pa[3], pb[3], np = 0;
            if (p.na > 1) { pa[np] = 1; pb[np] = 0; ++np; }
            if (p.nb > 1) { pa[np] = 0; pb[np] = 1; ++np; }
            pa[np] = 0;
            pb[np] = 0;
            ++np;
            int stage = 0;
            uint32_t phase = 0, acc = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                if (!ptx::mbar_wait(ptx::smem_u32(&full[stage]), phase, err)) break;
                ptx::tc_fence_after();
                for (int pr = 0; pr < np; ++pr) {
                    const uint32_t a0 = ptx::smem_u32(a_tile(stage, pa[pr]));
                    const uint32_t b0 = ptx::smem_u32(b_tile(stage, pb[pr]));
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        ptx::mma_bf16(tmem_base, ptx::desc_k_sw64(a0 + kk * 32),
                                      ptx::desc_k_sw64(b0 + kk * 32), kIdesc, acc);
                        acc = 1u;
                    }
                }
                ptx::mma_commit(ptx::smem_u32(&empty[stage]));
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            ptx::mma_commit(ptx::smem_u32(tfull));
            ptx::mma_commit(ptx::smem_u32(drain));
            ptx::mbar_wait(ptx::smem_u32(drain), 0u, err, 200000000ull);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        ptx::mbar_wait(ptx::smem_u32(tfull), 0u, err);
        ptx::tc_fence_after();
        const int quarter = warp & 3;
        const int row = m0 + quarter * 32 + lane;
        const bool live = row < p.rows_valid;
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        for (int c0 = 0; c0 < kBN; c0 += 32) {
            float v[32];
            ptx::tmem_ld32(lane_base + (uint32_t)c0, v);
            ptx::tmem_ld_wait();
            const int col0 = n0 + c0;
            if (p.mode == kEpiHidden) {
                float h[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float y = live ? v[i] + p.bias[col0 + i] : 0.0f;
                    v[i] = y;
                    h[i] = live ? silu_f(y) : 0.0f;
                }
                store_row_f32(p.out + (size_t)row * p.ld_out + col0, v);
                store_row_planes(p.hi + (size_t)row * p.ld_bf + col0,
                                 p.lo + (size_t)row * p.ld_bf + col0, h);
                store_col_planes(p.thi, p.tlo, p.ld_t, col0, row, h);
            } else if (p.mode == kEpiOut) {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] += p.bias[col0 + i];
                store_row_f32(p.out + (size_t)row * p.ld_out + col0, v);
            } else if (p.mode == kEpiBwd) {
                const float *pre = p.aux + (size_t)row * p.ld_aux + col0;
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = live ? v[i] * silu_grad_f(pre[i]) : 0.0f;
                store_row_f32(p.out + (size_t)row * p.ld_out + col0, v);
                store_row_planes(p.hi + (size_t)row * p.ld_bf + col0,
                                 p.lo + (size_t)row * p.ld_bf + col0, v);
                store_col_planes(p.thi, p.tlo, p.ld_t, col0, row, v);
            } else if (col0 < p.cols_valid) {  // kEpiGrad
                store_row_f32(p.out + blockIdx.z * p.split_stride + (size_t)row * p.ld_out + col0,
                              v);
            }
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, 256);
    }
}

// Inputs X [B][in_dim] FP32 -> planes [B_pad][32] and transposed [32][ld_t];
// padding rows and columns are 0.
__global__ void k_mlp_input(const float *__restrict__ X, int B, int in_dim, int B_pad,
                            __nv_bfloat16 *hi, __nv_bfloat16 *lo, __nv_bfloat16 *thi,
                            __nv_bfloat16 *tlo, int ld_t) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B_pad * kInPad) return;
    const int row = idx / kInPad;
    const int c = idx % kInPad;
    const float x = (row < B && c < in_dim) ? X[(size_t)row * in_dim + c] : 0.0f;
    __nv_bfloat16 h, l;
    split_bf16(x, h, l);
    hi[idx] = h;
    lo[idx] = l;
    thi[(size_t)c * ld_t + row] = h;
    tlo[(size_t)c * ld_t + row] = l;
}

// Loss gradient dL/dy = 2 (y - t) / (B O) for rows < B (0 for padding rows),
// written FP32 [B_pad][O], as planes and transposed planes; per 32 x 32 tile
// the squared errors of each row into part[col tile][row].  Block (32, 8).
// One thread also advances the step counters and the Adam bias corrections.
__global__ void k_mlp_loss(const float *__restrict__ Y, const float *__restrict__ T, int B, int O,
                           int B_pad, float *__restrict__ dy, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                           __nv_bfloat16 *thi, __nv_bfloat16 *tlo, int ld_t,
                           float *__restrict__ part, int count_step, long long *step,
                           float *corr) {
    __shared__ float th[32][33];
    __shared__ float tl[32][33];
    __shared__ float se[8][32];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const float scale = 2.0f / ((float)B * (float)O);
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int k = 0; k < 4; ++k) {
        const int rr = ty + 8 * k;
        const int row = r0 + rr;
        const int col = c0 + tx;
        float g = 0.0f;
        if (row < B) {
            const float e = Y[(size_t)row * O + col] - T[(size_t)row * O + col];
            g = scale * e;
            acc[k] = e * e;
        }
        dy[(size_t)row * O + col] = g;
        __nv_bfloat16 h, l;
        split_bf16(g, h, l);
        hi[(size_t)row * O + col] = h;
        lo[(size_t)row * O + col] = l;
        th[rr][tx] = __bfloat162float(h);
        tl[rr][tx] = __bfloat162float(l);
    }
    __syncthreads();
    for (int k = 0; k < 4; ++k) {
        const int cc = ty + 8 * k;
        thi[(size_t)(c0 + cc) * ld_t + r0 + tx] = __float2bfloat16_rn(th[tx][cc]);
        tlo[(size_t)(c0 + cc) * ld_t + r0 + tx] = __float2bfloat16_rn(tl[tx][cc]);
    }
    // squared errors: sum over the 32 columns of each row, fixed order
    for (int k = 0; k < 4; ++k) {
        float s = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (tx == 0) se[ty][k] = s;
    }
    __syncthreads();
    if (ty == 0) {
        const int rr = tx;  // row r0 + rr came from thread row (rr % 8), k = rr / 8
        part[(size_t)blockIdx.x * B_pad + r0 + rr] = se[rr % 8][rr / 8];
    }
    if (count_step && blockIdx.x == 0 && blockIdx.y == 0 && tx == 0 && ty == 0) {
        const long long t = step[0] + 1;
        step[0] = t;
        step[1] += 1;  // steps of the current training call
        corr[0] = (float)(1.0 - pow(0.9, (double)t));
        corr[1] = (float)(1.0 - pow(0.999, (double)t));
    }
}

// loss = sum of the row partials (fixed order) / (B O), into out[index].
__global__ void k_mlp_loss_reduce(const float *__restrict__ part, int ntiles, int B_pad, int B,
                                  int O, const long long *step, int use_step, float *out,
                                  double *out64) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < B_pad; i += blockDim.x)
        for (int t = 0; t < ntiles; ++t) s += (double)part[(size_t)t * B_pad + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double l = red[0] / ((double)B * (double)O);
        const long long idx = use_step ? step[1] - 1 : 0;
        if (out) out[idx] = (float)l;
        if (out64) *out64 = l;
    }
}

struct BiasJob {
    const float *dy[kMaxLayers];
    float *db[kMaxLayers];
    int n[kMaxLayers];
};

// db_l[c] = sum over the batch rows of dy_l[row][c] (fixed order).
__global__ void k_mlp_bias_grad(BiasJob job, int B) {
    const int l = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= job.n[l]) return;
    const float *d = job.dy[l];
    const int n = job.n[l];
    float s = 0.0f;
    for (int r = 0; r < B; ++r) s += d[(size_t)r * n + c];
    job.db[l][c] = s;
}

struct Layout {
    int L;
    int n_out[kMaxLayers], k_pad[kMaxLayers];
    int64_t off_W[kMaxLayers], off_b[kMaxLayers], end[kMaxLayers];  // master layout
    const float *dw[kMaxLayers];  // [S][n_out][k_pad] partials
    const float *db[kMaxLayers];
    int S[kMaxLayers];
    __nv_bfloat16 *wbf[kMaxLayers], *wtbf[kMaxLayers];
};

// Gradient of master element i (fixed-order sum of the split partials).
__device__ __forceinline__ float grad_of(const Layout &lay, int64_t i, int &l, int &n, int &k,
                                         bool &is_w) {
    l = 0;
    while (l + 1 < lay.L && i >= lay.end[l]) ++l;
    if (i < lay.off_b[l]) {
        is_w = true;
        const int64_t j = i - lay.off_W[l];
        n = (int)(j / lay.k_pad[l]);
        k = (int)(j % lay.k_pad[l]);
        const int64_t plane = (int64_t)lay.n_out[l] * lay.k_pad[l];
        float g = 0.0f;
        for (int z = 0; z < lay.S[l]; ++z) g += lay.dw[l][z * plane + j];
        return g;
    }
    is_w = false;
    n = (int)(i - lay.off_b[l]);
    k = 0;
    return lay.db[l][n];
}

// Adam on every master element; refreshes the BF16 W and W^T copies.  With
// grad_out != NULL only writes the gradient (no update).
__global__ void k_mlp_adam(Layout lay, int64_t total, float *__restrict__ master,
                           float *__restrict__ mom1, float *__restrict__ mom2,
                           const float *__restrict__ lr_tab, const long long *step,
                           const float *corr, float *__restrict__ grad_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int l, n, k;
    bool is_w;
    const float g = grad_of(lay, i, l, n, k, is_w);
    if (grad_out) {
        grad_out[i] = g;
        return;
    }
    const float lr = lr_tab[step[1] - 1];
    const float m1 = 0.9f * mom1[i] + 0.1f * g;
    const float m2 = 0.999f * mom2[i] + 0.001f * g * g;
    mom1[i] = m1;
    mom2[i] = m2;
    const float w = master[i] - lr * (m1 / corr[0]) / (sqrtf(m2 / corr[1]) + 1e-8f);
    master[i] = w;
    if (is_w) {
        const __nv_bfloat16 wb = __float2bfloat16_rn(w);
        lay.wbf[l][(size_t)n * lay.k_pad[l] + k] = wb;
        if (lay.wtbf[l]) lay.wtbf[l][(size_t)k * lay.n_out[l] + n] = wb;
    }
}

// BF16 copies of the master weights (after gbs_mlp_set_params).
__global__ void k_mlp_refresh(Layout lay, int64_t total, const float *__restrict__ master) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int l = 0;
    while (l + 1 < lay.L && i >= lay.end[l]) ++l;
    if (i >= lay.off_b[l]) return;
    const int64_t j = i - lay.off_W[l];
    const int n = (int)(j / lay.k_pad[l]);
    const int k = (int)(j % lay.k_pad[l]);
    const __nv_bfloat16 wb = __float2bfloat16_rn(master[i]);
    lay.wbf[l][j] = wb;
    if (lay.wtbf[l]) lay.wtbf[l][(size_t)k * lay.n_out[l] + n] = wb;
}

template <typename T>
int mlp_alloc(T **p, size_t count, std::vector<void *> &owned) {
    *p = nullptr;
    if (count == 0) return GBS_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(GBS_ENOMEM, "cudaMalloc(%zu bytes) for the MLP failed: %s",
                         count * sizeof(T), cudaGetErrorString(e));
    }
    owned.push_back(*p);
    e = cudaMemset(*p, 0, count * sizeof(T));
    if (e != cudaSuccess) return set_error(GBS_ECUDA, "cudaMemset failed: %s", cudaGetErrorString(e));
    return GBS_OK;
}

bool g_attr_done[64] = {};

}  // namespace
}  // namespace gbs

using namespace gbs;

struct gbs_mlp {
    int in_dim = 0, width = 0, out_dim = 0, L = 0, max_batch = 0, Bmax = 0;  // Bmax: padded
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    std::vector<void *> owned;
    Layout lay = {};
    int64_t nmaster = 0, nparams = 0;
    float *master = nullptr, *m1 = nullptr, *m2 = nullptr, *grad = nullptr;
    __nv_bfloat16 *xp = nullptr, *xtp = nullptr;           // 2 planes each
    float *pre[kMaxLayers] = {};                            // hidden layers
    __nv_bfloat16 *hp[kMaxLayers] = {}, *htp[kMaxLayers] = {};
    float *y = nullptr;
    float *dy[kMaxLayers] = {};
    __nv_bfloat16 *dyp[kMaxLayers] = {}, *dytp[kMaxLayers] = {};
    float *dw[kMaxLayers] = {}, *db[kMaxLayers] = {};
    float *part = nullptr;
    long long *step = nullptr;  // [2]: Adam steps, steps of the current training call
    float *corr = nullptr;      // [2]: 1 - beta1^t, 1 - beta2^t
    float *lr = nullptr;
    int lr_cap = 0;
    float *loss_hist = nullptr;
    int hist_cap = 0;
    double *loss64 = nullptr;
    unsigned long long *err = nullptr;
    // the training graph and what it was captured for
    cudaGraphExec_t graph = nullptr;
    const float *g_X = nullptr, *g_T = nullptr;
    int g_batch = -1;
};

namespace {

size_t plane_elems(int rows, int cols) { return (size_t)rows * cols; }

// Plan of one GEMM launch.
struct Launch {
    MlpGemm p;
    dim3 grid;
};

int make_gemm(gbs_mlp *m, Launch &out, int mode, __nv_bfloat16 *a0, __nv_bfloat16 *a1,
              int a_rows, int a_ld, __nv_bfloat16 *b0, __nv_bfloat16 *b1, int b_rows, int b_ld,
              int K, int M, int N, int split) {
    MlpGemm &p = out.p;
    p = MlpGemm{};
    int rc;
    if ((rc = encode_2d(&p.a[0], a0, (uint64_t)a_ld, (uint64_t)a_rows, (uint64_t)a_ld * 2, 32, 128)))
        return rc;
    p.na = 1;
    if (a1) {
        if ((rc = encode_2d(&p.a[1], a1, (uint64_t)a_ld, (uint64_t)a_rows, (uint64_t)a_ld * 2, 32,
                            128)))
            return rc;
        p.na = 2;
    }
    if ((rc = encode_2d(&p.b[0], b0, (uint64_t)b_ld, (uint64_t)b_rows, (uint64_t)b_ld * 2, 32, 256)))
        return rc;
    p.nb = 1;
    if (b1) {
        if ((rc = encode_2d(&p.b[1], b1, (uint64_t)b_ld, (uint64_t)b_rows, (uint64_t)b_ld * 2, 32,
                            256)))
            return rc;
        p.nb = 2;
    }
    p.kb_total = K / 32;
    const int S = std::max(1, std::min(split, p.kb_total));
    p.kb_split = (p.kb_total + S - 1) / S;
    const int Z = (p.kb_total + p.kb_split - 1) / p.kb_split;
    p.mode = mode;
    p.err = m->err;
    out.grid = dim3((unsigned)(M / kBM), (unsigned)((N + kBN - 1) / kBN), (unsigned)Z);
    return GBS_OK;
}

int launch(gbs_mlp *m, const Launch &l) {
    k_mlp_gemm<<<l.grid, kThreads, kSmem, m->stream>>>(l.p);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int ensure_attr() {
    int dev = 0;
    GBS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && g_attr_done[dev]) return GBS_OK;
    GBS_CUDA_TRY(cudaFuncSetAttribute(k_mlp_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
    if (dev >= 0 && dev < 64) g_attr_done[dev] = true;
    return GBS_OK;
}

int split_count(int kb_total) { return std::max(1, std::min(kMaxSplit, kb_total / 2)); }

// Forward of `batch` rows (B_pad = batch rounded up to 128); input planes
// must be written already.  Output into m->y.
int run_forward(gbs_mlp *m, int batch) {
    const int Bp = (batch + kBM - 1) / kBM * kBM;
    int rc;
    for (int l = 0; l < m->L; ++l) {
        Launch g;
        const bool last = l == m->L - 1;
        __nv_bfloat16 *a0 = l == 0 ? m->xp : m->hp[l - 1];
        __nv_bfloat16 *a1 = a0 + (size_t)m->Bmax * (l == 0 ? kInPad : m->width);
        const int k = m->lay.k_pad[l];
        const int n = m->lay.n_out[l];
        if ((rc = make_gemm(m, g, last ? kEpiOut : kEpiHidden, a0, a1, m->Bmax, k,
                            m->lay.wbf[l], nullptr, n, k, k, Bp, n, 1)))
            return rc;
        g.p.rows_valid = batch;
        g.p.bias = m->master + m->lay.off_b[l];
        if (last) {
            g.p.out = m->y;
            g.p.ld_out = n;
        } else {
            g.p.out = m->pre[l];
            g.p.ld_out = n;
            g.p.hi = m->hp[l];
            g.p.lo = m->hp[l] + (size_t)m->Bmax * n;
            g.p.ld_bf = n;
            g.p.thi = m->htp[l];
            g.p.tlo = m->htp[l] + (size_t)n * m->Bmax;
            g.p.ld_t = m->Bmax;
        }
        if ((rc = launch(m, g))) return rc;
    }
    return GBS_OK;
}

int run_input(gbs_mlp *m, const float *X, int batch) {
    const int Bp = (batch + kBM - 1) / kBM * kBM;
    const int total = Bp * kInPad;
    k_mlp_input<<<(total + 255) / 256, 256, 0, m->stream>>>(
        X, batch, m->in_dim, Bp, m->xp, m->xp + (size_t)m->Bmax * kInPad, m->xtp,
        m->xtp + (size_t)kInPad * m->Bmax, m->Bmax);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

// Loss, backward and the gradient partials of one batch (after run_forward).
int run_backward(gbs_mlp *m, const float *T, int batch, int count_step, float *hist) {
    const int Bp = (batch + kBM - 1) / kBM * kBM;
    const int L = m->L;
    const int O = m->out_dim;
    int rc;
    {
        dim3 grid((unsigned)(O / 32), (unsigned)(Bp / 32));
        k_mlp_loss<<<grid, dim3(32, 8), 0, m->stream>>>(
            m->y, T, batch, O, Bp, m->dy[L - 1], m->dyp[L - 1],
            m->dyp[L - 1] + (size_t)m->Bmax * O, m->dytp[L - 1],
            m->dytp[L - 1] + (size_t)O * m->Bmax, m->Bmax, m->part, count_step, m->step, m->corr);
        GBS_LAUNCH_CHECK();
        k_mlp_loss_reduce<<<1, 256, 0, m->stream>>>(m->part, O / 32, Bp, batch, O, m->step,
                                                     count_step, hist, m->loss64);
        GBS_LAUNCH_CHECK();
    }
    // data gradients, layer L-1 .. 1 (0-based l: dY_{l-1} from dY_l)
    for (int l = L - 1; l >= 1; --l) {
        const int n = m->lay.n_out[l];
        const int k = m->lay.k_pad[l];  // = width
        Launch g;
        if ((rc = make_gemm(m, g, kEpiBwd, m->dyp[l], m->dyp[l] + (size_t)m->Bmax * n, m->Bmax, n,
                            m->lay.wtbf[l], nullptr, k, n, n, Bp, k, 1)))
            return rc;
        g.p.rows_valid = batch;
        g.p.aux = m->pre[l - 1];
        g.p.ld_aux = k;
        g.p.out = m->dy[l - 1];
        g.p.ld_out = k;
        g.p.hi = m->dyp[l - 1];
        g.p.lo = m->dyp[l - 1] + (size_t)m->Bmax * k;
        g.p.ld_bf = k;
        g.p.thi = m->dytp[l - 1];
        g.p.tlo = m->dytp[l - 1] + (size_t)k * m->Bmax;
        g.p.ld_t = m->Bmax;
        if ((rc = launch(m, g))) return rc;
    }
    // weight gradients: dW_l = dY_l^T H_{l-1}, K = the batch
    for (int l = 0; l < L; ++l) {
        const int n = m->lay.n_out[l];
        const int k = m->lay.k_pad[l];
        __nv_bfloat16 *b0 = l == 0 ? m->xtp : m->htp[l - 1];
        __nv_bfloat16 *b1 = b0 + (size_t)k * m->Bmax;
        Launch g;
        if ((rc = make_gemm(m, g, kEpiGrad, m->dytp[l], m->dytp[l] + (size_t)n * m->Bmax, n,
                            m->Bmax, b0, b1, k, m->Bmax, Bp, n, k, split_count(Bp / 32))))
            return rc;
        g.p.cols_valid = k;
        g.p.out = m->dw[l];
        g.p.ld_out = k;
        g.p.split_stride = (int64_t)n * k;
        m->lay.S[l] = (int)g.grid.z;
        if ((rc = launch(m, g))) return rc;
    }
    BiasJob job = {};
    int nmax = 0;
    for (int l = 0; l < L; ++l) {
        job.dy[l] = m->dy[l];
        job.db[l] = m->db[l];
        job.n[l] = m->lay.n_out[l];
        nmax = std::max(nmax, job.n[l]);
    }
    k_mlp_bias_grad<<<dim3((unsigned)((nmax + 127) / 128), (unsigned)L), 128, 0, m->stream>>>(job,
                                                                                             batch);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int run_adam(gbs_mlp *m, float *grad_out) {
    for (int l = 0; l < m->L; ++l) {
        m->lay.dw[l] = m->dw[l];
        m->lay.db[l] = m->db[l];
    }
    const int64_t total = m->nmaster;
    k_mlp_adam<<<(unsigned)((total + 255) / 256), 256, 0, m->stream>>>(
        m->lay, total, m->master, m->m1, m->m2, m->lr, m->step, m->corr, grad_out);
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

int check_err(gbs_mlp *m) {
    unsigned long long h = 0;
    GBS_CUDA_TRY(cudaMemcpyAsync(&h, m->err, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (h) {
        cudaMemsetAsync(m->err, 0, sizeof(unsigned long long), m->stream);
        return set_error(GBS_ETIMEOUT, "an MLP GEMM gave up waiting on its pipeline");
    }
    return GBS_OK;
}

int check_batch(gbs_mlp *m, int batch) {
    if (batch < 1 || batch > m->max_batch)
        return set_error(GBS_EINVAL, "batch %d outside [1, %d]", batch, m->max_batch);
    return GBS_OK;
}

// packed (user) index <-> master (padded) index
template <typename F>
void for_each_param(const gbs_mlp *m, F f) {
    int64_t u = 0;
    for (int l = 0; l < m->L; ++l) {
        const int kin = l == 0 ? m->in_dim : m->width;
        for (int n = 0; n < m->lay.n_out[l]; ++n)
            for (int k = 0; k < kin; ++k) f(u++, m->lay.off_W[l] + (int64_t)n * m->lay.k_pad[l] + k);
        for (int n = 0; n < m->lay.n_out[l]; ++n) f(u++, m->lay.off_b[l] + n);
    }
}

void destroy(gbs_mlp *m) {
    if (!m) return;
    if (m->graph) cudaGraphExecDestroy(m->graph);
    for (void *p : m->owned) cudaFree(p);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

}  // namespace

extern "C" {

int gbs_mlp_create(int in_dim, int width, int out_dim, int layers, int max_batch, void *stream,
                   gbs_mlp_t *out) {
    if (!out) return set_error(GBS_EINVAL, "out is NULL");
    *out = nullptr;
    if (in_dim < 1 || in_dim > kInPad) return set_error(GBS_EINVAL, "in_dim must be in [1, 32]");
    if (width < 256 || width > 4096 || width % 256 || out_dim < 256 || out_dim > 4096 ||
        out_dim % 256)
        return set_error(GBS_EINVAL, "width and out_dim must be multiples of 256 in [256, 4096]");
    if (layers < 2 || layers > kMaxLayers)
        return set_error(GBS_EINVAL, "layers must be in [2, %d]", kMaxLayers);
    if (max_batch < 1 || max_batch > 65536) return set_error(GBS_EINVAL, "max_batch must be in [1, 65536]");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return set_error(GBS_ECUDA, "no usable CUDA device");
    }
    if (!device_has_tcgen05(dev)) return set_error(GBS_ENOTSUP, "this library is built for sm_103a (GB300) only");
    int rc;
    if ((rc = ensure_attr())) return rc;
    gbs_mlp *m = new (std::nothrow) gbs_mlp();
    if (!m) return set_error(GBS_ENOMEM, "host allocation failed");
    m->in_dim = in_dim;
    m->width = width;
    m->out_dim = out_dim;
    m->L = layers;
    m->max_batch = max_batch;
    m->Bmax = (max_batch + kBM - 1) / kBM * kBM;
    m->device = dev;
    if (stream) {
        m->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete m;
            return set_error(GBS_ECUDA, "cudaStreamCreate failed");
        }
        m->own_stream = true;
    }
    auto fail = [&](int code) {
        destroy(m);
        return code;
    };
    Layout &lay = m->lay;
    lay.L = layers;
    int64_t off = 0;
    m->nparams = 0;
    for (int l = 0; l < layers; ++l) {
        lay.n_out[l] = l == layers - 1 ? out_dim : width;
        lay.k_pad[l] = l == 0 ? kInPad : width;
        lay.off_W[l] = off;
        off += (int64_t)lay.n_out[l] * lay.k_pad[l];
        lay.off_b[l] = off;
        off += lay.n_out[l];
        lay.end[l] = off;
        m->nparams += (int64_t)lay.n_out[l] * (l == 0 ? in_dim : width) + lay.n_out[l];
    }
    m->nmaster = off;
    const int B = m->Bmax;
    if ((rc = mlp_alloc(&m->master, (size_t)off, m->owned)) ||
        (rc = mlp_alloc(&m->m1, (size_t)off, m->owned)) ||
        (rc = mlp_alloc(&m->m2, (size_t)off, m->owned)) ||
        (rc = mlp_alloc(&m->grad, (size_t)off, m->owned)) ||
        (rc = mlp_alloc(&m->xp, 2 * plane_elems(B, kInPad), m->owned)) ||
        (rc = mlp_alloc(&m->xtp, 2 * plane_elems(kInPad, B), m->owned)) ||
        (rc = mlp_alloc(&m->y, plane_elems(B, out_dim), m->owned)) ||
        (rc = mlp_alloc(&m->part, plane_elems(out_dim / 32, B), m->owned)) ||
        (rc = mlp_alloc(&m->step, 2, m->owned)) || (rc = mlp_alloc(&m->corr, 2, m->owned)) ||
        (rc = mlp_alloc(&m->loss64, 1, m->owned)) || (rc = mlp_alloc(&m->err, 1, m->owned)))
        return fail(rc);
    for (int l = 0; l < layers; ++l) {
        const int n = lay.n_out[l], k = lay.k_pad[l];
        const int S = split_count(B / 32);
        if ((rc = mlp_alloc(&lay.wbf[l], plane_elems(n, k), m->owned)) ||
            (l > 0 && (rc = mlp_alloc(&lay.wtbf[l], plane_elems(k, n), m->owned))) ||
            (rc = mlp_alloc(&m->dy[l], plane_elems(B, n), m->owned)) ||
            (rc = mlp_alloc(&m->dyp[l], 2 * plane_elems(B, n), m->owned)) ||
            (rc = mlp_alloc(&m->dytp[l], 2 * plane_elems(n, B), m->owned)) ||
            (rc = mlp_alloc(&m->dw[l], (size_t)S * plane_elems(n, k), m->owned)) ||
            (rc = mlp_alloc(&m->db[l], (size_t)n, m->owned)))
            return fail(rc);
        if (l < layers - 1) {
            if ((rc = mlp_alloc(&m->pre[l], plane_elems(B, n), m->owned)) ||
                (rc = mlp_alloc(&m->hp[l], 2 * plane_elems(B, n), m->owned)) ||
                (rc = mlp_alloc(&m->htp[l], 2 * plane_elems(n, B), m->owned)))
                return fail(rc);
        }
    }
    *out = m;
    return GBS_OK;
}

int gbs_mlp_param_count(gbs_mlp_t m, int64_t *count) {
    if (!m || !count) return set_error(GBS_EINVAL, "NULL argument");
    *count = m->nparams;
    return GBS_OK;
}

int gbs_mlp_set_params(gbs_mlp_t m, const float *params) {
    if (!m || !params) return set_error(GBS_EINVAL, "NULL argument");
    for (int64_t i = 0; i < m->nparams; ++i)
        if (!std::isfinite(params[i])) return set_error(GBS_EINVAL, "parameter %lld is not finite", (long long)i);
    std::vector<float> h((size_t)m->nmaster, 0.0f);
    for_each_param(m, [&](int64_t u, int64_t i) { h[(size_t)i] = params[u]; });
    GBS_CUDA_TRY(cudaMemcpyAsync(m->master, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice,
                                 m->stream));
    GBS_CUDA_TRY(cudaMemsetAsync(m->m1, 0, h.size() * sizeof(float), m->stream));
    GBS_CUDA_TRY(cudaMemsetAsync(m->m2, 0, h.size() * sizeof(float), m->stream));
    GBS_CUDA_TRY(cudaMemsetAsync(m->step, 0, 2 * sizeof(long long), m->stream));
    k_mlp_refresh<<<(unsigned)((m->nmaster + 255) / 256), 256, 0, m->stream>>>(m->lay, m->nmaster,
                                                                                m->master);
    GBS_LAUNCH_CHECK();
    GBS_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return GBS_OK;
}

static int copy_packed(gbs_mlp_t m, const float *src_dev, float *dst) {
    std::vector<float> h((size_t)m->nmaster);
    GBS_CUDA_TRY(cudaMemcpyAsync(h.data(), src_dev, h.size() * sizeof(float), cudaMemcpyDeviceToHost,
                                 m->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(m->stream));
    for_each_param(m, [&](int64_t u, int64_t i) { dst[u] = h[(size_t)i]; });
    return GBS_OK;
}

int gbs_mlp_get_params(gbs_mlp_t m, float *params) {
    if (!m || !params) return set_error(GBS_EINVAL, "NULL argument");
    return copy_packed(m, m->master, params);
}

int gbs_mlp_get_adam_state(gbs_mlp_t m, float *mom1, float *mom2, int64_t *step) {
    if (!m) return set_error(GBS_EINVAL, "NULL argument");
    int rc;
    if (mom1 && (rc = copy_packed(m, m->m1, mom1))) return rc;
    if (mom2 && (rc = copy_packed(m, m->m2, mom2))) return rc;
    if (step) {
        long long h[2] = {0, 0};
        GBS_CUDA_TRY(cudaMemcpyAsync(h, m->step, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
        GBS_CUDA_TRY(cudaStreamSynchronize(m->stream));
        *step = h[0];
    }
    return GBS_OK;
}

int gbs_mlp_forward(gbs_mlp_t m, const float *X_dev, int batch, float *Y_dev) {
    if (!m || !X_dev || !Y_dev) return set_error(GBS_EINVAL, "NULL argument");
    int rc;
    if ((rc = check_batch(m, batch))) return rc;
    if ((rc = run_input(m, X_dev, batch)) || (rc = run_forward(m, batch))) return rc;
    GBS_CUDA_TRY(cudaMemcpyAsync(Y_dev, m->y, sizeof(float) * (size_t)batch * m->out_dim,
                                 cudaMemcpyDeviceToDevice, m->stream));
    return GBS_OK;
}

int gbs_mlp_gradients(gbs_mlp_t m, const float *X_dev, const float *T_dev, int batch, double *loss,
                      float *grad) {
    if (!m || !X_dev || !T_dev) return set_error(GBS_EINVAL, "NULL argument");
    int rc;
    if ((rc = check_batch(m, batch))) return rc;
    if ((rc = run_input(m, X_dev, batch)) || (rc = run_forward(m, batch)) ||
        (rc = run_backward(m, T_dev, batch, 0, nullptr)) || (rc = run_adam(m, m->grad)))
        return rc;
    if ((rc = check_err(m))) return rc;
    if (loss) {
        GBS_CUDA_TRY(cudaMemcpyAsync(loss, m->loss64, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
        GBS_CUDA_TRY(cudaStreamSynchronize(m->stream));
    }
    if (grad && (rc = copy_packed(m, m->grad, grad))) return rc;
    return GBS_OK;
}

int gbs_mlp_train(gbs_mlp_t m, const float *X_dev, const float *T_dev, int batch, int steps,
                  const float *lr, float *loss_hist) {
    if (!m || !X_dev || !T_dev || !lr) return set_error(GBS_EINVAL, "NULL argument");
    if (steps < 0) return set_error(GBS_EINVAL, "steps must be >= 0");
    int rc;
    if ((rc = check_batch(m, batch))) return rc;
    if (steps == 0) return GBS_OK;
    for (int i = 0; i < steps; ++i)
        if (!std::isfinite(lr[i]) || lr[i] < 0.0f) return set_error(GBS_EINVAL, "lr[%d] invalid", i);
    if (steps > m->lr_cap) {
        float *p = nullptr;
        if ((rc = mlp_alloc(&p, (size_t)steps, m->owned))) return rc;
        m->lr = p;
        m->lr_cap = steps;
        float *h = nullptr;
        if ((rc = mlp_alloc(&h, (size_t)steps, m->owned))) return rc;
        m->loss_hist = h;
        m->hist_cap = steps;
        if (m->graph) {  // the graph holds the old pointers
            cudaGraphExecDestroy(m->graph);
            m->graph = nullptr;
        }
    }
    GBS_CUDA_TRY(cudaMemcpyAsync(m->lr, lr, sizeof(float) * steps, cudaMemcpyHostToDevice, m->stream));
    GBS_CUDA_TRY(cudaMemsetAsync(m->step + 1, 0, sizeof(long long), m->stream));
    if ((rc = run_input(m, X_dev, batch))) return rc;
    if (!m->graph || m->g_X != X_dev || m->g_T != T_dev || m->g_batch != batch) {
        if (m->graph) {
            cudaGraphExecDestroy(m->graph);
            m->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        GBS_CUDA_TRY(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
        rc = run_forward(m, batch);
        if (!rc) rc = run_backward(m, T_dev, batch, 1, m->loss_hist);
        if (!rc) rc = run_adam(m, nullptr);
        cudaError_t ce = cudaStreamEndCapture(m->stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ce != cudaSuccess) return set_error(GBS_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&m->graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            m->graph = nullptr;
            return set_error(GBS_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
        }
        m->g_X = X_dev;
        m->g_T = T_dev;
        m->g_batch = batch;
    }
    for (int i = 0; i < steps; ++i) GBS_CUDA_TRY(cudaGraphLaunch(m->graph, m->stream));
    if ((rc = check_err(m))) return rc;
    if (loss_hist)
        GBS_CUDA_TRY(cudaMemcpyAsync(loss_hist, m->loss_hist, sizeof(float) * steps,
                                     cudaMemcpyDeviceToHost, m->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return GBS_OK;
}

void gbs_mlp_free(gbs_mlp_t m) { destroy(m); }

}  // extern "C"
