// K2 + K3, BF16 split path: propagation alpha' = T alpha, beta' = T* beta
// ("Applications to GBS") on the tcgen05 tensor cores, fused with the
// occupation epilogue n'_i = alpha'_i beta'_i and its sum over the tile's
// output modes.
//
// GEMM: C = A B^T with A = [Re T_i.; Im T_i.] (rows interleaved per output
// mode, 2M x N) and B = per 128-trajectory tile [alpha rows; beta rows]
// (256 x N), both K-major BF16.  FP32-level accuracy comes from splitting
// A = A0 + A1 + A2 and B = B0 + B1 + B2 into BF16 planes and summing the
// products A_i B_j with i + j <= 1 (3 products) or i + j <= 2 (6 products)
// (the split-precision pattern, e.g. Henry, Tang, Heinecke, "Leveraging the
// bfloat16 artificial intelligence datatype for higher-precision
// computations", ARITH 2019).
//
// Accumulator promotion: the tensor core's FP32 accumulation truncates each
// MMA's result, a bias of ~1 ulp of the running sum per instruction that
// grows linearly with the number of MMAs chained into one accumulator
// (measured: ~2^-24 of the amplitude scale per instruction).  So each
// 64-wide K segment's products go into a fresh TMEM accumulator, and the
// epilogue warps add every segment's result into FP32
// registers with round-to-nearest (the promotion interval idea of, e.g.,
// the DeepSeek-V3 report's FP8 GEMMs).  Two TMEM buffers alternate per
// segment of 64 K, so the MMAs of segment s+1 overlap the promotion of s.
//
// Kernel structure (one CTA per SM, clusters of 2 CTAs, persistent over tile
// groups, 320 threads).  The CTAs of a cluster compute mode tiles 2g, 2g+1
// of the same trajectory tile: each loads its own A planes and half of the
// B planes, which TMA multicasts into both CTAs' shared memory, so the L2
// delivers each B tile once per pair.  A stage is refilled only after
// every CTA's MMAs released it (their commits arrive on all CTAs' barriers).
//   warp 0      TMA producer: per 32-wide K block one box per BF16 plane used
//               (A: 32 x 128, B: 32 x 256, 64-byte swizzle), every plane loaded
//               once per K block, into a 4-stage (3 products) or 3-stage
//               (6 products) shared-memory ring;
//   warp 1      allocates 512 TMEM columns; one thread issues
//               tcgen05.mma M=128 N=256 K=16, per segment of two K blocks the
//               correction products first and A0 B0 last, into the segment's
//               buffer;
//   warps 2..9  epilogue: warp w reads TMEM lanes 32 (w mod 4).. (its A rows)
//               and half (w - 2) / 4 of the tile's trajectories: running
//               sums of 64 alpha' and 64 beta' columns per thread.  After the
//               last K block: occupations, butterfly transpose-reduction over
//               the 32 lanes, then the 4 lane quarters in a fixed order -> one
//               n_S partial per (mode tile, trajectory).  alpha', beta' never
//               leave the SM.
// Every mbarrier wait is bounded; on a timeout the kernel raises an error
// flag, drains its own TMA loads and MMAs, frees TMEM and returns.
#include "gbs_internal.cuh"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>

#include <algorithm>

namespace gbs {

struct TcPlan {
    CUtensorMap mapA[3];
    CUtensorMap mapB[3];
    int P = 0;
    int ia[6] = {0, 0, 0, 0, 0, 0};
    int ib[6] = {0, 0, 0, 0, 0, 0};
    int64_t rowsB = 0;
    bool attr_set = false;
};

namespace {

// One pipeline stage holds every BF16 plane of one 32-wide K block: A planes
// of 128 rows x 64 B, B planes of 256 rows x 64 B (64-byte swizzle).
template <int P>
struct Cfg {
    static constexpr int kPlanes = (P == 3) ? 2 : 3;  // planes of A and of B used
    static constexpr int kAPlane = 128 * 64;
    static constexpr int kBPlane = 256 * 64;
    static constexpr int kStageBytes = kPlanes * (kAPlane + kBPlane);
    static constexpr int kStages = (P == 3) ? 4 : 3;
};
constexpr int kBarBytes = 1024;
constexpr int kRedBytes = 4 * 128 * 2 * 4;  // float [4 quarters][128 trajectories][re, im]
template <int P>
constexpr int smem_bytes() {
    return 1024 + Cfg<P>::kStages * Cfg<P>::kStageBytes + kBarBytes + kRedBytes;
}
constexpr uint32_t kIdesc = ptx::idesc_bf16_f32(128, 256);
constexpr int kCluster = 2;  // CTAs sharing one trajectory tile's B operand
constexpr uint16_t kClusterMask = (1u << kCluster) - 1;
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = 64 + kEpiThreads;

struct TcParams {
    int KB;  // 32-wide K blocks
    int P;   // products
    int ia[6];
    int ib[6];
    int mtiles;
    int stiles;
    int64_t count;
    int64_t ld_part;
    double2 *nS_part;
    unsigned long long *err;
};

__device__ __forceinline__ void named_bar_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Butterfly transpose-reduction of 32 values per lane over the warp: on
// return v[0] of lane l holds the sum over all lanes of input value l.
__device__ __forceinline__ void warp_transpose_reduce32(float (&v)[32], int lane) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const bool up = (lane & 16) != 0;
        const float send = up ? v[i] : v[i + 16];
        const float keep = up ? v[i + 16] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool up = (lane & 8) != 0;
        const float send = up ? v[i] : v[i + 8];
        const float keep = up ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = (lane & 4) != 0;
        const float send = up ? v[i] : v[i + 4];
        const float keep = up ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = (lane & 2) != 0;
        const float send = up ? v[i] : v[i + 2];
        const float keep = up ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    {
        const bool up = (lane & 1) != 0;
        const float send = up ? v[0] : v[1];
        const float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
    }
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
              const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB0,
              const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2,
              const TcParams p) {
    using C = Cfg<P>;
    constexpr int kStages = C::kStages;
    constexpr int kPl = C::kPlanes;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    // stage s: [A plane 0..kPl-1][B plane 0..kPl-1]
    auto a_tile = [&](int stage, int plane) {
        return smem + stage * C::kStageBytes + plane * C::kAPlane;
    };
    auto b_tile = [&](int stage, int plane) {
        return smem + stage * C::kStageBytes + kPl * C::kAPlane + plane * C::kBPlane;
    };
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * C::kStageBytes);
    uint64_t *full = bars;
    uint64_t *empty = bars + kStages;
    uint64_t *tfull = bars + 2 * kStages;
    uint64_t *tempty = bars + 2 * kStages + 2;
    uint64_t *drain = bars + 2 * kStages + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 5);
    float *red = reinterpret_cast<float *>(smem + kStages * C::kStageBytes + kBarBytes);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    volatile unsigned long long *err = p.err;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(ptx::smem_u32(&full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&empty[s]), kCluster);  // released by every CTA of the cluster
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(ptx::smem_u32(&tfull[b]), 1);
            ptx::mbar_init(ptx::smem_u32(&tempty[b]), kEpiThreads);
        }
        ptx::mbar_init(ptx::smem_u32(drain), 1);
        ptx::fence_barrier_init();
        ptx::prefetch_tmap(&mA0);
        ptx::prefetch_tmap(&mA1);
        ptx::prefetch_tmap(&mB0);
        ptx::prefetch_tmap(&mB1);
        if (kPl > 2) {
            ptx::prefetch_tmap(&mA2);
            ptx::prefetch_tmap(&mB2);
        }
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(tmem_slot), 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::cluster_sync();  // the peer's barriers exist before anything is multicast to them
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    // A cluster of kCluster CTAs works on a tile group: the same trajectory
    // tile, mode tiles kCluster*g + rank; each CTA loads 1/kCluster of the B
    // rows and multicasts them to all.
    const uint32_t rank = ptx::cluster_ctarank();
    const int cluster = blockIdx.x / kCluster;
    const int nclusters = gridDim.x / kCluster;
    const int mpairs = (p.mtiles + kCluster - 1) / kCluster;
    const int ntiles = mpairs * p.stiles;
    const int nseg = (p.KB + 1) / 2;  // promotion segments of two 32-wide K blocks

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------- TMA producer
            int stage = 0;
            uint32_t phase = 0;
            uint32_t used = 0, last_phase = 0;  // stages ever filled, parity of their last fill
            bool ok = true;
            for (int tile = cluster; ok && tile < ntiles; tile += nclusters) {
                const int mt = kCluster * (tile % mpairs) + (int)rank;  // >= p.mtiles: A reads zeros
                const int st = tile / mpairs;
                for (int kb = 0; kb < p.KB; ++kb) {
                    if (!ptx::mbar_wait(ptx::smem_u32(&empty[stage]), phase ^ 1u, err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = ptx::smem_u32(&full[stage]);
                    ptx::mbar_arrive_expect_tx(fb, C::kStageBytes);
                    ptx::tma_load_2d(ptx::smem_u32(a_tile(stage, 0)), &mA0, fb, kb * 32, mt * 128);
                    ptx::tma_load_2d(ptx::smem_u32(a_tile(stage, 1)), &mA1, fb, kb * 32, mt * 128);
                    if (kPl > 2)
                        ptx::tma_load_2d(ptx::smem_u32(a_tile(stage, 2)), &mA2, fb, kb * 32,
                                         mt * 128);
                    const int brow = st * 256 + (int)rank * (256 / kCluster);
                    const uint32_t bpart = rank * (uint32_t)(C::kBPlane / kCluster);
                    ptx::tma_load_2d_mc(ptx::smem_u32(b_tile(stage, 0)) + bpart, &mB0, fb, kb * 32,
                                        brow, kClusterMask);
                    ptx::tma_load_2d_mc(ptx::smem_u32(b_tile(stage, 1)) + bpart, &mB1, fb, kb * 32,
                                        brow, kClusterMask);
                    if (kPl > 2)
                        ptx::tma_load_2d_mc(ptx::smem_u32(b_tile(stage, 2)) + bpart, &mB2, fb,
                                            kb * 32, brow, kClusterMask);
                    used |= 1u << stage;
                    last_phase = (last_phase & ~(1u << stage)) | (phase << stage);
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            // drain: every load issued by this thread has landed, and both
            // CTAs' MMAs have released every stage (their arrivals are in)
            for (int s = 0; s < kStages; ++s)
                if (used & (1u << s)) {
                    ptx::mbar_wait(ptx::smem_u32(&full[s]), (last_phase >> s) & 1u, err,
                                   200000000ull);
                    ptx::mbar_wait(ptx::smem_u32(&empty[s]), (last_phase >> s) & 1u, err,
                                   200000000ull);
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------- MMA issuer
            // Per segment (two K blocks): the correction products of both
            // blocks first, then A0 B0 of both, into a fresh accumulator.
            int stage = 0;
            uint32_t phase = 0;
            uint32_t seg = 0;  // segments issued so far (selects the TMEM buffer)
            bool ok = true;
            for (int tile = cluster; ok && tile < ntiles; tile += nclusters) {
                for (int sg = 0; ok && sg < nseg; ++sg, ++seg) {
                    const uint32_t b = seg & 1u;
                    if (!ptx::mbar_wait(ptx::smem_u32(&tempty[b]), ((seg >> 1) & 1u) ^ 1u, err)) {
                        ok = false;
                        break;
                    }
                    const int nst = (2 * sg + 1 < p.KB) ? 2 : 1;
                    int stg[2];
                    stg[0] = stage;
                    stg[1] = (stage + 1 == kStages) ? 0 : stage + 1;
                    for (int q = 0; q < nst; ++q) {
                        // stage stg[q] has fill parity phase (q = 0) or, after a wrap, phase ^ 1
                        const uint32_t par = (q == 1 && stg[1] == 0) ? (phase ^ 1u) : phase;
                        if (!ptx::mbar_wait(ptx::smem_u32(&full[stg[q]]), par, err)) {
                            ok = false;
                            break;
                        }
                    }
                    if (!ok) break;
                    ptx::tc_fence_after();
                    const uint32_t d = tmem_base + b * 256u;
                    uint32_t acc = 0u;
                    for (int pr = 0; pr < P; ++pr) {
                        for (int q = 0; q < nst; ++q) {
                            const uint32_t a0 = ptx::smem_u32(a_tile(stg[q], p.ia[pr]));
                            const uint32_t b0 = ptx::smem_u32(b_tile(stg[q], p.ib[pr]));
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                ptx::mma_bf16(d, ptx::desc_k_sw64(a0 + kk * 32),
                                              ptx::desc_k_sw64(b0 + kk * 32), kIdesc, acc);
                                acc = 1u;
                            }
                        }
                    }
                    // the stage is free once every CTA's MMAs have read it
                    for (int q = 0; q < nst; ++q)
                        ptx::mma_commit_mc(ptx::smem_u32(&empty[stg[q]]), kClusterMask);
                    ptx::mma_commit(ptx::smem_u32(&tfull[b]));
                    for (int q = 0; q < nst; ++q) {
                        if (++stage == kStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            // drain: all MMAs issued by this thread have completed
            ptx::mma_commit(ptx::smem_u32(drain));
            ptx::mbar_wait(ptx::smem_u32(drain), 0u, err, 200000000ull);
        }
    } else {
        // -------------------------------------------------------- epilogue
        const int quarter = warp & 3;        // TMEM lanes this warp may access
        const int half = (warp - 2) >> 2;    // which 64 trajectories of the tile
        const int row = quarter * 32 + lane; // A row of the tile = TMEM lane
        const bool im_row = (row & 1) != 0;  // odd A rows hold Im T_i.
        const int et = threadIdx.x - 64;     // 0..255
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        uint32_t seg = 0;
        for (int tile = cluster; tile < ntiles; tile += nclusters) {
            const int mt = kCluster * (tile % mpairs) + (int)rank;
            const int st = tile / mpairs;
            float ra[64], rb[64];  // running alpha', beta' parts of this row
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                ra[i] = 0.0f;
                rb[i] = 0.0f;
            }
            for (int sg = 0; sg < nseg; ++sg, ++seg) {
                const uint32_t b = seg & 1u;
                // on a timeout every epilogue thread keeps going (without
                // waiting) so that all of them reach the same barriers
                ptx::mbar_wait(ptx::smem_u32(&tfull[b]), (seg >> 1) & 1u, err);
                ptx::tc_fence_after();
                const uint32_t tb = lane_base + b * 256u + (uint32_t)(half * 64);
                float t[32];
                ptx::tmem_ld32(tb, t);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 32; ++i) ra[i] += t[i];
                ptx::tmem_ld32(tb + 32u, t);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 32; ++i) ra[32 + i] += t[i];
                ptx::tmem_ld32(tb + 128u, t);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 32; ++i) rb[i] += t[i];
                ptx::tmem_ld32(tb + 160u, t);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 32; ++i) rb[32 + i] += t[i];
                ptx::tc_fence_before();
                ptx::mbar_arrive(ptx::smem_u32(&tempty[b]));
            }
            // occupations of this row for the thread's 64 trajectories, in
            // groups of 16: real part a*b from the own row, imaginary part with
            // the partner row (Re <-> Im of the same mode, lane ^ 1)
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                float v[32];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float a = ra[g * 16 + q];
                    const float bb = rb[g * 16 + q];
                    const float pb = __shfl_xor_sync(0xffffffffu, bb, 1);
                    v[2 * q] = a * bb;
                    v[2 * q + 1] = im_row ? a * pb : -a * pb;
                }
                warp_transpose_reduce32(v, lane);
                const int traj = half * 64 + g * 16 + (lane >> 1);
                red[(quarter * 128 + traj) * 2 + (lane & 1)] = v[0];
            }
            named_bar_sync(1, kEpiThreads);
            if (et < 128) {
                double re = 0.0, im = 0.0;
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    re += (double)red[(w * 128 + et) * 2];
                    im += (double)red[(w * 128 + et) * 2 + 1];
                }
                const int64_t s = (int64_t)st * 128 + et;
                if (s < p.count && mt < p.mtiles)
                    p.nS_part[(size_t)mt * p.ld_part + s] = make_double2(re, im);
            }
            named_bar_sync(1, kEpiThreads);
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    // no multicast or remote arrive from the peer is in flight past this point
    ptx::cluster_sync();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, 512);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

int encode_2d(CUtensorMap *map, void *base, uint64_t inner, uint64_t rows, uint64_t row_bytes,
              uint32_t box_inner, uint32_t box_rows) {
    // box_inner = 32 bf16 = 64 bytes per row: the 64-byte swizzle
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc) return set_error(GBS_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(GBS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GBS_OK;
}

}  // namespace

int tc_plan_create(gbs_net *net) {
    TcPlan *plan = new (std::nothrow) TcPlan();
    if (!plan) return set_error(GBS_ENOMEM, "host allocation failed");
    net->tc = plan;
    const size_t planeA = (size_t)net->rowsA * net->ldK;
    const int64_t tiles = (net->chunk + kTcTileSamples - 1) / kTcTileSamples;
    plan->rowsB = tiles * 256;
    const size_t planeB = (size_t)plan->rowsB * net->ldK;
    int rc;
    for (int q = 0; q < 3; ++q) {
        if ((rc = encode_2d(&plan->mapA[q], net->d_A + q * planeA, (uint64_t)net->N,
                            (uint64_t)net->rowsA, (uint64_t)net->ldK * 2, 32, 256 / kCluster)))
            return rc;
        __nv_bfloat16 *bbase = static_cast<__nv_bfloat16 *>(net->d_B) +
                               (q < net->planesB ? q : 0) * planeB;
        if ((rc = encode_2d(&plan->mapB[q], bbase, (uint64_t)net->N, (uint64_t)plan->rowsB,
                            (uint64_t)net->ldK * 2, 32, 256 / kCluster)))
            return rc;
    }
    // products A_i B_j with i + j <= 1 (3) or <= 2 (6), issued smallest
    // first: the correction products accumulate while the accumulator is
    // small, and only the 4 MMAs of the dominant A0 B0 product truncate at
    // the full magnitude of the K block's sum
    const int ia3[3] = {0, 1, 0}, ib3[3] = {1, 0, 0};
    const int ia6[6] = {1, 0, 2, 0, 1, 0}, ib6[6] = {1, 2, 0, 1, 0, 0};
    plan->P = (net->precision == GBS_BF16X3) ? 3 : 6;
    for (int q = 0; q < plan->P; ++q) {
        plan->ia[q] = plan->P == 3 ? ia3[q] : ia6[q];
        plan->ib[q] = plan->P == 3 ? ib3[q] : ib6[q];
    }
    return GBS_OK;
}

void tc_plan_destroy(gbs_net *net) {
    delete net->tc;
    net->tc = nullptr;
}

int launch_gemm_tc(gbs_net *net, int64_t count) {
    if (count <= 0) return GBS_OK;
    TcPlan *plan = net->tc;
    if (!plan) return set_error(GBS_EINVAL, "no tensor-core plan");
    if (!plan->attr_set) {
        GBS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<3>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          smem_bytes<3>()));
        GBS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<6>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          smem_bytes<6>()));
        plan->attr_set = true;
    }
    TcParams p;
    p.KB = (net->N + 31) / 32;
    p.P = plan->P;
    for (int q = 0; q < 6; ++q) {
        p.ia[q] = plan->ia[q];
        p.ib[q] = plan->ib[q];
    }
    p.mtiles = net->mtiles;
    p.stiles = (int)((count + kTcTileSamples - 1) / kTcTileSamples);
    p.count = count;
    p.ld_part = net->chunk;
    p.nS_part = net->d_nS_part;
    p.err = net->d_flags + 1;
    const int64_t ntiles = (int64_t)((p.mtiles + kCluster - 1) / kCluster) * p.stiles;
    const int clusters = (int)std::min<int64_t>(ntiles, net->sm_count / kCluster);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCluster * clusters);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = plan->P == 3 ? smem_bytes<3>() : smem_bytes<6>();
    cfg.stream = net->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t le;
    if (plan->P == 3)
        le = cudaLaunchKernelEx(&cfg, k_gemm_tc<3>, plan->mapA[0], plan->mapA[1], plan->mapA[2],
                                plan->mapB[0], plan->mapB[1], plan->mapB[2], p);
    else
        le = cudaLaunchKernelEx(&cfg, k_gemm_tc<6>, plan->mapA[0], plan->mapA[1], plan->mapA[2],
                                plan->mapB[0], plan->mapB[1], plan->mapB[2], p);
    if (le != cudaSuccess)
        return set_error(GBS_ECUDA, "cluster launch of the GEMM failed: %s", cudaGetErrorString(le));
    GBS_LAUNCH_CHECK();
    return GBS_OK;
}

}  // namespace gbs
