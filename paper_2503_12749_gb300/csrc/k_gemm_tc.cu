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
// (measured: ~2^-24 of the amplitude scale per instruction).  So each K
// segment's products (seg_blocks<P>() blocks of 32 K) go into a fresh TMEM
// accumulator, and the epilogue warps add every segment's result into FP32
// registers with round-to-nearest (the promotion interval idea of, e.g.,
// the DeepSeek-V3 report's FP8 GEMMs).  Two TMEM buffers alternate per
// segment, so the MMAs of segment s+1 overlap the promotion of s.
//
// A tile is one 64-mode tile (128 A rows) times one 128-trajectory tile
// (256 B rows).  Kernel structure (persistent over tiles, one CTA per SM,
// 320 threads):
//   warp 0      TMA producer: per 32-wide K block one box per BF16 plane used
//               (A: 32 x 128, B: 32 x 256, 64-byte swizzle; the operands are
//               stored K-blocked, [K/32][rows][32], so each box is one
//               contiguous run of 8 or 16 KB and no row fetch moves unused
//               bytes), every plane loaded once per K block, into a
//               multi-stage shared-memory ring;
//   warp 1      allocates 512 TMEM columns; one thread issues
//               tcgen05.mma M=128 N=256 K=16 into the segment's buffer,
//               block by block as the stages land, the correction products
//               first and A0 B0 last (3 products: A1 B0, A0 B1, A0 B0),
//               releasing each stage at once;
//   warps 2..9  epilogue: warp w reads TMEM lanes 32 (w mod 4).. (its A rows)
//               and half (w - 2) / 4 of the tile's trajectories: running
//               sums of 64 alpha' and 64 beta' columns per thread (packed
//               FP32x2 additions, round to nearest per element).  After the
//               last K block: occupations, butterfly transpose-reduction over
//               the 32 lanes, then the 4 lane quarters in a fixed order -> one
//               n_S partial per (mode tile, trajectory).  alpha', beta' never
//               leave the SM.  On request (moments and marginals) the
//               epilogue also writes every n'_i: with 3 products each warp
//               stages its 32 x 16 values in shared memory and stores rows
//               of 64 bytes, 8 rows per instruction.
// CTA pairs (cta_group::2; clusters of 2 CTAs on the two SMs of a pair):
// the pair computes mode tiles 2g and 2g+1 of one trajectory tile as one
// M = 256 MMA issued by the pair's first CTA.  Each CTA loads its own A
// tile (128 rows) and one half of the tile's B rows (the 128 alpha rows in
// the first CTA, the 128 beta rows in the second) into its own shared
// memory, and the pair's MMA reads B from both: every B byte crosses from
// L2 to shared memory once per pair, and every load has one destination
// (its own CTA).  Both CTAs' loads complete on the first CTA's stage barrier;
// the first CTA's MMA commits arrive on the stage-free and accumulator-full
// barriers of both CTAs; the epilogue warps of both CTAs arrive on the first
// CTA's accumulator-free barrier.  Each CTA's TMEM then holds its own 128
// rows x 256 columns, so the epilogue is the same in both.
// Tile order (closed-form tiles of one network): bands of `band` mode-tile
// groups (a group = the 1 or 2 mode tiles one CTA or pair computes); within
// a band the trajectory tiles in order, the band's groups fastest.  A wave
// of resident CTAs then shares each A tile among about (units / band)
// trajectory tiles and each B tile among `band` groups, and the next wave of
// the band reads the same A tiles again (from L2 while the band fits); a
// band at least the number of groups is the plain order (every mode tile of
// one trajectory tile side by side), which streams all of A through L2 once
// per wave.
// Sampling variant (3 products, 512 threads): warps 4..11 are the
// epilogue, and warps 2, 3, 12..15 run the BF16 sampler (sampler_dev.cuh)
// on the NEXT chunk's trajectories (of the one network, or of several
// networks of a batch round taken as one list), into the second sample
// operand, while the tensor cores work on this one: the sampler is
// issue-bound and the GEMM leaves most issue slots idle.  Registers: launched at 128 per thread
// (65,536 per CTA), the two epilogue warpgroups take 168 each and the other
// two give up theirs down to 88 (setmaxnreg; 2 x 128 x 168 + 2 x 128 x 88 =
// 65,536); the host launches this variant only after checking that the
// kernel was built with exactly 128 registers per thread.
// Every mbarrier wait is bounded; on a timeout the kernel raises an error
// flag, waits (bounded) for its own TMA loads and MMAs, frees TMEM and
// returns; the host then rejects the launch's results.
#include "gbs_internal.cuh"
#include "tc_ptx.cuh"
#include "sampler_dev.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace gbs {

struct TcPlan {
    GemmNetDesc desc;               // host copy
    GemmNetDesc *d_desc = nullptr;  // device copy (single-network launches)
    GemmNetDesc desc_alt;           // the same over the second sample operand
    GemmNetDesc *d_desc_alt = nullptr;
    int P = 0;
    // tile configuration of the plain launches ([0]) and of the launches
    // that also sample the next chunk ([1]); pair 0 = pick by the autotuner
    GemmCfg cfg[2];
    bool forced = false;            // set by gbs_set_gemm_config
    unsigned int *d_sync = nullptr; // wave-alignment counter of this network's launches
};

namespace {

// One pipeline stage holds every BF16 plane of one 32-wide K block: A planes
// of 128 rows x 64 B, B planes of the CTA's B rows (256, or 128 in a pair)
// x 64 B (64-byte swizzle).
template <int P, int kPair>
struct Cfg {
    static constexpr int kPlanes = (P == 3) ? 2 : 3;  // planes of A and of B used
    static constexpr int kAPlane = 128 * 64;
    static constexpr int kBPlane = (256 / kPair) * 64;
    static constexpr int kStageBytes = kPlanes * (kAPlane + kBPlane);
    // the deepest ring that fits in shared memory (the default); the
    // autotuners also time a ring one stage shallower
    static constexpr int kStages = (P == 3) ? (kPair == 1 ? 4 : 6) : (kPair == 1 ? 3 : 4);
};
constexpr int kBarBytes = 1024;
constexpr int kEpiWarpsFwd = 8;  // epilogue warps (kEpiWarps below)
constexpr int kRedBytes = 4 * 128 * 2 * 4;  // float [4 quarters][128 trajectories][re, im]
// Occupation staging (3 products only; the 6-product ring leaves no room):
// per epilogue warp 32 rows (Re/Im plane x 16 modes) of 16 trajectories,
// rows padded to 20 floats so that the row-wise float4 writes are free of
// bank conflicts.
constexpr int kOccRow = 20;
constexpr int kOccWarpFloats = 32 * kOccRow;
template <int P>
constexpr int occ_stage_bytes() {
    return P == 3 ? kEpiWarpsFwd * kOccWarpFloats * 4 : 0;
}
template <int P, int kPair, int kSt = Cfg<P, kPair>::kStages>
constexpr int smem_bytes() {
    return 1024 + kSt * Cfg<P, kPair>::kStageBytes + kBarBytes + kRedBytes + occ_stage_bytes<P>();
}
static_assert(smem_bytes<3, 1>() <= 227 * 1024, "shared memory of the 3-product GEMM");
static_assert(smem_bytes<6, 1>() <= 227 * 1024, "shared memory of the 6-product GEMM");
static_assert(smem_bytes<3, 2>() <= 227 * 1024, "shared memory of the 3-product pair GEMM");
static_assert(smem_bytes<6, 2>() <= 227 * 1024, "shared memory of the 6-product pair GEMM");
template <int kPair>
constexpr uint32_t idesc() {
    return ptx::idesc_bf16_f32(128 * kPair, 256);
}
constexpr int kEpiWarps = kEpiWarpsFwd;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = 64 + kEpiThreads;
// sampling variants: kSW warpgroups of sampler warps after the epilogue
// (kSW = 0: the plain GEMM)
template <int kSW>
__host__ __device__ constexpr int threads_of() {
    return kSW ? 128 * (3 + kSW) : kThreads;
}
template <int kSW>
__host__ __device__ constexpr int epi_warp0() {
    return kSW ? 4 : 2;
}
template <int kSW>
__host__ __device__ constexpr int sampler_warps() {
    return kSW ? 2 + 4 * kSW : 0;
}
// registers per thread at launch (the CTA's 65,536 at most, in units of 8)
template <int kSW>
__host__ __device__ constexpr int regs_launch() {
    return (65536 / threads_of<kSW>()) / 8 * 8;
}
constexpr int kRegsEpi = 168;
// what the warpgroups other than the two epilogue ones keep
template <int kSW>
__host__ __device__ constexpr int regs_rest() {
    return (threads_of<kSW>() * regs_launch<kSW>() - 256 * kRegsEpi) / (threads_of<kSW>() - 256) /
           8 * 8;
}
static_assert(regs_launch<1>() == 128 && regs_rest<1>() == 88, "register split, 6 sampler warps");
static_assert(regs_launch<2>() == 96 && regs_rest<2>() == 48, "register split, 10 sampler warps");
static_assert(256 * kRegsEpi + (threads_of<1>() - 256) * regs_rest<1>() <=
                  threads_of<1>() * regs_launch<1>(), "register pool, 6 sampler warps");
static_assert(256 * kRegsEpi + (threads_of<2>() - 256) * regs_rest<2>() <=
                  threads_of<2>() * regs_launch<2>(), "register pool, 10 sampler warps");
// The sampling GEMM's sampler warps: kSampWG warpgroups after the
// epilogue, plus warps 2 and 3 of warpgroup 0; within a CTA's range of
// trajectories the warps take fixed strides.  The sampler's issue slots come
// out of the epilogue's, so the fewest warps that still finish within the
// GEMM are best (measured at N = M = 1000: 4 warps leave the sampler as the
// launch's tail, 10 warps, or a shared counter that keeps all 6 busy to the
// end, lengthen the launch).
constexpr int kSampWG = 1;
constexpr int kSampWarpsUsed = 4 * kSampWG + 2;
// K blocks (of 32) per accumulator promotion segment.  The tensor core
// truncates each MMA's FP32 result, which shrinks the magnitude of the
// accumulated value by about half an ulp for every MMA that lands on an
// accumulator already at full magnitude; the promoted sums inherit that
// relative bias (it is linear in the values), so n_S comes out low by a
// factor 1 - 2c, and the longer the segment, the more MMAs land on a full
// accumulator (each K block's products are issued with the corrections
// first and A0 B0 last).  Measured on lossless networks (n_S = n exactly),
// (n - n_S) / n with 3 products = 0.9-1.2e-7 (1-block segments), 2.5e-7
// (2), 3.8-4.2e-7 (3), 5.8-6.0e-7 (4).  Short segments cost time: the MMAs
// of one segment must outlast the promotion of the previous one, which
// holds from 3 blocks on (m8000 GEMM ms per step x median SM MHz / 10^6:
// 2 blocks 1.53, 3 blocks 1.39, 4 blocks 1.38; m1000 GEMM 15.3-15.6, 14.40,
// 14.34 ms per step; 1 block 14 % slower than 2).  The 3-product split takes
// 3-block segments
// (its bias moves P(m) by about 0.15 sigma at the named workloads' sizes);
// the 6-product split, the accuracy mode, promotes every K block.
// Longest wait of a producer at the wave alignment (keep_a bit 8): a tile
// takes hundreds of microseconds where the alignment pays, and the CTAs of a
// wave arrive within a few of each other.
constexpr uint64_t kAlignWaitNs = 50000;

template <int P>
constexpr int seg_blocks() {
    return P == 3 ? 3 : 1;
}

// A tile of the grouped GEMM: which network, which mode tile (of this CTA),
// which 128-trajectory tile.
struct TileRef {
    const GemmNetDesc *d;
    int mt;  // this CTA's mode tile (may be >= mtiles: then A reads zeros, nothing is written)
    int st;
    int64_t count;
};

// Tile t of a launch.  Listed tiles: {network, group, trajectory tile}.
// Closed-form tiles of one network: bands of `band` groups (module
// comment), a group being kPair consecutive mode tiles; CTA `rank` of the
// pair takes mode tile kPair * group + rank.
template <int kPair>
__device__ __forceinline__ TileRef decode_tile(int t, const GemmNetDesc *nets, const int4 *tiles,
                                               int64_t count0, int band, uint32_t rank) {
    TileRef r;
    int g;
    if (tiles) {
        const int4 e = tiles[t];
        r.d = nets + e.x;
        g = e.y;
        r.st = e.z;
        r.count = r.d->count;
    } else {
        r.d = nets;
        r.count = count0;
        const int groups = (nets->mtiles + kPair - 1) / kPair;
        if (band <= 0 || band >= groups) {
            g = t % groups;
            r.st = t / groups;
        } else {
            const int stiles = (int)((count0 + kTcTileSamples - 1) / kTcTileSamples);
            const int per = band * stiles;
            const int bi = t / per;
            const int rem = t - bi * per;
            const int bw = min(band, groups - bi * band);
            g = bi * band + rem % bw;
            r.st = rem / bw;
        }
    }
    r.mt = kPair * g + (int)rank;
    return r;
}

// a0 += b0, a1 += b1 as one packed FP32x2 addition (round to nearest per
// element, the same results as two scalar additions)
__device__ __forceinline__ void add_f32x2(float &a0, float &a1, float b0, float b1) {
    asm("{\n"
        ".reg .b64 x, y;\n"
        "mov.b64 x, {%0, %1};\n"
        "mov.b64 y, {%2, %3};\n"
        "add.rn.f32x2 x, x, y;\n"
        "mov.b64 {%0, %1}, x;\n"
        "}\n"
        : "+f"(a0), "+f"(a1)
        : "f"(b0), "f"(b1));
}

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

template <int P, int kPair, int kSW, int kSt = Cfg<P, kPair>::kStages>
__global__ void __launch_bounds__(threads_of<kSW>(), 1)
    k_gemm_tc(const GemmNetDesc *__restrict__ nets, const int4 *__restrict__ tiles, int ntiles,
              int64_t count0, int band, int keep_a, uint64_t wait_ns,
              unsigned long long *err_ptr, OccOut occ, const SampleJobs sj) {
    static_assert(kSW == 0 || P == 3, "the sampling variant runs the 3-product GEMM");
    static_assert(kPair == 1 || kPair == 2, "one CTA or a CTA pair per tile group");
    using C = Cfg<P, kPair>;
    static_assert(kSt >= 2 && kSt <= C::kStages, "ring of 2 .. kStages stages");
    constexpr int kE0 = epi_warp0<kSW>();  // first epilogue warp
    constexpr int kStages = kSt;
    constexpr int kPl = C::kPlanes;
    constexpr uint32_t kIdesc = idesc<kPair>();
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
    uint64_t *never = bars + 2 * kStages + 6;  // no thread ever arrives on it
    float *red = reinterpret_cast<float *>(smem + kStages * C::kStageBytes + kBarBytes);
    float *ostage = reinterpret_cast<float *>(smem + kStages * C::kStageBytes + kBarBytes + kRedBytes);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    volatile unsigned long long *err = err_ptr;
    // split products A_i B_j, smallest first, A0 B0 last
    constexpr int kIa3[3] = {0, 1, 0}, kIb3[3] = {1, 0, 0};
    constexpr int kIa6[6] = {1, 0, 2, 0, 1, 0}, kIb6[6] = {1, 2, 0, 1, 0, 0};

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(ptx::smem_u32(&full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(ptx::smem_u32(&tfull[b]), 1);
            // one arrival per epilogue warp of every CTA of the pair
            ptx::mbar_init(ptx::smem_u32(&tempty[b]), kEpiWarps * kPair);
        }
        ptx::mbar_init(ptx::smem_u32(drain), 1);
        ptx::mbar_init(ptx::smem_u32(never), 1);
        ptx::fence_barrier_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc<kPair>(ptx::smem_u32(tmem_slot), 512);
        ptx::tmem_relinquish<kPair>();
    }
    ptx::tc_fence_before();
    __syncthreads();
    // both CTAs' barriers and TMEM columns exist before either signals the other
    if (kPair > 1) ptx::cluster_sync();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    // A pair (kPair = 2) works on tile groups: the same trajectory tile, mode
    // tiles 2g + rank; CTA rank 0 issues the pair's MMAs.
    const uint32_t rank = kPair > 1 ? ptx::cluster_ctarank() : 0u;
    const bool leader = rank == 0u;
    const int unit = blockIdx.x / kPair;
    const int nunits = gridDim.x / kPair;

    auto producer = [&]() {
        if (lane == 0) {
            // ---------------------------------------------------- TMA producer
            int stage = 0;
            uint32_t phase = 0;
            uint32_t used = 0, last_phase = 0;  // stages ever filled, parity of their last fill
            bool ok = true;
            const GemmNetDesc *cur = nullptr;
            // banded order with keep_a: the band's A tiles are read again by
            // every wave of the band, so they are loaded with the evict-last
            // L2 policy (the trajectory tiles, read by one wave only, stay
            // normal).  Whether that pays depends on how much of the L2 the
            // band's A tiles leave to the trajectory tiles: a tuned choice.
            // keep_a bits: 1 = the evict-last policy on a band's A tiles
            // (4: on half of their lines), 2 = the evict-first policy on the
            // trajectory tiles
            const bool keepA = (keep_a & 1) && band > 0 && !tiles;
            const uint64_t polA = (keep_a & 4) ? ptx::policy_evict_last_half()
                                               : ptx::policy_evict_last();
            const bool firstB = (keep_a & 2) && !tiles;
            const uint64_t polB = ptx::policy_evict_first();
            // keep_a bit 8 (single-network launches): before each tile of
            // the full waves after the first, every producer waits (for at
            // most kAlignWaitNs) until all CTAs have issued the previous
            // tile's loads, so that the CTAs of a wave read the A and B tiles
            // they share close together in time, while the L2 still holds
            // them (at m8000 the DRAM traffic falls to a third, and the
            // power it saves raises the clock under the power limit).  A
            // producer whose wait times out (CTAs of the launch that are not
            // resident, e.g. SMs held by another context) stops waiting for
            // the rest of the launch but keeps counting its tiles, so that
            // such a launch loses at most one wait per CTA
            const bool align = (keep_a & 8) && !tiles && nets->wave_sync != nullptr;
            bool waiting = align;
            const int full_waves = ntiles / nunits;
            int j = 0;
            for (int tile = unit; ok && tile < ntiles; tile += nunits, ++j) {
                if (align && j >= 1 && j < full_waves) {
                    atomicAdd(nets->wave_sync, 1u);
                    if (waiting && !ptx::counter_wait_soft(nets->wave_sync, (unsigned)j * gridDim.x,
                                                           kAlignWaitNs))
                        waiting = false;
                }
                const TileRef tr = decode_tile<kPair>(tile, nets, tiles, count0, band, rank);
                const GemmNetDesc *d = tr.d;
                const CUtensorMap *mA[3] = {&d->mapA[0], &d->mapA[1], &d->mapA[2]};
                const CUtensorMap *mB[3] = {&d->mapB[kPair - 1][0], &d->mapB[kPair - 1][1],
                                            &d->mapB[kPair - 1][2]};
                if (d != cur) {
                    for (int q = 0; q < kPl; ++q) {
                        ptx::prefetch_tmap(mA[q]);
                        ptx::prefetch_tmap(mB[q]);
                    }
                    cur = d;
                }
                // this CTA's B rows: the whole tile, or in a pair its half
                const int brow = tr.st * 256 + (int)rank * (256 / kPair);
                for (int kb = 0; kb < d->KB; ++kb) {
                    if (!ptx::mbar_wait(ptx::smem_u32(&empty[stage]), phase ^ 1u, err, wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = ptx::smem_u32(&full[stage]);
                    // operands are K-blocked ([K/32][rows][32]): each box is
                    // one contiguous block of global memory
                    if constexpr (kPair == 1) {
                        ptx::mbar_arrive_expect_tx(fb, C::kStageBytes);
#pragma unroll
                        for (int q = 0; q < kPl; ++q) {
                            if (keepA)
                                ptx::tma_load_3d_hint(ptx::smem_u32(a_tile(stage, q)), mA[q], fb,
                                                      0, tr.mt * 128, kb, polA);
                            else
                                ptx::tma_load_3d(ptx::smem_u32(a_tile(stage, q)), mA[q], fb, 0,
                                                 tr.mt * 128, kb);
                        }
#pragma unroll
                        for (int q = 0; q < kPl; ++q) {
                            if (firstB)
                                ptx::tma_load_3d_hint(ptx::smem_u32(b_tile(stage, q)), mB[q], fb,
                                                      0, brow, kb, polB);
                            else
                                ptx::tma_load_3d(ptx::smem_u32(b_tile(stage, q)), mB[q], fb, 0,
                                                 brow, kb);
                        }
                    } else {
                        // both CTAs' halves of the stage complete on the
                        // first CTA's barrier, which expects them all
                        if (leader) ptx::mbar_arrive_expect_tx(fb, 2 * C::kStageBytes);
                        const uint32_t fb0 = ptx::cluster_addr(fb, 0u);
#pragma unroll
                        for (int q = 0; q < kPl; ++q) {
                            if (keepA)
                                ptx::tma_load_3d_pair_hint(ptx::smem_u32(a_tile(stage, q)), mA[q],
                                                           fb0, 0, tr.mt * 128, kb, polA);
                            else
                                ptx::tma_load_3d_pair(ptx::smem_u32(a_tile(stage, q)), mA[q], fb0,
                                                      0, tr.mt * 128, kb);
                        }
#pragma unroll
                        for (int q = 0; q < kPl; ++q) {
                            if (firstB)
                                ptx::tma_load_3d_pair_hint(ptx::smem_u32(b_tile(stage, q)), mB[q],
                                                           fb0, 0, brow, kb, polB);
                            else
                                ptx::tma_load_3d_pair(ptx::smem_u32(b_tile(stage, q)), mB[q], fb0,
                                                      0, brow, kb);
                        }
                    }
                    used |= 1u << stage;
                    last_phase = (last_phase & ~(1u << stage)) | (phase << stage);
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            // drain.  Normally: every load issued by this thread has landed
            // and the MMAs have released every stage (in a pair the second
            // CTA sees only the releases, which follow its loads' completion
            // on the first CTA's barrier).  After an error (the flag is up and
            // the host rejects the launch) the releases may never come: one
            // CTA waits only for its own loads to land; a pair, whose second
            // CTA cannot see its loads complete, waits a fixed 100 us (a load
            // takes microseconds) before the final cluster barrier.
            bool failed = !ok || *err != 0ull;
            for (int s = 0; !failed && s < kStages; ++s) {
                if (!(used & (1u << s))) continue;
                const uint32_t par = (last_phase >> s) & 1u;
                if (leader && !ptx::mbar_wait(ptx::smem_u32(&full[s]), par, err, 200000000ull))
                    failed = true;
                else if (!ptx::mbar_wait(ptx::smem_u32(&empty[s]), par, err, 200000000ull))
                    failed = true;
            }
            if (failed) {
                if constexpr (kPair == 1) {
                    for (int s = 0; s < kStages; ++s)
                        if (used & (1u << s))
                            ptx::mbar_wait(ptx::smem_u32(&full[s]), (last_phase >> s) & 1u, err,
                                           200000000ull, false);
                } else {
                    const uint64_t t0 = ptx::globaltimer();
                    while (ptx::globaltimer() - t0 < 100000ull) {
                    }
                }
            }
        }
    };
    // the stage-free / accumulator-full commit of the pair's MMAs: on this
    // CTA's barrier and, in a pair, on the same barrier of the second CTA
    auto commit_both = [&](uint64_t *bar) {
        const uint32_t a = ptx::smem_u32(bar);
        if constexpr (kPair == 1) {
            ptx::mma_commit(a);
        } else {
            ptx::mma_commit_pair(a);
            ptx::mma_commit_pair(ptx::cluster_addr(a, 1u));
        }
    };
    auto mma = [&](uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
        if constexpr (kPair == 1)
            ptx::mma_bf16(d, a, b, kIdesc, acc);
        else
            ptx::mma_bf16_pair(d, a, b, kIdesc, acc);
    };
    auto mma_issuer = [&]() {
        if (lane == 0 && leader) {
            // ---------------------------------------------------- MMA issuer
            // Per promotion segment (seg_blocks<P>() K blocks) a fresh
            // accumulator; each K block's products as soon as its stage
            // lands, the correction products first and A0 B0 last, and the
            // stage released right after.
            int stage = 0;
            uint32_t phase = 0;
            uint32_t seg = 0;  // segments issued so far (selects the TMEM buffer)
            bool ok = true;
            // a wait limit of 0 asks for the timeout path itself: the first
            // wait is on a barrier that no thread arrives on, so it gives up
            // (raising the flag) before any MMA is issued
            if (wait_ns == 0ull) ok = ptx::mbar_wait(ptx::smem_u32(never), 0u, err, 0ull);
            for (int tile = unit; ok && tile < ntiles; tile += nunits) {
                const TileRef tr = decode_tile<kPair>(tile, nets, tiles, count0, band, rank);
                const int KB = tr.d->KB;
                constexpr int kSegBlocks = seg_blocks<P>();
                const int nseg = (KB + kSegBlocks - 1) / kSegBlocks;
                for (int sg = 0; ok && sg < nseg; ++sg, ++seg) {
                    const uint32_t b = seg & 1u;
                    // the epilogue warps of both CTAs have read this buffer
                    if (!ptx::mbar_wait(ptx::smem_u32(&tempty[b]), ((seg >> 1) & 1u) ^ 1u, err,
                                        wait_ns)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const int nst = min(kSegBlocks, KB - sg * kSegBlocks);
                    const uint32_t d = tmem_base + b * 256u;
                    uint32_t acc = 0u;
                    for (int q = 0; q < nst; ++q) {
                        if (!ptx::mbar_wait(ptx::smem_u32(&full[stage]), phase, err, wait_ns)) {
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        // the stage's plane descriptors once; the second K16
                        // half is 32 bytes on (2 in the descriptor's 16-byte
                        // address field, which cannot carry: shared addresses
                        // stay below 2^18)
                        uint64_t dA[kPl], dB[kPl];
#pragma unroll
                        for (int pl = 0; pl < kPl; ++pl) {
                            dA[pl] = ptx::desc_k_sw64(ptx::smem_u32(a_tile(stage, pl)));
                            dB[pl] = ptx::desc_k_sw64(ptx::smem_u32(b_tile(stage, pl)));
                        }
#pragma unroll
                        for (int pr = 0; pr < P; ++pr) {
                            const int ia = (P == 3) ? kIa3[pr] : kIa6[pr];
                            const int ib = (P == 3) ? kIb3[pr] : kIb6[pr];
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                mma(d, dA[ia] + 2u * kk, dB[ib] + 2u * kk, acc);
                                acc = 1u;
                            }
                        }
                        // the stage is free once the MMAs have read it
                        commit_both(&empty[stage]);
                        if (++stage == kStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    commit_both(&tfull[b]);
                }
            }
            // drain: all MMAs issued by this thread have completed
            if constexpr (kPair == 1)
                ptx::mma_commit(ptx::smem_u32(drain));
            else
                ptx::mma_commit_pair(ptx::smem_u32(drain));
            // (also after an error: issued MMAs always complete)
            ptx::mbar_wait(ptx::smem_u32(drain), 0u, err, 200000000ull, false);
        }
    };
    auto epilogue = [&]() {
        // -------------------------------------------------------- epilogue
        const int quarter = warp & 3;        // TMEM lanes this warp may access
        const int half = (warp - kE0) >> 2;  // which 64 trajectories of the tile
        const int row = quarter * 32 + lane; // A row of the tile = TMEM lane
        const bool im_row = (row & 1) != 0;  // odd A rows hold Im T_i.
        const int et = threadIdx.x - 32 * kE0;  // 0..255
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        uint32_t seg = 0;
        for (int tile = unit; tile < ntiles; tile += nunits) {
            const TileRef tr = decode_tile<kPair>(tile, nets, tiles, count0, band, rank);
            const int mt = tr.mt;
            const int st = tr.st;
            constexpr int kSegBlocks = seg_blocks<P>();
            const int nseg = (tr.d->KB + kSegBlocks - 1) / kSegBlocks;
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
                ptx::mbar_wait(ptx::smem_u32(&tfull[b]), (seg >> 1) & 1u, err, wait_ns);
                ptx::tc_fence_after();
                const uint32_t tb = lane_base + b * 256u + (uint32_t)(half * 64);
                float t[32];
                ptx::tmem_ld32(tb, t);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 32; i += 2) add_f32x2(ra[i], ra[i + 1], t[i], t[i + 1]);
                ptx::tmem_ld32(tb + 32u, t);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 32; i += 2) add_f32x2(ra[32 + i], ra[33 + i], t[i], t[i + 1]);
                ptx::tmem_ld32(tb + 128u, t);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 32; i += 2) add_f32x2(rb[i], rb[i + 1], t[i], t[i + 1]);
                ptx::tmem_ld32(tb + 160u, t);
                ptx::tmem_ld_wait();
                // the warp's reads are done (the last values are in
                // registers): one arrival per warp on the buffer's free
                // barrier (the first CTA's, in a pair) before the last adds
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    const uint32_t tb_bar = ptx::smem_u32(&tempty[b]);
                    if constexpr (kPair == 1)
                        ptx::mbar_arrive(tb_bar);
                    else
                        ptx::mbar_arrive_remote(ptx::cluster_addr(tb_bar, 0u));
                }
#pragma unroll
                for (int i = 0; i < 32; i += 2) add_f32x2(rb[32 + i], rb[33 + i], t[i], t[i + 1]);
            }
            // occupations of this row for the thread's 64 trajectories, in
            // groups of 16: real part a*b from the own row, imaginary part with
            // the partner row (Re <-> Im of the same mode, lane ^ 1)
            const bool want_occ = occ.p != nullptr && mt < tr.d->mtiles;
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
                if (want_occ) {
                    // per-mode n'_i: the Re row (even lane) completes Re n'_i
                    // with the Im row's a_i b_i, the Im row (odd lane) Im n'_i
                    // with the Re row's -a_r b_i; 16 trajectories per lane
                    const size_t tcol = (size_t)st * 128 + half * 64 + g * 16;
                    float *dst = occ.p + (size_t)(lane & 1) * occ.plane +
                                 (size_t)(mt * 64 + (row >> 1)) * occ.ld + tcol;
                    float *srow = ostage + (warp - kE0) * kOccWarpFloats + lane * kOccRow;
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        float o[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int q = q4 * 4 + u;
                            const float send = im_row ? v[2 * q] : v[2 * q + 1];
                            const float own = im_row ? v[2 * q + 1] : v[2 * q];
                            o[u] = own + __shfl_xor_sync(0xffffffffu, send, 1);
                        }
                        const float4 o4 = make_float4(o[0], o[1], o[2], o[3]);
                        if (P == 3) *reinterpret_cast<float4 *>(srow + q4 * 4) = o4;
                        else __stcs(reinterpret_cast<float4 *>(dst + q4 * 4), o4);
                    }
                    if (P == 3) {
                        // rows of 64 bytes out of the staging area: 4 lanes per
                        // row, 8 rows per store instruction (instead of 32
                        // rows of 16 bytes)
                        __syncwarp();
                        const float *wst = ostage + (warp - kE0) * kOccWarpFloats;
#pragma unroll
                        for (int pass = 0; pass < 4; ++pass) {
                            const int sr = pass * 8 + (lane >> 2);  // producing lane
                            const float4 v4 =
                                *reinterpret_cast<const float4 *>(wst + sr * kOccRow + (lane & 3) * 4);
                            float *d = occ.p + (size_t)(sr & 1) * occ.plane +
                                       (size_t)(mt * 64 + quarter * 16 + (sr >> 1)) * occ.ld + tcol +
                                       (lane & 3) * 4;
                            __stcs(reinterpret_cast<float4 *>(d), v4);  // evict-first in L2
                        }
                        __syncwarp();
                    }
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
                if (s < tr.count && mt < tr.d->mtiles)
                    tr.d->nS_part[(size_t)mt * tr.d->ld_part + s] = make_double2(re, im);
            }
            named_bar_sync(1, kEpiThreads);
        }
    };

    if constexpr (kSW > 0) {
        // The register reallocation comes first in each warpgroup-uniform
        // branch (all warps of a warpgroup execute the same instruction,
        // and it dominates the code that relies on it): warpgroups 1, 2
        // are the epilogue; 0 (producer, MMA issuer, 2 sampler warps) and
        // 3.. (sampler warps) give up registers.
        const int wg = warp >> 2;
        if (wg == 1 || wg == 2) {
            ptx::setmaxnreg_inc<kRegsEpi>();
            epilogue();
        } else {
            ptx::setmaxnreg_dec<regs_rest<kSW>()>();
            if (warp == 0) {
                producer();
            } else if (warp == 1) {
                mma_issuer();
            } else {
                // ---------------------------------------------- sampler warps
                // (2, 3, 12..): the next chunk's operand(s), evict-first
                // stores; each CTA samples a contiguous range of the job
                // list
                const int sw = warp < 4 ? warp - 2 : warp - 10;
                const int64_t total = sj.n ? sj.prefix[sj.n] : sj.one.count;
                const int64_t lo = total * (int64_t)blockIdx.x / gridDim.x;
                const int64_t hi = total * ((int64_t)blockIdx.x + 1) / gridDim.x;
                if (sj.n == 0) {
                    for (int64_t i = lo + sw; i < hi; i += kSampWarpsUsed)
                        samp::sample_trajectory_bf16<true, true>(sj.one, i, lane);
                } else if (lo + sw < hi) {
                    // the job holding list position lo + sw: the last j with
                    // prefix[j] <= lo + sw (binary search), then forward
                    int a = 0, c = sj.n;  // prefix[a] <= pos < prefix[c]
                    const int64_t pos0 = lo + sw;
                    while (c - a > 1) {
                        const int m = (a + c) >> 1;
                        if (sj.prefix[m] <= pos0) a = m;
                        else c = m;
                    }
                    int j = a;
                    SampleJob jb = sj.jobs[j];
                    int64_t base = sj.prefix[j], end = sj.prefix[j + 1];
                    for (int64_t i = pos0; i < hi; i += kSampWarpsUsed) {
                        while (i >= end) {
                            ++j;
                            jb = sj.jobs[j];
                            base = end;
                            end = sj.prefix[j + 1];
                        }
                        samp::sample_trajectory_bf16<true, true>(jb, i - base, lane);
                    }
                }
            }
        }
    } else {
        if (warp == 0)
            producer();
        else if (warp == 1)
            mma_issuer();
        else
            epilogue();
    }

    ptx::tc_fence_before();
    __syncthreads();
    // a pair: the second CTA's TMEM is no longer read or written, and no
    // signal between the two CTAs is pending, before either frees its columns
    if (kPair > 1) ptx::cluster_sync();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc<kPair>(tmem_base, 512);
    }
}

}  // namespace


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

namespace {

std::mutex g_tc_mu;
bool g_attr_set[64] = {};
// (log2 N, log2 M, products) -> (CTA pair, band) chosen by the autotuner
// (log2 N, log2 M, products, sampling launch) -> configuration
std::map<std::tuple<int, int, int, int>, GemmCfg> g_tune;
// Whether the autotuner also times CTA pairs (gbs_set_gemm_config can always
// ask for them).
bool g_pair_autotune = true;

template <int P, int kPair, int kSW, int kSt = Cfg<P, kPair>::kStages>
cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(k_gemm_tc<P, kPair, kSW, kSt>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_bytes<P, kPair, kSt>());
}
// the ring one stage shallower than the deepest (an autotuner candidate)
template <int P, int kPair>
constexpr int shallow_stages() {
    return Cfg<P, kPair>::kStages - 1;
}

int ensure_attrs() {
    int dev = 0;
    GBS_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_tc_mu);
    if (dev >= 0 && dev < 64 && g_attr_set[dev]) return GBS_OK;
    GBS_CUDA_TRY((set_smem_attr<3, 1, 0>()));
    GBS_CUDA_TRY((set_smem_attr<3, 2, 0>()));
    GBS_CUDA_TRY((set_smem_attr<6, 1, 0>()));
    GBS_CUDA_TRY((set_smem_attr<6, 2, 0>()));
    GBS_CUDA_TRY((set_smem_attr<3, 1, kSampWG>()));
    GBS_CUDA_TRY((set_smem_attr<3, 2, kSampWG>()));
    GBS_CUDA_TRY((set_smem_attr<3, 1, 0, shallow_stages<3, 1>()>()));
    GBS_CUDA_TRY((set_smem_attr<3, 2, 0, shallow_stages<3, 2>()>()));
    GBS_CUDA_TRY((set_smem_attr<6, 1, 0, shallow_stages<6, 1>()>()));
    GBS_CUDA_TRY((set_smem_attr<6, 2, 0, shallow_stages<6, 2>()>()));
    GBS_CUDA_TRY((set_smem_attr<3, 1, kSampWG, shallow_stages<3, 1>()>()));
    GBS_CUDA_TRY((set_smem_attr<3, 2, kSampWG, shallow_stages<3, 2>()>()));
    if (dev >= 0 && dev < 64) g_attr_set[dev] = true;
    return GBS_OK;
}

// The sampling variant's register split holds only if every thread starts
// with exactly regs_launch() registers: checked once per process from the
// built kernels' attributes (otherwise the plain GEMM and sampler run).
bool sampling_kernels_ok() {
    static int state = -1;  // -1 unknown, 0 no, 1 yes
    std::lock_guard<std::mutex> lock(g_tc_mu);
    if (state < 0) {
        cudaFuncAttributes a1 = {}, a2 = {};
        constexpr int R = regs_launch<kSampWG>(), T = threads_of<kSampWG>();
        const bool ok = cudaFuncGetAttributes(&a1, k_gemm_tc<3, 1, kSampWG>) == cudaSuccess &&
                        cudaFuncGetAttributes(&a2, k_gemm_tc<3, 2, kSampWG>) == cudaSuccess &&
                        a1.numRegs == R && a2.numRegs == R && a1.maxThreadsPerBlock >= T &&
                        a2.maxThreadsPerBlock >= T;
        if (!ok) cudaGetLastError();
        state = ok ? 1 : 0;
    }
    return state == 1;
}

// The same check for the sampling variants with the shallower ring (the
// batch autotuner leaves them out of its candidates when it fails).
bool shallow_sampling_kernels_ok() {
    static int state = -1;
    std::lock_guard<std::mutex> lock(g_tc_mu);
    if (state < 0) {
        cudaFuncAttributes a1 = {}, a2 = {};
        constexpr int R = regs_launch<kSampWG>(), T = threads_of<kSampWG>();
        const bool ok =
            cudaFuncGetAttributes(&a1, k_gemm_tc<3, 1, kSampWG, shallow_stages<3, 1>()>) ==
                cudaSuccess &&
            cudaFuncGetAttributes(&a2, k_gemm_tc<3, 2, kSampWG, shallow_stages<3, 2>()>) ==
                cudaSuccess &&
            a1.numRegs == R && a2.numRegs == R && a1.maxThreadsPerBlock >= T &&
            a2.maxThreadsPerBlock >= T;
        if (!ok) cudaGetLastError();
        state = ok ? 1 : 0;
    }
    return state == 1;
}

template <int P, int kPair, int kSW, int kSt = Cfg<P, kPair>::kStages>
int launch_variant(cudaStream_t stream, int sm_count, const GemmNetDesc *d_nets, const int4 *d_tiles,
                   int ntiles, int64_t count0, int band, int keep_a, uint64_t wait_ns,
                   unsigned long long *err, OccOut occ, const SampleJobs &jobs) {
    if (ntiles <= 0) return GBS_OK;
    const int units = std::max(1, std::min(ntiles, sm_count / kPair));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kPair * units);
    cfg.blockDim = dim3(threads_of<kSW>());
    cfg.dynamicSmemBytes = smem_bytes<P, kPair, kSt>();
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    int na = 0;
    if (kPair > 1) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = kPair;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    cudaError_t le = cudaLaunchKernelEx(&cfg, k_gemm_tc<P, kPair, kSW, kSt>, d_nets, d_tiles, ntiles,
                                        count0, band, keep_a, wait_ns, err, occ, jobs);
    if (le != cudaSuccess)
        return set_error(GBS_ECUDA, "launch of the GEMM (%d products, %s%s) failed: %s", P,
                         kPair > 1 ? "CTA pairs" : "one CTA per tile", kSW ? ", sampling" : "",
                         cudaGetErrorString(le));
    return GBS_OK;
}

// Tensor map of a K-blocked BF16 plane [KB][rows][32] read in boxes of
// 32 x box_rows x 1 (one K block of box_rows rows: box_rows * 64 contiguous
// bytes), 64-byte swizzle.  Out-of-range rows read as zeros.
int encode_kblocked(CUtensorMap *map, void *base, uint64_t rows, uint64_t KB, uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc) return set_error(GBS_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[3] = {32, rows, KB};
    cuuint64_t strides[2] = {64, rows * 64};
    cuuint32_t box[3] = {32, box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(GBS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GBS_OK;
}

int encode_net_maps(gbs_net *net, void *B, GemmNetDesc &d) {
    const int KB = net->ldK / 32;
    const size_t planeA = (size_t)net->rowsA * net->ldK;
    const int64_t tiles = (net->chunk + kTcTileSamples - 1) / kTcTileSamples;
    const int64_t rowsB = tiles * 256;
    const size_t planeB = (size_t)rowsB * net->ldK;
    int rc;
    for (int q = 0; q < 3; ++q) {
        if ((rc = encode_kblocked(&d.mapA[q], net->d_A + q * planeA, (uint64_t)net->rowsA,
                                  (uint64_t)KB, 128)))
            return rc;
        __nv_bfloat16 *bbase = static_cast<__nv_bfloat16 *>(B) +
                               (q < net->planesB ? q : 0) * planeB;
        for (int c = 0; c < 2; ++c)
            if ((rc = encode_kblocked(&d.mapB[c][q], bbase, (uint64_t)rowsB, (uint64_t)KB,
                                      256 / (c + 1))))
                return rc;
    }
    d.KB = (net->N + 31) / 32;
    d.mtiles = net->mtiles;
    d.stiles = 0;
    d.pad = 0;
    d.count = 0;
    d.ld_part = net->chunk;
    d.nS_part = net->d_nS_part;
    return GBS_OK;
}

int bucket(int v) {
    int b = 0;
    while ((1 << (b + 1)) <= v) ++b;
    return b;
}

// Dispatch of a grouped launch to the instantiation of (pair, ring depth):
// shallow = 0 the deepest ring, 1 one stage less.
template <int P, int kSW>
int launch_grouped_ring(cudaStream_t stream, int sm_count, int pair, int shallow,
                        const GemmNetDesc *d_nets, const int4 *d_tiles, int ntiles,
                        int64_t count0, int band, int keep_a, uint64_t wait_ns,
                        unsigned long long *err, OccOut occ, const SampleJobs &jobs) {
    if (pair == 1)
        return shallow
                   ? launch_variant<P, 1, kSW, shallow_stages<P, 1>()>(
                         stream, sm_count, d_nets, d_tiles, ntiles, count0, band, keep_a, wait_ns,
                         err, occ, jobs)
                   : launch_variant<P, 1, kSW>(stream, sm_count, d_nets, d_tiles, ntiles, count0,
                                               band, keep_a, wait_ns, err, occ, jobs);
    return shallow ? launch_variant<P, 2, kSW, shallow_stages<P, 2>()>(
                         stream, sm_count, d_nets, d_tiles, ntiles, count0, band, keep_a, wait_ns,
                         err, occ, jobs)
                   : launch_variant<P, 2, kSW>(stream, sm_count, d_nets, d_tiles, ntiles, count0,
                                               band, keep_a, wait_ns, err, occ, jobs);
}

}  // namespace

int tc_ring_stages(int P, int pair, int shallow) {
    const int deep = P == 3 ? (pair == 1 ? Cfg<3, 1>::kStages : Cfg<3, 2>::kStages)
                            : (pair == 1 ? Cfg<6, 1>::kStages : Cfg<6, 2>::kStages);
    return deep - (shallow ? 1 : 0);
}

bool tc_shallow_sampling_ok() { return sampling_kernels_ok() && shallow_sampling_kernels_ok(); }

int launch_gemm_grouped(cudaStream_t stream, int sm_count, int P, int pair, int band, int keep_a,
                        uint64_t wait_ns, const GemmNetDesc *d_nets, const int4 *d_tiles,
                        int ntiles, int64_t count0, unsigned long long *err, OccOut occ,
                        int shallow) {
    int rc;
    if ((rc = ensure_attrs())) return rc;
    if (occ.p && (d_tiles || occ.ld % 128 != 0 || occ.ld < count0))
        return set_error(GBS_EINVAL, "occupation output needs closed-form tiles and ld >= count, ld %% 128 == 0");
    if (pair != 1 && pair != 2) return set_error(GBS_EINVAL, "GEMM tiles per CTA pair must be 1 or 2");
    if (shallow != 0 && shallow != 1) return set_error(GBS_EINVAL, "ring depth option must be 0 or 1");
    const SampleJobs none;
    if (P == 3)
        return launch_grouped_ring<3, 0>(stream, sm_count, pair, shallow, d_nets, d_tiles, ntiles,
                                         count0, band, keep_a, wait_ns, err, occ, none);
    return launch_grouped_ring<6, 0>(stream, sm_count, pair, shallow, d_nets, d_tiles, ntiles,
                                     count0, band, keep_a, wait_ns, err, occ, none);
}

int tc_fill_desc(gbs_net *net, GemmNetDesc *out, bool alt) {
    if (!net->tc) return set_error(GBS_EINVAL, "network has no tensor-core plan");
    if (alt && !net->tc->d_desc_alt) return set_error(GBS_EINVAL, "network has no second operand");
    *out = alt ? net->tc->desc_alt : net->tc->desc;
    out->wave_sync = nullptr;  // grouped launches do not align waves
    return GBS_OK;
}

int launch_gemm_grouped_sampling(cudaStream_t stream, int sm_count, int pair, uint64_t wait_ns,
                                 const GemmNetDesc *d_nets, const int4 *d_tiles, int ntiles,
                                 unsigned long long *err, const SampleJobs &jobs, int shallow) {
    int rc;
    if ((rc = ensure_attrs())) return rc;
    if (!sampling_kernels_ok()) return set_error(GBS_EINVAL, "sampling GEMM unavailable");
    if (pair != 1 && pair != 2) return set_error(GBS_EINVAL, "GEMM tiles per CTA pair must be 1 or 2");
    if (shallow != 0 && shallow != 1) return set_error(GBS_EINVAL, "ring depth option must be 0 or 1");
    if (shallow && !shallow_sampling_kernels_ok())
        return set_error(GBS_EINVAL, "sampling GEMM with the shallower ring unavailable");
    return launch_grouped_ring<3, kSampWG>(stream, sm_count, pair, shallow, d_nets, d_tiles,
                                           ntiles, 0, 0, 0, wait_ns, err, OccOut(), jobs);
}

int tc_products(gbs_net *net) { return net->tc ? net->tc->P : 0; }

int tc_plan_create(gbs_net *net) {
    TcPlan *plan = new (std::nothrow) TcPlan();
    if (!plan) return set_error(GBS_ENOMEM, "host allocation failed");
    net->tc = plan;
    plan->P = (net->precision == GBS_BF16X3) ? 3 : 6;
    int rc;
    if ((rc = encode_net_maps(net, net->d_B, plan->desc))) return rc;
    if ((rc = pool_alloc(reinterpret_cast<void **>(&plan->d_sync), sizeof(unsigned int),
                         net->stream, "GEMM wave counter")))
        return rc;
    plan->desc.wave_sync = plan->d_sync;
    // the descriptor block lives beside the network's buffers on its stream
    // (the host copy outlives the asynchronous upload: it is the plan's)
    if ((rc = pool_alloc(reinterpret_cast<void **>(&plan->d_desc), sizeof(GemmNetDesc),
                         net->stream, "GEMM descriptors")))
        return rc;
    GBS_CUDA_TRY(cudaMemcpyAsync(plan->d_desc, &plan->desc, sizeof(GemmNetDesc),
                                 cudaMemcpyHostToDevice, net->stream));
    return GBS_OK;
}

void tc_plan_destroy(gbs_net *net) {
    if (net->tc) {
        pool_free_raw(net->tc->d_desc, net->stream);
        pool_free_raw(net->tc->d_desc_alt, net->stream);
        pool_free_raw(net->tc->d_sync, net->stream);
    }
    delete net->tc;
    net->tc = nullptr;
}

int tc_set_config(gbs_net *net, const GemmCfg &cfg) {
    if (!net->tc) return set_error(GBS_EINVAL, "network has no tensor-core GEMM");
    if (cfg.pair < 0 || cfg.pair > 2) return set_error(GBS_EINVAL, "pair must be 0 (auto), 1 or 2");
    if (cfg.band < 0) return set_error(GBS_EINVAL, "band must be >= 0");
    if (cfg.keep < 0 || cfg.keep > 31) return set_error(GBS_EINVAL, "keep_a must be in [0, 31]");
    net->tc->forced = cfg.pair != 0;
    GemmCfg c = cfg;
    if (!c.pair) c = GemmCfg();
    net->tc->cfg[0] = net->tc->cfg[1] = c;
    return GBS_OK;
}

GemmCfg tc_get_config(gbs_net *net) {
    if (!net->tc) return GemmCfg();
    return net->tc->cfg[1].pair ? net->tc->cfg[1] : net->tc->cfg[0];
}

void tc_set_pair_autotune(bool on) {
    std::lock_guard<std::mutex> lock(g_tc_mu);
    g_pair_autotune = on;
    g_tune.clear();
}

bool tc_pair_autotune() {
    std::lock_guard<std::mutex> lock(g_tc_mu);
    return g_pair_autotune;
}

// The candidates the autotuner times: one CTA or CTA pairs per tile group,
// each with bands of 16 and 8 groups (where the network has more groups than
// that; the bands with and without the evict-last policy on their A tiles)
// and the plain tile order.  The plain order streams all of A through L2 once
// per wave of CTAs; when A is larger than half the L2 that moves several
// times the bytes of a banded order from HBM, and although short timings can
// favour it (m8000: by about 1 %), over a long run the extra DRAM power lowers
// the clock under the power limit (m8000: 1063 against 1012 ms per step), so
// it is offered only for networks whose A fits in half the L2.  Each
// candidate runs with the deepest operand ring that fits in shared memory
// and, where `shallow` allows, with one stage less (keep_a bit 16).
std::vector<GemmCfg> tc_candidates(int mtiles, bool pairs, bool plain, bool shallow) {
    std::vector<GemmCfg> c;
    for (int pair = 1; pair <= (pairs ? 2 : 1); ++pair) {
        const int groups = (mtiles + pair - 1) / pair;
        bool banded = false;
        for (int band : {16, 8})
            if (groups > band) {
                banded = true;
                for (int keep : {0, 1}) c.push_back({pair, band, keep});
            }
        if (plain || !banded) c.push_back({pair, 0, 0});
    }
    const size_t deep = c.size();
    for (size_t i = 0; shallow && i < deep; ++i) c.push_back({c[i].pair, c[i].band, c[i].keep | 16});
    return c;
}

// One launch over the closed-form tiles of the network's current chunk in
// configuration g; with a job, the sampling variant that also runs it.
// keep_a bit 16 selects the operand ring one stage shallower; the kernel
// sees the other bits.
int launch_closed(gbs_net *net, const GemmCfg &g, int ntiles, int64_t count, const SampleJob *job,
                  OccOut occ) {
    TcPlan *plan = net->tc;
    if ((g.keep & 8) && plan->d_sync)
        GBS_CUDA_TRY(cudaMemsetAsync(plan->d_sync, 0, sizeof(unsigned int), net->stream));
    const int shallow = (g.keep & 16) ? 1 : 0;
    const int keep = g.keep & 15;
    if (!job)
        return launch_gemm_grouped(net->stream, net->sm_count, plan->P, g.pair, g.band, keep,
                                   net->wait_ns, plan->d_desc, nullptr, ntiles, count,
                                   net->d_flags + 1, occ, shallow);
    if (g.pair != 1 && g.pair != 2) return set_error(GBS_EINVAL, "GEMM tiles per CTA pair must be 1 or 2");
    if (shallow && !shallow_sampling_kernels_ok())
        return set_error(GBS_EINVAL, "sampling GEMM with the shallower ring unavailable");
    SampleJobs jobs;
    jobs.one = *job;
    return launch_grouped_ring<3, kSampWG>(net->stream, net->sm_count, g.pair, shallow,
                                           plan->d_desc, nullptr, ntiles, count, g.band, keep,
                                           net->wait_ns, net->d_flags + 1, occ, jobs);
}

// Time the candidate configurations on this chunk (as the launch to be
// configured runs: plain, or with `job` as the sampling variant; the job's
// samples are written again by that launch) and keep the fastest for this
// network and every network of the same size bucket.  The candidates
// are compared in the state a long run reaches: a first pass launches each
// once (it brings the GPU to the clock its power limit allows under this
// load), then kTunePasses passes time kTuneReps launches of each candidate,
// the candidates interleaved, and the times of the passes are summed.  (One
// launch each from an idle GPU favoured configurations that move more data:
// fast while the clock is high, slower once the power limit lowers it.)
constexpr int kTunePasses = 2, kTuneReps = 2;

int tc_autotune(gbs_net *net, int64_t count, const SampleJob *job, GemmCfg *out) {
    TcPlan *plan = net->tc;
    const auto key = std::make_tuple(bucket(net->N), bucket(net->M), plan->P, job ? 1 : 0);
    bool pairs;
    {
        std::lock_guard<std::mutex> lock(g_tc_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            *out = it->second;
            return GBS_OK;
        }
        pairs = g_pair_autotune;
    }
    *out = GemmCfg{1, 0, 0};
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    GBS_CUDA_TRY(cudaStreamIsCapturing(net->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) return GBS_OK;  // no timing inside a capture: default
    const int stiles = (int)((count + kTcTileSamples - 1) / kTcTileSamples);
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, net->device) != cudaSuccess) {
        cudaGetLastError();
        l2 = 0;
    }
    const double a_bytes = (double)(plan->P == 3 ? 2 : 3) * net->rowsA * net->ldK * 2.0;
    const std::vector<GemmCfg> cand =
        tc_candidates(net->mtiles, pairs, a_bytes <= 0.5 * l2, !job || shallow_sampling_kernels_ok());
    std::vector<float> total(cand.size(), 0.0f);
    cudaEvent_t e0, e1;
    GBS_CUDA_TRY(cudaEventCreate(&e0));
    GBS_CUDA_TRY(cudaEventCreate(&e1));
    int rc = GBS_OK;
    for (int pass = 0; pass <= kTunePasses && rc == GBS_OK; ++pass) {
        for (size_t c = 0; c < cand.size() && rc == GBS_OK; ++c) {
            const GemmCfg &g = cand[c];
            const int nt = ((net->mtiles + g.pair - 1) / g.pair) * stiles;
            const int reps = pass == 0 ? 1 : kTuneReps;
            cudaEventRecord(e0, net->stream);
            for (int q = 0; q < reps && rc == GBS_OK; ++q)
                rc = launch_closed(net, g, nt, count, job, OccOut());
            if (rc) break;
            cudaEventRecord(e1, net->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = set_error(GBS_ECUDA, "autotuner timing failed");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (pass > 0) total[c] += ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    size_t best = 0;
    for (size_t c = 1; c < cand.size(); ++c)
        if (total[c] < total[best]) best = c;
    *out = cand[best];
    // banded orders (operands beyond the L2) with the wave alignment: it
    // changes no cycle count the interleaved timing above can see, only the
    // DRAM traffic, whose power lowers the clock in a long run (m8000: 1.07
    // against 0.99 M trajectories/s); the plain order keeps A in L2 and
    // gains nothing from it (m1000: 2 % slower)
    if (out->band > 0) out->keep |= 8;
    std::lock_guard<std::mutex> lock(g_tc_mu);
    g_tune[key] = *out;
    return GBS_OK;
}

namespace {

const GemmCfg *pick_config(gbs_net *net, int64_t count, const SampleJob *job, int *rc) {
    TcPlan *plan = net->tc;
    GemmCfg &c = plan->cfg[job ? 1 : 0];
    *rc = GBS_OK;
    if (!c.pair) *rc = tc_autotune(net, count, job, &c);
    return &c;
}

}  // namespace

int launch_gemm_tc(gbs_net *net, int64_t count, OccOut occ) {
    if (count <= 0) return GBS_OK;
    TcPlan *plan = net->tc;
    if (!plan) return set_error(GBS_EINVAL, "no tensor-core plan");
    int rc;
    if ((rc = ensure_attrs())) return rc;
    const GemmCfg *c = pick_config(net, count, nullptr, &rc);
    if (rc) return rc;
    const int groups = (net->mtiles + c->pair - 1) / c->pair;
    const int stiles = (int)((count + kTcTileSamples - 1) / kTcTileSamples);
    return launch_closed(net, *c, groups * stiles, count, nullptr, occ);
}

int launch_gemm_tc_sampling(gbs_net *net, int64_t count, const SampleJob &job, OccOut occ) {
    if (count <= 0) return GBS_OK;
    TcPlan *plan = net->tc;
    if (!plan || plan->P != 3 || !plan->d_desc_alt)
        return set_error(GBS_EINVAL, "sampling GEMM needs a 3-product plan with a second operand");
    if (occ.p && (occ.ld % 128 != 0 || occ.ld < count))
        return set_error(GBS_EINVAL, "occupation output needs ld >= count, ld %% 128 == 0");
    int rc;
    if ((rc = ensure_attrs())) return rc;
    if (!sampling_kernels_ok()) return set_error(GBS_EINVAL, "sampling GEMM unavailable");
    const GemmCfg *c = pick_config(net, count, &job, &rc);
    if (rc) return rc;
    const int groups = (net->mtiles + c->pair - 1) / c->pair;
    const int stiles = (int)((count + kTcTileSamples - 1) / kTcTileSamples);
    return launch_closed(net, *c, groups * stiles, count, &job, occ);
}

bool tc_sampling_ready(gbs_net *net, bool allocate) {
    TcPlan *plan = net->tc;
    if (!plan || plan->P != 3 || !net->fuse_sampler || !net->d_B) return false;
    if (ensure_attrs() != GBS_OK) {
        cudaGetLastError();
        return false;
    }
    if (!sampling_kernels_ok()) return false;
    if (plan->d_desc_alt) return true;
    if (!allocate) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(net->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;  // no allocation inside a capture
    }
    // the second operand and n[] (from the stream-ordered pool, like the
    // first; the sampler writes every element the GEMM reads for valid
    // trajectories); without room the plain path runs
    void *B = nullptr, *n = nullptr;
    GemmNetDesc *d = nullptr;
    bool ok = pool_alloc(&B, net->B_bytes, net->stream, "second sample operand") == GBS_OK &&
              pool_alloc(&n, (size_t)net->chunk * sizeof(double), net->stream, "second n") == GBS_OK &&
              pool_alloc(reinterpret_cast<void **>(&d), sizeof(GemmNetDesc), net->stream,
                         "second GEMM descriptors") == GBS_OK;
    if (ok) ok = encode_net_maps(net, B, plan->desc_alt) == GBS_OK;
    plan->desc_alt.wave_sync = plan->d_sync;
    if (ok)
        ok = cudaMemcpyAsync(d, &plan->desc_alt, sizeof(GemmNetDesc), cudaMemcpyHostToDevice,
                             net->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pool_free_raw(B, net->stream);
        pool_free_raw(n, net->stream);
        pool_free_raw(d, net->stream);
        return false;
    }
    net->d_B_alt = B;
    net->d_n_alt = static_cast<double *>(n);
    plan->d_desc_alt = d;
    return true;
}

void tc_swap_sample_buffers(gbs_net *net) {
    TcPlan *plan = net->tc;
    std::swap(net->d_B, net->d_B_alt);
    std::swap(net->d_n, net->d_n_alt);
    std::swap(plan->desc, plan->desc_alt);
    std::swap(plan->d_desc, plan->d_desc_alt);
}

}  // namespace gbs
