// Batched ensembles over many networks of uneven size (one launch per round
// for the propagation of all networks).
//
// A batch groups networks that share a stream, a device and a BF16 split
// precision.  gbs_sample_batch draws every network's trajectories in rounds
// of one chunk per network; per round the samplers of all networks run, then
// ONE persistent grouped GEMM covers the tiles of all networks (a tile list
// ordered by decreasing K so the long tiles start first and the short ones
// fill the tail), then each network's finalize and generating-function sums.
// With the 3-product split and more than one round, the networks with at
// least kFoldMinModes output modes are sampled by their own sampler only in
// round 0: the grouped GEMM of round r also draws their round r + 1 (its
// spare warps take those networks' trajectories as one list) into each one's
// second operand, and their operands swap roles between rounds (round r
// reads operand r mod 2; the roles are restored at the end of the call).
// Smaller networks keep a sampler launch per round (their sampling would
// outlast their share of the GEMM).  The samples are bitwise those of the
// plain rounds.
// The whole call is captured into a CUDA graph and launched once; in the
// graph the per-network launches of a phase (samplers; finalize + generating
// functions) are independent branches over up to 8 auxiliary streams, so
// small networks' kernels run side by side instead of one after another
// (each network's own launches keep their order, so the results do not
// change).  The
// grouped GEMM's configuration (one CTA per tile or CTA pairs; plain or
// banded tile order; the deepest operand ring or one stage less) is chosen
// by timing the candidates on the batch's first round (cached per batch).
#include "gbs_internal.cuh"

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

struct gbs_batch {
    std::vector<gbs_net *> nets;
    cudaStream_t stream = nullptr;
    int P = 0;
    int pair = 0;     // GEMM tiles per CTA (1) or per CTA pair (2); 0 = not tuned yet
    int band = 0;     // tile order within a network: 0 plain, > 0 bands of that many groups
    int shallow = 0;  // operand ring: 0 the deepest that fits, 1 one stage less
    bool forced = false;  // set by gbs_set_batch_config
    int sm_count = 0;
    // device copies of the per-round descriptors and tile lists
    gbs::GemmNetDesc *d_desc = nullptr;
    int4 *d_tiles = nullptr;
    size_t desc_cap = 0, tiles_cap = 0;
    // sampler jobs of rounds 1.. (folded sampling): [rounds][nets] and the
    // per-round list offsets [rounds][nets + 1]
    gbs::SampleJob *d_jobs = nullptr;
    int64_t *d_prefix = nullptr;
    size_t jobs_cap = 0, prefix_cap = 0;
    int last_rounds = 0;
    int64_t last_tiles = 0;
    bool last_fold = false;
    // fork/join streams and events of the captured graph
    std::vector<cudaStream_t> aux;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
};

using namespace gbs;

namespace {

struct RoundPlan {
    std::vector<GemmNetDesc> desc;  // [rounds][nets]
    std::vector<int4> tiles;        // all rounds, concatenated
    std::vector<int> tile_off;      // [rounds + 1]
    std::vector<std::vector<int64_t>> count;  // [rounds][nets]
    int rounds = 0;
    bool fold = false;              // some network's sampling runs in the GEMMs
    std::vector<char> fold_net;     // [nets]: round r reads operand r mod 2, r + 1 sampled in r's GEMM
    std::vector<SampleJob> jobs;    // [rounds][nets] (round 0 unused)
    std::vector<int64_t> prefix;    // [rounds][nets + 1]
    std::vector<int64_t> step;      // [nets]: trajectories per round (chunk_step)
};

int build_rounds(gbs_batch *b, const int64_t *E, int pair, int band, RoundPlan &rp,
                 const std::vector<char> *fold_net = nullptr, const uint64_t *seeds = nullptr,
                 const uint64_t *first = nullptr) {
    const int nn = (int)b->nets.size();
    // round r holds chunk r of every network, chunks of chunk_step (as
    // gbs_sample cuts them, so that a batch and per-network calls sum in
    // the same order)
    int rounds = 0;
    std::vector<int64_t> step(nn);
    for (int i = 0; i < nn; ++i) {
        step[i] = chunk_step(b->nets[i], E[i]);
        rounds = std::max<int>(rounds, (int)((E[i] + step[i] - 1) / step[i]));
    }
    rp.rounds = rounds;
    rp.step = step;
    rp.desc.resize((size_t)rounds * nn);
    rp.count.assign(rounds, std::vector<int64_t>(nn, 0));
    rp.tile_off.assign(rounds + 1, 0);
    rp.tiles.clear();
    for (int r = 0; r < rounds; ++r) {
        // networks in order of decreasing K, so long tiles are issued first
        std::vector<int> order(nn);
        for (int i = 0; i < nn; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int c) { return b->nets[a]->N > b->nets[c]->N; });
        rp.tile_off[r] = (int)rp.tiles.size();
        for (int i = 0; i < nn; ++i) {
            gbs_net *net = b->nets[i];
            const int64_t done = (int64_t)r * step[i];
            const int64_t c = std::max<int64_t>(0, std::min<int64_t>(step[i], E[i] - done));
            rp.count[r][i] = c;
            GemmNetDesc d;
            int rc;
            const bool alt = fold_net && (*fold_net)[i] && (r & 1);
            if ((rc = tc_fill_desc(net, &d, alt))) return rc;
            d.count = c;
            d.stiles = (int)((c + kTcTileSamples - 1) / kTcTileSamples);
            rp.desc[(size_t)r * nn + i] = d;
        }
        for (int oi = 0; oi < nn; ++oi) {
            const int i = order[oi];
            const GemmNetDesc &d = rp.desc[(size_t)r * nn + i];
            const int groups = (d.mtiles + pair - 1) / pair;
            // plain: every group of one trajectory tile side by side; banded:
            // bands of `band` groups, the trajectory tiles of a band in order
            const int bw = (band > 0 && band < groups) ? band : groups;
            for (int g0 = 0; g0 < groups; g0 += bw)
                for (int st = 0; st < d.stiles; ++st)
                    for (int g = g0; g < std::min(groups, g0 + bw); ++g)
                        rp.tiles.push_back(make_int4(i, g, st, 0));
        }
    }
    rp.tile_off[rounds] = (int)rp.tiles.size();
    rp.fold_net.assign(nn, 0);
    rp.fold = false;
    for (int i = 0; fold_net && i < nn; ++i) {
        rp.fold_net[i] = (*fold_net)[i];
        rp.fold = rp.fold || rp.fold_net[i];
    }
    if (rp.fold) {
        rp.jobs.assign((size_t)rounds * nn, SampleJob());
        rp.prefix.assign((size_t)rounds * (nn + 1), 0);
        for (int r = 1; r < rounds; ++r) {
            int64_t acc = 0;
            for (int i = 0; i < nn; ++i) {
                gbs_net *net = b->nets[i];
                const uint64_t e0 = first[i] + (uint64_t)r * (uint64_t)rp.step[i];
                const int64_t c = rp.fold_net[i] ? rp.count[r][i] : 0;
                if (c > 0) {
                    void *B = (r & 1) ? net->d_B_alt : net->d_B;
                    double *n = (r & 1) ? net->d_n_alt : net->d_n;
                    rp.jobs[(size_t)r * nn + i] = sample_job_bf16(net, B, n, seeds[i], e0, c);
                }
                rp.prefix[(size_t)r * (nn + 1) + i] = acc;
                acc += c;
            }
            rp.prefix[(size_t)r * (nn + 1) + nn] = acc;
        }
    }
    return GBS_OK;
}

int upload_rounds(gbs_batch *b, const RoundPlan &rp) {
    const size_t nd = rp.desc.size(), nt = std::max<size_t>(rp.tiles.size(), 1);
    if (nd > b->desc_cap) {
        if (b->d_desc) cudaFree(b->d_desc);
        b->d_desc = nullptr;
        GBS_CUDA_TRY(cudaMalloc(&b->d_desc, nd * sizeof(GemmNetDesc)));
        b->desc_cap = nd;
    }
    if (nt > b->tiles_cap) {
        if (b->d_tiles) cudaFree(b->d_tiles);
        b->d_tiles = nullptr;
        GBS_CUDA_TRY(cudaMalloc(&b->d_tiles, nt * sizeof(int4)));
        b->tiles_cap = nt;
    }
    // synchronous copies: the descriptors must be in place before the graph
    // that reads them is launched, and the host vectors are temporaries
    if (rp.fold) {
        if (rp.jobs.size() > b->jobs_cap) {
            if (b->d_jobs) cudaFree(b->d_jobs);
            b->d_jobs = nullptr;
            GBS_CUDA_TRY(cudaMalloc(&b->d_jobs, rp.jobs.size() * sizeof(SampleJob)));
            b->jobs_cap = rp.jobs.size();
        }
        if (rp.prefix.size() > b->prefix_cap) {
            if (b->d_prefix) cudaFree(b->d_prefix);
            b->d_prefix = nullptr;
            GBS_CUDA_TRY(cudaMalloc(&b->d_prefix, rp.prefix.size() * sizeof(int64_t)));
            b->prefix_cap = rp.prefix.size();
        }
    }
    GBS_CUDA_TRY(cudaStreamSynchronize(b->stream));
    GBS_CUDA_TRY(cudaMemcpy(b->d_desc, rp.desc.data(), nd * sizeof(GemmNetDesc),
                            cudaMemcpyHostToDevice));
    if (!rp.tiles.empty())
        GBS_CUDA_TRY(cudaMemcpy(b->d_tiles, rp.tiles.data(), rp.tiles.size() * sizeof(int4),
                                cudaMemcpyHostToDevice));
    if (rp.fold) {
        GBS_CUDA_TRY(cudaMemcpy(b->d_jobs, rp.jobs.data(), rp.jobs.size() * sizeof(SampleJob),
                                cudaMemcpyHostToDevice));
        GBS_CUDA_TRY(cudaMemcpy(b->d_prefix, rp.prefix.data(), rp.prefix.size() * sizeof(int64_t),
                                cudaMemcpyHostToDevice));
    }
    return GBS_OK;
}

int round_gemm(gbs_batch *b, const RoundPlan &rp, int r, int pair, int shallow) {
    const int nn = (int)b->nets.size();
    const int off = rp.tile_off[r], nt = rp.tile_off[r + 1] - off;
    gbs_net *n0 = b->nets[0];
    prof_mark(n0, GBS_PHASE_GEMM, 0, true);
    int rc;
    if (rp.fold && r + 1 < rp.rounds && rp.prefix[(size_t)(r + 1) * (nn + 1) + nn] > 0) {
        // this round's GEMM also draws round r + 1 of every network
        SampleJobs sj;
        sj.jobs = b->d_jobs + (size_t)(r + 1) * nn;
        sj.prefix = b->d_prefix + (size_t)(r + 1) * (nn + 1);
        sj.n = nn;
        rc = launch_gemm_grouped_sampling(b->stream, b->sm_count, pair, n0->wait_ns,
                                          b->d_desc + (size_t)r * nn, b->d_tiles + off, nt,
                                          n0->d_flags + 1, sj, shallow);
    } else {
        rc = launch_gemm_grouped(b->stream, b->sm_count, b->P, pair, 0, 0, n0->wait_ns,
                                 b->d_desc + (size_t)r * nn, b->d_tiles + off, nt, 0,
                                 n0->d_flags + 1, OccOut(), shallow);
    }
    prof_mark(n0, GBS_PHASE_GEMM, 1, false);
    return rc;
}

// Run body(i, net) for every network of the round; with auxiliary streams
// (graph capture) network i's launches go to branch i mod |aux|, forked from
// and joined back into the batch stream.
template <typename Body>
int per_network(gbs_batch *b, const RoundPlan &rp, int r, bool branches, Body &&body) {
    const int nn = (int)b->nets.size();
    const int nb = branches ? (int)b->aux.size() : 0;
    if (nb > 0) {
        GBS_CUDA_TRY(cudaEventRecord(b->fork, b->stream));
        for (int k = 0; k < nb; ++k) GBS_CUDA_TRY(cudaStreamWaitEvent(b->aux[k], b->fork, 0));
    }
    int rc = GBS_OK;
    for (int i = 0; i < nn && rc == GBS_OK; ++i) {
        if (rp.count[r][i] <= 0) continue;
        gbs_net *net = b->nets[i];
        cudaStream_t own = net->stream;
        if (nb > 0) net->stream = b->aux[i % nb];
        rc = body(i, net);
        net->stream = own;
    }
    if (nb > 0) {
        for (int k = 0; k < nb; ++k) {
            GBS_CUDA_TRY(cudaEventRecord(b->join[k], b->aux[k]));
            GBS_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->join[k], 0));
        }
    }
    return rc;
}

int round_front(gbs_batch *b, const RoundPlan &rp, int r, const uint64_t *seeds,
                const uint64_t *first, bool branches = false) {
    return per_network(b, rp, r, branches, [&](int i, gbs_net *net) {
        // networks whose rounds 1.. are drawn by the GEMMs
        if (r > 0 && rp.fold && rp.fold_net[i]) return (int)GBS_OK;
        const uint64_t e0 = first[i] + (uint64_t)r * (uint64_t)rp.step[i];
        return launch_sample_bf16(net, seeds[i], e0, rp.count[r][i]);
    });
}

// Every network's finalize and generating functions (per-network branches).
// A single grouped generating-function launch per round over all networks'
// chunks (a persistent kernel over a heaviest-first work list) was measured
// 2 % slower per batch64 step (325 against 318 ms on one box): the branches
// overlap one network's finalize with the others' generating functions, and
// the grouped launch also walks the slot blocks past every chunk's window,
// which the host cannot know.
int round_back(gbs_batch *b, const RoundPlan &rp, int r, const uint64_t *first,
               bool branches = false) {
    return per_network(b, rp, r, branches, [&](int i, gbs_net *net) {
        const uint64_t e0 = first[i] + (uint64_t)r * (uint64_t)rp.step[i];
        int rc;
        if ((rc = launch_finalize(net, rp.count[r][i]))) return rc;
        prof_mark(net, GBS_PHASE_GF, 0, true);
        if ((rc = launch_gf(net, e0, rp.count[r][i]))) return rc;
        prof_mark(net, GBS_PHASE_GF, 1, false);
        return (int)GBS_OK;
    });
}

// Folded rounds: the networks' operands swap roles after each round, so that
// round r's finalize and generating functions read operand r mod 2's n[].
void swap_all(gbs_batch *b, const RoundPlan &rp) {
    for (size_t i = 0; i < b->nets.size(); ++i)
        if (rp.fold_net[i]) tc_swap_sample_buffers(b->nets[i]);
}

// Every round of the call: samplers (round 0 only when folded), GEMM,
// finalize + generating functions.
int run_rounds(gbs_batch *b, const RoundPlan &rp, const uint64_t *seeds, const uint64_t *first,
               bool branches) {
    int rc = GBS_OK, swaps = 0;
    for (int r = 0; r < rp.rounds && rc == GBS_OK; ++r) {
        if ((rc = round_front(b, rp, r, seeds, first, branches))) break;
        if ((rc = round_gemm(b, rp, r, b->pair, b->shallow))) break;
        if ((rc = round_back(b, rp, r, first, branches))) break;
        if (rp.fold) {
            swap_all(b, rp);
            ++swaps;
        }
    }
    if (swaps & 1) swap_all(b, rp);
    return rc;
}

// The batch GEMM's candidate configurations: one CTA per tile or CTA pairs
// (where the autotuner takes pairs), each with the plain tile order and
// bands of 8 groups within every network, each with the deepest operand ring
// that fits in shared memory and a ring one stage shallower.
struct BatchCand {
    int pair, band, shallow;
};
std::vector<BatchCand> batch_candidates() {
    std::vector<BatchCand> c;
    for (int pair = 1; pair <= (tc_pair_autotune() ? 2 : 1); ++pair)
        for (int band : {0, 8})
            for (int shallow : {0, 1}) c.push_back({pair, band, shallow});
    return c;
}

// Time the candidates on round 0 (the samplers of round 0 run first so the
// operands are real) and keep the fastest; as the single-network autotuner:
// a first pass launches each candidate once, then two passes time two
// launches of each, candidates interleaved, times summed.  Every candidate
// gives bitwise the same sums.
int tune_batch(gbs_batch *b, const int64_t *E, const uint64_t *seeds, const uint64_t *first) {
    const std::vector<BatchCand> cand = batch_candidates();
    std::vector<RoundPlan> plans(cand.size());
    std::vector<float> total(cand.size(), 0.0f);
    int rc = GBS_OK;
    cudaEvent_t e0, e1;
    GBS_CUDA_TRY(cudaEventCreate(&e0));
    GBS_CUDA_TRY(cudaEventCreate(&e1));
    for (size_t c = 0; c < cand.size() && rc == GBS_OK; ++c)
        rc = build_rounds(b, E, cand[c].pair, cand[c].band, plans[c]);
    // round 0's operands (the samplers do not depend on the tile list)
    if (rc == GBS_OK && (rc = upload_rounds(b, plans[0])) == GBS_OK)
        rc = round_front(b, plans[0], 0, seeds, first);
    for (int pass = 0; pass <= 2 && rc == GBS_OK; ++pass) {
        for (size_t c = 0; c < cand.size() && rc == GBS_OK; ++c) {
            if ((rc = upload_rounds(b, plans[c]))) break;
            const int reps = pass == 0 ? 1 : 2;
            cudaEventRecord(e0, b->stream);
            for (int q = 0; q < reps && rc == GBS_OK; ++q)
                rc = round_gemm(b, plans[c], 0, cand[c].pair, cand[c].shallow);
            if (rc) break;
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = set_error(GBS_ECUDA, "batch autotuner timing failed");
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
    b->pair = cand[best].pair;
    b->band = cand[best].band;
    b->shallow = cand[best].shallow;
    return GBS_OK;
}

}  // namespace

extern "C" {

int gbs_make_batch(gbs_net_t *nets, int count, gbs_batch_t *out) {
    if (!out) return set_error(GBS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!nets || count < 1 || count > 4096)
        return set_error(GBS_EINVAL, "need 1..4096 networks");
    for (int i = 0; i < count; ++i) {
        if (!nets[i]) return set_error(GBS_EINVAL, "network %d is NULL", i);
        if (simt_precision(nets[i]->precision))
            return set_error(GBS_EINVAL, "batches need a BF16 split precision (network %d is FP64 or FP32)",
                             i);
        if (nets[i]->precision != nets[0]->precision)
            return set_error(GBS_EINVAL, "all networks of a batch must share the precision");
        if (nets[i]->stream != nets[0]->stream || nets[i]->device != nets[0]->device)
            return set_error(GBS_EINVAL, "all networks of a batch must share stream and device");
        for (int j = 0; j < i; ++j)
            if (nets[j] == nets[i]) return set_error(GBS_EINVAL, "network %d appears twice", i);
    }
    gbs_batch *b = new (std::nothrow) gbs_batch();
    if (!b) return set_error(GBS_ENOMEM, "host allocation failed");
    b->nets.assign(nets, nets + count);
    b->stream = nets[0]->stream;
    b->P = tc_products(nets[0]);
    b->sm_count = nets[0]->sm_count;
    const int nb = std::min(count, 8);
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < nb; ++k) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) b->aux.push_back(st);
        ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
        if (ok) b->join.push_back(ev);
    }
    if (!ok) {
        cudaGetLastError();
        gbs_free_batch(b);
        return set_error(GBS_ECUDA, "could not create the batch's streams and events");
    }
    *out = b;
    return GBS_OK;
}

int gbs_sample_batch(gbs_batch_t b, const uint64_t *seeds, const uint64_t *first_sample,
                     const int64_t *E, const int *n_sub, const int *K1) {
    if (!b || !seeds || !first_sample || !E || !n_sub || !K1)
        return set_error(GBS_EINVAL, "NULL argument");
    const int nn = (int)b->nets.size();
    int rc;
    for (int i = 0; i < nn; ++i) {
        if (E[i] < 0) return set_error(GBS_EINVAL, "E[%d] < 0", i);
        if ((rc = fix_estimator(b->nets[i], n_sub[i], K1[i]))) return rc;
    }
    if (!b->pair) {
        if ((rc = tune_batch(b, E, seeds, first_sample))) return rc;
    }
    // fold a network's sampling into the GEMMs when it has more than one
    // round, its setting asks for it (by default from kFoldMinModes output
    // modes) and its second operand exists (allocated here, outside the
    // capture)
    std::vector<char> fold_net(nn, 0);
    bool fold = false;
    for (int i = 0; i < nn; ++i) {
        gbs_net *net = b->nets[i];
        fold_net[i] = b->P == 3 && E[i] > net->chunk && fold_wanted(net) &&
                      (!b->shallow || tc_shallow_sampling_ok()) && tc_sampling_ready(net, true);
        fold = fold || fold_net[i];
    }
    RoundPlan rp;
    if ((rc = build_rounds(b, E, b->pair, b->band, rp, &fold_net, seeds, first_sample))) return rc;
    if ((rc = upload_rounds(b, rp))) return rc;
    b->last_rounds = rp.rounds;
    b->last_tiles = (int64_t)rp.tiles.size();
    b->last_fold = fold;

    if (b->stream == nullptr || b->nets[0]->prof.on) {
        // the legacy default stream cannot be captured, and phase timing
        // (gbs_profile_enable on the first network) needs the launches
        // bracketed one by one: issue the rounds directly
        if ((rc = run_rounds(b, rp, seeds, first_sample, false))) return rc;
        for (int i = 0; i < nn; ++i) count_samples(b->nets[i], first_sample[i], E[i]);
        return GBS_OK;
    }
    // capture every round into one graph and launch it
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    GBS_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    rc = run_rounds(b, rp, seeds, first_sample, true);
    cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess)
        return set_error(GBS_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_error(GBS_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
    }
    ce = cudaGraphLaunch(exec, b->stream);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess)
        return set_error(GBS_ECUDA, "graph launch failed: %s", cudaGetErrorString(ce));
    for (int i = 0; i < nn; ++i) count_samples(b->nets[i], first_sample[i], E[i]);
    return GBS_OK;
}

int gbs_set_batch_config(gbs_batch_t b, int pair, int band, int stages) {
    if (!b) return set_error(GBS_EINVAL, "null batch");
    if (pair < 0 || pair > 2) return set_error(GBS_EINVAL, "pair must be 0 (auto), 1 or 2");
    if (band < 0) return set_error(GBS_EINVAL, "band must be >= 0");
    int shallow = 0;
    if (pair && stages) {
        if (stages == tc_ring_stages(b->P, pair, 1))
            shallow = 1;
        else if (stages != tc_ring_stages(b->P, pair, 0))
            return set_error(GBS_EINVAL, "stages must be 0 (deepest), %d or %d for %d products and pair %d",
                             tc_ring_stages(b->P, pair, 0), tc_ring_stages(b->P, pair, 1), b->P, pair);
    } else if (stages < 0) {
        return set_error(GBS_EINVAL, "stages must be >= 0");
    }
    b->pair = pair;
    b->band = pair ? band : 0;
    b->shallow = pair ? shallow : 0;
    b->forced = pair != 0;
    return GBS_OK;
}

int gbs_batch_info(gbs_batch_t b, int *pair, int *band, int *stages, int *rounds, int64_t *tiles) {
    if (!b) return set_error(GBS_EINVAL, "null batch");
    if (pair) *pair = b->pair;
    if (band) *band = b->band;
    if (stages) *stages = b->pair ? tc_ring_stages(b->P, b->pair, b->shallow) : 0;
    if (rounds) *rounds = b->last_rounds;
    if (tiles) *tiles = b->last_tiles;
    return GBS_OK;
}

void gbs_free_batch(gbs_batch_t b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_jobs) cudaFree(b->d_jobs);
    if (b->d_prefix) cudaFree(b->d_prefix);
    for (cudaStream_t st : b->aux) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

}  // extern "C"
