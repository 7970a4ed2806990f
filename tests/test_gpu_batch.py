"""Tile configurations of the tcgen05 GEMM and batched uneven networks.

The tile configurations (one CTA per tile or CTA pairs, plain or banded
tile order) differ only in which CTA computes which tile and how the
operands reach shared memory; each output element's MMA chain is the same,
so per-trajectory results must agree bitwise.  A
batch issues the same kernels per network (one grouped GEMM per round), so
its sub-ensemble sums must equal per-network runs bitwise, and every
network's P(m) must match its exact distribution within sampling error.
"""

import numpy as np
import pytest

import oracle
import oracle.exact as ex
import workloads as wl
from stats import agreement

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gbs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_12749_gb300 as g
    g.build()
    return g


CONFIGS = [pytest.param((1, 0, 0), id="cta"), pytest.param((1, 1, 0), id="cta-band1"),
           pytest.param((1, 2, 1), id="cta-band2-keep"), pytest.param((2, 0, 0), id="pair"),
           pytest.param((2, 1, 1), id="pair-band1-keep"),
           pytest.param((1, 2, 8), id="cta-band2-aligned"),
           pytest.param((2, 1, 9), id="pair-band1-keep-aligned"),
           pytest.param((2, 1, 6), id="pair-band1-policies"),
           pytest.param((1, 0, 16), id="cta-shallow-ring"),
           pytest.param((2, 0, 16), id="pair-shallow-ring"),
           pytest.param((2, 1, 25), id="pair-band1-keep-aligned-shallow-ring")]


@pytest.mark.parametrize("config", CONFIGS)
@pytest.mark.parametrize("shape", [(16, 16), (9, 9), (300, 300), (130, 200), (257, 100)])
def test_tile_configurations_agree_bitwise(gbs, shape, config):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    N, M = shape
    net_def = wl.small_network(N, M=M, r=0.8, t2=0.93, seed=31 + N)
    res = []
    for cfg in ((1, 0, 0), config):
        net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
        gbs.gbs_set_gemm_config(net, *cfg)
        n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, 100, 333)
        assert gbs.gbs_gemm_config(net) == cfg
        res.append(nS)
        gbs.gbs_free_network(net)
    assert np.array_equal(res[0], res[1])
    no, nSo = oracle.samples(net_def.T, net_def.r, net_def.seed_s, 100, 333)
    assert np.max(np.abs(res[0] - nSo) / np.maximum(np.abs(nSo), 1.0)) < 2.0 ** -12


@pytest.mark.parametrize("config", CONFIGS)
def test_tile_configurations_agree_on_many_tiles(gbs, config):
    """A network of 10 mode tiles over 3 waves of trajectory tiles (the
    bands, pairs and the ragged last band all in use), 6 products: the
    per-trajectory totals of every configuration are bitwise those of the
    plain one."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    net_def = wl.small_network(320, M=640, r=0.6, t2=0.9, seed=77)
    res = []
    for cfg in ((1, 0, 0), config):
        net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x6", stream)
        gbs.gbs_set_gemm_config(net, *cfg)
        n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, 0, 3 * 152 * 128 + 77)
        res.append(nS)
        gbs.gbs_free_network(net)
    assert np.array_equal(res[0], res[1])


def test_autotuner_picks_a_configuration(gbs):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    net_def = wl.small_network(200, r=0.7, t2=0.9, seed=3)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    assert gbs.gbs_gemm_config(net) == (0, 0, 0)
    gbs.gbs_sample(net, net_def.seed_s, 0, 5000, 10, 256)
    pair, band, keep = gbs.gbs_gemm_config(net)
    assert pair in (1, 2) and band >= 0 and (keep & ~16) in (0, 1, 8, 9)
    # the waves of banded orders are aligned, those of the plain order not
    assert bool(keep & 8) == (band > 0)
    gbs.gbs_free_network(net)


def _uneven_defs():
    sizes = [(40, 0.6, 0.8), (100, 0.9, 0.95), (257, 0.7, 0.9), (300, 0.5, 0.99),
             (64, 1.1, 0.85), (130, 0.8, 0.97)]
    return [wl.small_network(N, r=r, t2=t2, seed=50 + i) for i, (N, r, t2) in enumerate(sizes)]


@pytest.mark.parametrize("own_stream", [True, False])
def test_batch_equals_per_network_runs(gbs, own_stream):
    import torch
    s = torch.cuda.Stream() if own_stream else None
    sptr = s.cuda_stream if own_stream else 0
    defs = _uneven_defs()
    E = [3000, 7000, 20000, 1000, 12345, 2048]
    n_sub = [10, 8, 16, 4, 7, 16]
    K1 = [64, 128, 256, 512, 64, 256]
    seeds = [d.seed_s for d in defs]
    first = [11 * i for i in range(len(defs))]
    nets = [gbs.gbs_make_network(d.T, d.r, "bf16x3", sptr) for d in defs]
    singles = [gbs.gbs_make_network(d.T, d.r, "bf16x3", sptr) for d in defs]
    batch = gbs.gbs_make_batch(nets)
    gbs.gbs_sample_batch(batch, seeds, first, E, n_sub, K1)
    (pair, band, stages), rounds, tiles = gbs.gbs_batch_info(batch)
    assert pair in (1, 2) and band >= 0 and rounds >= 1 and tiles > 0
    # the deepest ring that fits, or one stage less (3 products)
    assert stages in ((3, 4) if pair == 1 else (5, 6))
    for i, d in enumerate(defs):
        gbs.gbs_sample(singles[i], seeds[i], first[i], E[i], n_sub[i], K1[i])
        _, _, acc_b, cnt_b = gbs.gbs_get_accumulators(nets[i])
        _, _, acc_s, cnt_s = gbs.gbs_get_accumulators(singles[i])
        assert np.array_equal(cnt_b, cnt_s)
        assert np.array_equal(acc_b, acc_s), i
    # a second call continues the trajectory stream
    gbs.gbs_sample_batch(batch, seeds, [f + e for f, e in zip(first, E)], E, n_sub, K1)
    for i in range(len(defs)):
        _, _, _, cnt = gbs.gbs_get_accumulators(nets[i])
        assert cnt.sum() == 2 * E[i]
    gbs.gbs_free_batch(batch)
    for n in nets + singles:
        gbs.gbs_free_network(n)


@pytest.mark.parametrize("config", [pytest.param((1, 0, 4), id="cta"), pytest.param((1, 8, 4), id="cta-band8"),
                                    pytest.param((2, 0, 6), id="pair"),
                                    pytest.param((2, 8, 6), id="pair-band8"),
                                    pytest.param((1, 0, 3), id="cta-ring3"),
                                    pytest.param((1, 8, 3), id="cta-band8-ring3"),
                                    pytest.param((2, 0, 5), id="pair-ring5"),
                                    pytest.param((2, 8, 5), id="pair-band8-ring5")])
def test_batch_candidates_agree_bitwise(gbs, config):
    """Every configuration the batch autotuner times (one CTA per tile or CTA
    pairs, plain tile order or bands of 8 groups within each network, the
    deepest operand ring or one stage less) gives bitwise the sums of
    per-network runs; one network has 18 mode tiles (9 pair groups), so the
    bands are in use."""
    import torch
    sptr = torch.cuda.current_stream().cuda_stream
    defs = [wl.small_network(1100, r=0.6, t2=0.9, seed=71), wl.small_network(150, r=0.9, t2=0.8, seed=72),
            wl.small_network(520, r=0.7, t2=0.95, seed=73)]
    E, n_sub, K1 = [4000, 9000, 5000], [8, 8, 8], [2048, 512, 1024]
    seeds = [d.seed_s for d in defs]
    first = [0, 0, 0]
    nets = [gbs.gbs_make_network(d.T, d.r, "bf16x3", sptr) for d in defs]
    batch = gbs.gbs_make_batch(nets)
    gbs.gbs_set_batch_config(batch, *config)
    gbs.gbs_sample_batch(batch, seeds, first, E, n_sub, K1)
    assert gbs.gbs_batch_info(batch)[0] == config
    for i, d in enumerate(defs):
        single = gbs.gbs_make_network(d.T, d.r, "bf16x3", sptr)
        gbs.gbs_sample(single, seeds[i], first[i], E[i], n_sub[i], K1[i])
        _, _, acc_b, cnt_b = gbs.gbs_get_accumulators(nets[i])
        _, _, acc_s, cnt_s = gbs.gbs_get_accumulators(single)
        gbs.gbs_free_network(single)
        assert np.array_equal(cnt_b, cnt_s)
        assert np.array_equal(acc_b.view(np.float64), acc_s.view(np.float64)), (config, i)
    gbs.gbs_free_batch(batch)
    for n in nets:
        gbs.gbs_free_network(n)


def test_batch_distributions_match_exact(gbs):
    """A batch of uneven Haar networks (N log-uniform, r_j ~ U[0.5, 1.5],
    amplitude t ~ U[0.5, 0.995]): each network's matrix-P P(m) agrees with
    its exact uniform-loss distribution within sampling error."""
    import torch
    s = torch.cuda.Stream()
    wls = wl.batched_networks(count=8, n_lo=60, n_hi=400)
    defs = [w.network() for w in wls]
    # correlated fluctuations across bins make 2^15 trajectories too few for
    # the chi^2 criterion at the batch's high losses (t^2 down to 0.25)
    E = [2 ** 17] * len(defs)
    n_sub = [64] * len(defs)
    K1s, offs = [], []
    for w, d in zip(wls, defs):
        K1, off = wl.dft_window(w.N, float(d.r.max()), w.t2, float(np.mean(np.sinh(d.r) ** 2)))
        K1s.append(K1)
        offs.append(off)
    nets = [gbs.gbs_make_network(d.T, d.r, "bf16x3", s.cuda_stream) for d in defs]
    batch = gbs.gbs_make_batch(nets)
    gbs.gbs_sample_batch(batch, [d.seed_s for d in defs], [0] * len(defs), E, n_sub, K1s)
    for i, (w, d) in enumerate(zip(wls, defs)):
        P = gbs.gbs_binned_counts(nets[i], offs[i], K1s[i])
        mu = ex.eigenvalues_uniform_loss(d.r, w.t2)
        Pex = ex.exact_distribution(mu, K1s[i], offs[i]).real
        res = agreement(P[0], P[1], Pex)
        assert res["ok"], (i, w.N, res)
        assert abs(P[0].sum() - 1.0) < 1e-9
    gbs.gbs_free_batch(batch)
    for n in nets:
        gbs.gbs_free_network(n)


@pytest.mark.parametrize("own_stream", [True, False])
def test_multi_round_batch_folds_the_sampler_bitwise(gbs, own_stream):
    """More than one round per call: the grouped GEMM of round r draws round
    r + 1 of every network (networks with 1, 2 or 3 rounds, ragged last
    rounds).  The sums equal per-network runs and a batch in which one
    network samples every round separately (its folding switched off), bit
    for bit; the captured graph (own stream) and the direct launches
    (legacy stream) agree."""
    import torch
    s = torch.cuda.Stream() if own_stream else None
    sptr = s.cuda_stream if own_stream else 0
    defs = _uneven_defs()
    probe = gbs.gbs_make_network(defs[0].T, defs[0].r, "bf16x3", sptr)
    chunk = gbs.gbs_network_info(probe)[3]
    gbs.gbs_free_network(probe)
    E = [2 * chunk + 777, chunk + 5, 20000, chunk, 2 * chunk, 3 * chunk - 1]
    n_sub = [10, 8, 16, 4, 7, 16]
    K1 = [64, 128, 256, 512, 64, 256]
    seeds = [d.seed_s for d in defs]
    first = [13 * i for i in range(len(defs))]
    sums = {}
    for mode in ("fold", "plain", "single"):
        nets = [gbs.gbs_make_network(d.T, d.r, "bf16x3", sptr) for d in defs]
        for net in nets:
            gbs.gbs_set_sampler_fusion(net, 2)  # fold also these small networks
        if mode == "single":
            for i, net in enumerate(nets):
                gbs.gbs_sample(net, seeds[i], first[i], E[i], n_sub[i], K1[i])
        else:
            if mode == "plain":
                gbs.gbs_set_sampler_fusion(nets[2], 0)
            batch = gbs.gbs_make_batch(nets)
            gbs.gbs_sample_batch(batch, seeds, first, E, n_sub, K1)
            _, rounds, _ = gbs.gbs_batch_info(batch)
            assert rounds == 3
            gbs.gbs_free_batch(batch)
        sums[mode] = [gbs.gbs_get_accumulators(n) for n in nets]
        if mode == "fold":  # networks of more than one round fold
            assert [gbs.gbs_sampler_fusion(n) for n in nets] == [e > chunk for e in E]
        for n in nets:
            gbs.gbs_free_network(n)
    for mode in ("plain", "single"):
        for i in range(len(defs)):
            assert np.array_equal(sums["fold"][i][3], sums[mode][i][3]), (mode, i)
            assert np.array_equal(sums["fold"][i][2], sums[mode][i][2]), (mode, i)


@pytest.mark.parametrize("config", [pytest.param((1, 0, 3), id="cta-ring3"),
                                    pytest.param((2, 8, 5), id="pair-band8-ring5")])
def test_folded_batch_with_the_shallower_ring(gbs, config):
    """A batch of 1 to 3 rounds per network run with the operand ring one
    stage shallower, so that its grouped GEMMs of rounds 0 and 1 are the
    sampling variants with that ring: every network folds and the sums equal
    per-network runs bit for bit."""
    import torch
    sptr = torch.cuda.current_stream().cuda_stream
    defs = _uneven_defs()
    probe = gbs.gbs_make_network(defs[0].T, defs[0].r, "bf16x3", sptr)
    chunk = gbs.gbs_network_info(probe)[3]
    gbs.gbs_free_network(probe)
    E = [2 * chunk + 777, chunk + 5, 20000, chunk, 2 * chunk, 3 * chunk - 1]
    n_sub = [10, 8, 16, 4, 7, 16]
    K1 = [64, 128, 256, 512, 64, 256]
    seeds = [d.seed_s for d in defs]
    first = [17 * i for i in range(len(defs))]
    nets = [gbs.gbs_make_network(d.T, d.r, "bf16x3", sptr) for d in defs]
    for net in nets:
        gbs.gbs_set_sampler_fusion(net, 2)
    batch = gbs.gbs_make_batch(nets)
    gbs.gbs_set_batch_config(batch, *config)
    gbs.gbs_sample_batch(batch, seeds, first, E, n_sub, K1)
    got, rounds, _ = gbs.gbs_batch_info(batch)
    assert got == config and rounds == 3
    assert [gbs.gbs_sampler_fusion(n) for n in nets] == [e > chunk for e in E]
    for i, d in enumerate(defs):
        single = gbs.gbs_make_network(d.T, d.r, "bf16x3", sptr)
        gbs.gbs_sample(single, seeds[i], first[i], E[i], n_sub[i], K1[i])
        _, _, acc_b, cnt_b = gbs.gbs_get_accumulators(nets[i])
        _, _, acc_s, cnt_s = gbs.gbs_get_accumulators(single)
        gbs.gbs_free_network(single)
        assert np.array_equal(cnt_b, cnt_s), (config, i)
        assert np.array_equal(acc_b.view(np.float64), acc_s.view(np.float64)), (config, i)
    gbs.gbs_free_batch(batch)
    for n in nets:
        gbs.gbs_free_network(n)
