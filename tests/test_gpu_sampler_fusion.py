"""The sampler folded into the propagation GEMM (gbs_set_sampler_fusion):
gbs_sample over several chunks draws chunk i + 1's samples in the spare warps
of chunk i's GEMM.  The draws are the same Philox counters through the same
device code, so the sub-ensemble sums must equal those of the plain chunk
loop bit for bit, for one CTA per tile and CTA pairs, ragged last chunks and calls that
start mid-ensemble; the other entry points run unchanged after it.  Mode 2
folds on any network (these are small); mode 1, the default, only from 900
output modes.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gbs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_12749_gb300 as g
    g.build()
    return g


@pytest.fixture(scope="module")
def stream():
    import torch
    return torch.cuda.Stream().cuda_stream


def _sums(gbs, stream, net_def, fuse, config, calls, n_sub, K1):
    net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    gbs.gbs_set_gemm_config(net, *config)
    gbs.gbs_set_sampler_fusion(net, 2 if fuse else 0)
    for first, E in calls:
        gbs.gbs_sample(net, net_def.seed_s, first, E, n_sub, K1)
    active = gbs.gbs_sampler_fusion(net)
    _, _, acc, counts = gbs.gbs_get_accumulators(net)
    P = gbs.gbs_binned_counts(net, 0, K1)
    gbs.gbs_free_network(net)
    return acc, counts, P, active


@pytest.mark.parametrize("config", [pytest.param((1, 0, 0), id="cta"), pytest.param((2, 0, 0), id="pair"),
                                    pytest.param((1, 0, 16), id="cta-shallow-ring"),
                                    pytest.param((2, 0, 16), id="pair-shallow-ring")])
@pytest.mark.parametrize("N,M", [(24, 40), (300, 260)])
def test_folded_sampler_is_bitwise_the_plain_loop(gbs, stream, config, N, M):
    net_def = wl.small_network(N, M, r=0.7, t2=0.9, seed=90 + N)
    probe = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    chunk = gbs.gbs_network_info(probe)[3]
    gbs.gbs_free_network(probe)
    # 2 full chunks + a ragged one, then a call starting mid-ensemble that
    # covers one full chunk and a 1-trajectory tail
    calls = [(0, 2 * chunk + 12345), (2 * chunk + 12345, chunk + 1)]
    n_sub, K1 = 20, 256
    a0, c0, P0, act0 = _sums(gbs, stream, net_def, False, config, calls, n_sub, K1)
    a1, c1, P1, act1 = _sums(gbs, stream, net_def, True, config, calls, n_sub, K1)
    assert not act0
    assert act1, "folded sampler not taken"
    assert np.array_equal(c0, c1)
    assert np.array_equal(a0.view(np.float64), a1.view(np.float64))
    for x, y in zip(P0, P1):
        assert np.array_equal(x, y)
    assert abs(P1[0].sum() - 1.0) < 1e-9


def test_single_chunk_calls_and_other_entry_points_after_folding(gbs, stream):
    """E <= one chunk runs the plain loop; after a folded call the network's
    first operand is current again, so per-trajectory reads and the binned
    path agree with a network that never folded."""
    net_def = wl.small_network(64, 64, r=0.6, t2=0.95, seed=97)
    a = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    b = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    gbs.gbs_set_sampler_fusion(a, 2)
    gbs.gbs_set_sampler_fusion(b, 0)
    chunk = gbs.gbs_network_info(a)[3]
    for net in (a, b):
        gbs.gbs_sample(net, net_def.seed_s, 0, 3 * chunk, 10, 128)
        gbs.gbs_sample(net, net_def.seed_s, 3 * chunk, 5000, 10, 128)   # one chunk
    n_a, s_a = gbs.gbs_debug_samples(a, net_def.seed_s, 777, 3000)
    n_b, s_b = gbs.gbs_debug_samples(b, net_def.seed_s, 777, 3000)
    assert np.array_equal(n_a, n_b) and np.array_equal(s_a, s_b)
    Pa = gbs.gbs_binned_counts(a, 0, 128)
    Pb = gbs.gbs_binned_counts(b, 0, 128)
    for x, y in zip(Pa, Pb):
        assert np.array_equal(x, y)
    # the profile of a folded call: one standalone sampler launch
    gbs.gbs_profile_enable(a, True)
    gbs.gbs_sample(a, net_def.seed_s, 0, 3 * chunk, 10, 128)
    prof = gbs.gbs_profile_read(a)
    assert prof["sample"][1] == 1 and prof["gemm"][1] == 3
    gbs.gbs_free_network(a)
    gbs.gbs_free_network(b)


def test_fusion_switch_rejects_bad_values(gbs, stream):
    net_def = wl.small_network(16, 16, r=0.5, t2=0.9, seed=98)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    with pytest.raises(gbs.GbsError) as ei:
        gbs._check(gbs.lib().gbs_set_sampler_fusion(net.handle, 3))
    assert ei.value.code == gbs.GBS_EINVAL
    gbs.gbs_free_network(net)
    # FP64 networks never fold
    net = gbs.gbs_make_network(net_def.T, net_def.r, "fp64", stream)
    gbs.gbs_sample(net, net_def.seed_s, 0, 300000, 4, 64)
    assert not gbs.gbs_sampler_fusion(net)
    gbs.gbs_free_network(net)


def test_folded_sampler_in_moments_and_binned_paths(gbs, stream):
    """gbs_moments (the GEMM also writes every n'_i) and gbs_sample_nd (d
    output bins) fold the sampler the same way: bitwise the same results
    with it on and off."""
    net_def = wl.small_network(40, 48, r=0.6, t2=0.9, seed=99)
    res = {}
    for fuse in (False, True):
        net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
        gbs.gbs_set_sampler_fusion(net, 2 if fuse else 0)
        chunk = gbs.gbs_network_info(net)[3]
        E = 2 * chunk + 4321
        res[("mom", fuse)] = gbs.gbs_moments(net, net_def.seed_s, 11, E, 16, 3, 4)
        assert gbs.gbs_sampler_fusion(net) == fuse
        gbs.gbs_free_network(net)
        bins = [b % 3 for b in range(48)]
        net = gbs.gbs_make_network_binned(net_def.T, net_def.r, bins, "bf16x3", stream)
        gbs.gbs_set_sampler_fusion(net, 2 if fuse else 0)
        gbs.gbs_sample_nd(net, net_def.seed_s, 5, E, 12, (16, 16, 16))
        res[("nd", fuse)] = gbs.gbs_binned_counts_nd(net, (16, 16, 16), (0, 0, 0))
        assert gbs.gbs_sampler_fusion(net) == fuse
        gbs.gbs_free_network(net)
    for key in ("mom", "nd"):
        for x, y in zip(res[(key, False)], res[(key, True)]):
            assert np.array_equal(np.asarray(x), np.asarray(y)), key


def test_automatic_mode_folds_from_900_output_modes(gbs, stream):
    """Mode 1 (the default) folds the sampler for networks with at least 900
    output modes only: below that the GEMM of a chunk is too short to hide
    the next chunk's sampling."""
    for M, want in ((896, False), (960, True)):
        net_def = wl.small_network(32, M, r=0.5, t2=0.9, seed=100 + M)
        net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
        chunk = gbs.gbs_network_info(net)[3]
        gbs.gbs_sample(net, net_def.seed_s, 0, chunk + 1000, 8, 256)
        assert gbs.gbs_sampler_fusion(net) == want, M
        gbs.gbs_free_network(net)


def test_next_calls_first_chunk_drawn_ahead(gbs, stream):
    """A folded gbs_sample that continues the previous call (same seed,
    first = its first + E) draws, in its last GEMM, the chunk a following
    call from first + E starts with; that call skips its own sampler.  A call
    that does not continue the previous one (the first call, another start)
    draws nothing ahead.  Sums equal the plain loop's bit for bit for a
    following call that matches (same or smaller E), one that does not (other
    start), and one after another entry point overwrote the operands."""
    net_def = wl.small_network(40, 40, r=0.6, t2=0.9, seed=101)
    probe = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    chunk = gbs.gbs_network_info(probe)[3]
    gbs.gbs_free_network(probe)
    E = 3 * chunk + 999
    plan = [(0, E), (E, E), (2 * E, E // 2), (2 * E + E // 2 + 7, E), ("debug",),
            (3 * E + E // 2 + 7, E)]
    res = {}
    for mode in (0, 2):
        net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
        gbs.gbs_set_sampler_fusion(net, mode)
        gbs.gbs_profile_enable(net, True)
        launches = []
        for step in plan:
            if step[0] == "debug":
                gbs.gbs_debug_samples(net, net_def.seed_s, 5, 100)
                gbs.gbs_profile_read(net)  # its own sampler launch is not counted below
                continue
            gbs.gbs_sample(net, net_def.seed_s, step[0], step[1], 8, 128)
            launches.append(gbs.gbs_profile_read(net)["sample"][1])
        res[mode] = (gbs.gbs_get_accumulators(net), launches)
        gbs.gbs_free_network(net)
    (a0, l0), (a2, l2) = res[0], res[2]
    assert np.array_equal(a0[3], a2[3])
    assert np.array_equal(a0[2].view(np.float64), a2[2].view(np.float64))
    # sampler launches (the plain loop: one per chunk): the first call draws
    # nothing ahead, the second (continuing it) draws the third call's first
    # chunk, the fourth starts elsewhere, the last follows the fourth, which
    # drew nothing ahead (it did not continue the third)
    assert l2 == [1, 1, 0, 1, 1], l2
