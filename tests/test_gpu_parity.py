"""CUDA path vs the CPU oracle, element by element on the same seeded inputs.

Tolerances:
  * FP64 path: per-trajectory n, n_S and generating-function values within
    1e-10 relative (absolute floor 2^-55 for values the kernels skip below
    2^-60); P(m) within 1e-10.
  * BF16 split paths: per-trajectory n_S within c * 2^-p * S, where
    S = sum_i |alpha'_i| |beta'_i| is the natural error scale of the sum
    and p = 14 (3 products) or 20 (6 products) from the split arithmetic
    (dropped cross terms ~2^-17 / 2^-25 relative plus FP32 accumulation);
    P(m) within one sampling error of the FP64 result on the same
    trajectories (|dP| <= sigma, sigma floored at 1e-13).
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


@pytest.fixture(scope="module")
def stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _amp_scale(net, e_list):
    """S_e = sum_i |alpha'_i| |beta'_i| from the oracle, per trajectory."""
    out = []
    for e in e_list:
        _, _, ap, bp = oracle.sample_amplitudes(net.T, net.r, net.seed_s, int(e))
        out.append(float(np.sum(np.abs(ap) * np.abs(bp))))
    return np.array(out)


# ---------------------------------------------------------------------------
# per-trajectory parity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(16, 16), (7, 9), (9, 7), (1, 1), (100, 130), (257, 200)])
def test_fp64_per_sample_totals(gbs, stream, shape):
    N, M = shape
    net_def = wl.small_network(N, M=M, r=0.7, t2=0.9, seed=N + M)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "fp64", stream)
    E = 300
    e0 = 12345
    n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, e0, E)
    no, nSo = oracle.samples(net_def.T, net_def.r, net_def.seed_s, e0, E)
    scale_n = np.maximum(np.abs(no), 1.0)
    assert np.max(np.abs(n - no) / scale_n) < 1e-10
    scale = np.maximum(np.abs(nSo), 1.0)
    assert np.max(np.abs(nS - nSo) / scale) < 1e-10
    gbs.gbs_free_network(net)


def test_fp64_per_sample_gf(gbs, stream):
    """n_sub = E: every trajectory is its own sub-ensemble, so the sums are
    the per-trajectory generating functions at all K1 points."""
    for general in (False, True):
        net_def = wl.small_network(10, r=[0.3, 0.9, 0.5, 1.2, 0.7, 0.2, 0.8, 1.0, 0.4, 0.6],
                                   t2=0.85, seed=3, general_loss=general)
        E, K1 = 256, 128
        net = gbs.gbs_make_network(net_def.T, net_def.r, "fp64", stream)
        gbs.gbs_sample(net, net_def.seed_s, 0, E, E, K1)
        _, _, acc, cnt = gbs.gbs_get_accumulators(net)
        assert np.all(cnt == 1)
        n, nS = oracle.samples(net_def.T, net_def.r, net_def.seed_s, 0, E)
        for e in range(E):
            gm, gp = oracle.gf_sample(n[e], nS[e], K1)
            for got, want in ((acc[0, e], gm), (acc[1, e], gp)):
                err = np.abs(got - want)
                assert np.all(err <= 1e-10 * np.abs(want) + 2.0 ** -55), (general, e, err.max())
        gbs.gbs_free_network(net)


# Per-term bound of the split paths' generating functions: 1e-11 relative
# plus an absolute floor of 2^-46.  Every term enters the sub-ensemble sums,
# and so P(m), with its absolute error; 2^-46 is the rounding the
# double-float evaluation commits on terms of order one, so terms below
# 2^-27, evaluated with FP32 exp and sin/cos (relative error below 2^-20.5),
# stay within it.
GF_TERM_FLOOR = 2.0 ** -46


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_split_path_per_sample_gf(gbs, stream, prec):
    """The BF16 paths evaluate the generating functions in double-float
    (FP32 for terms below 2^-27): per trajectory (n_sub = E) they match the
    oracle's FP64 formula applied to the device's own n, n_S within 1e-11
    relative plus GF_TERM_FLOOR, including negative n and complex n_S
    (non-uniform loss)."""
    for general in (False, True):
        net_def = wl.small_network(10, r=[0.3, 0.9, 0.5, 1.2, 0.7, 0.2, 0.8, 1.0, 0.4, 0.6],
                                   t2=0.85, seed=3, general_loss=general)
        E, K1 = 256, 128
        net = gbs.gbs_make_network(net_def.T, net_def.r, prec, stream)
        n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, 0, E)
        gbs.gbs_sample(net, net_def.seed_s, 0, E, E, K1)
        _, _, acc, cnt = gbs.gbs_get_accumulators(net)
        for e in range(E):
            gm, gp = oracle.gf_sample(n[e], nS[e], K1)
            for got, want in ((acc[0, e], gm), (acc[1, e], gp)):
                err = np.abs(got - want)
                assert np.all(err <= 1e-11 * np.abs(want) + GF_TERM_FLOOR), (general, e, err.max())
        gbs.gbs_free_network(net)


@pytest.mark.parametrize("K1", [2, 4, 8, 64])
def test_split_path_per_sample_gf_small_K1(gbs, stream, K1):
    """The double-float kernel at the smallest DFT sizes: every k pairs with
    K1 - k, k = 0 and K1/2 with themselves, and the windows cover the whole
    circle; per trajectory (n_sub = E, a ragged count of trajectories) the
    same per-term bound as above, uniform and non-uniform loss."""
    for general in (False, True):
        net_def = wl.small_network(3, r=[0.5, 1.0, 0.2], t2=0.9, seed=13, general_loss=general)
        E = 37
        net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
        n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, 0, E)
        gbs.gbs_sample(net, net_def.seed_s, 0, E, E, K1)
        _, _, acc, cnt = gbs.gbs_get_accumulators(net)
        gbs.gbs_free_network(net)
        assert np.all(cnt == 1)
        for e in range(E):
            gm, gp = oracle.gf_sample(n[e], nS[e], K1)
            for got, want in ((acc[0, e], gm), (acc[1, e], gp)):
                err = np.abs(got - want)
                assert np.all(err <= 1e-11 * np.abs(want) + GF_TERM_FLOOR), (K1, general, e)


def test_split_path_gf_sums_over_many_tiles(gbs, stream):
    """Sub-ensembles of 700 trajectories (two whole 256-trajectory tiles of
    the double-float kernel and a ragged third, partials flushed to FP64 in
    between): the device's sums against the oracle's sums of its FP64 terms
    at the device's own n, n_S, within the per-term bound summed (|G| <= 1 on
    uniform-loss trajectories)."""
    net_def = wl.small_network(16, r=1.0, t2=0.9, seed=17)
    E, n_sub, K1 = 2800, 4, 256
    net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, 0, E)
    gbs.gbs_sample(net, net_def.seed_s, 0, E, n_sub, K1)
    _, _, acc, cnt = gbs.gbs_get_accumulators(net)
    gbs.gbs_free_network(net)
    want, cnt_o = oracle.accumulate_gf(n, nS, 0, n_sub, K1)
    assert np.array_equal(cnt, cnt_o)
    tol = (1e-11 + GF_TERM_FLOOR) * cnt[None, :, None]
    assert np.all(np.abs(acc - want) <= tol), float(np.max(np.abs(acc - want)))


@pytest.mark.parametrize("general", [False, True])
def test_split_path_per_sample_gf_large_totals(gbs, stream, general):
    """The same per-term bound at photon totals of a few hundred (phases of
    ~10^2 rad at the window edges, a third of the in-window terms below
    2^-27): every term, including the smallest in-window ones, against the
    oracle's FP64 formula."""
    net_def = wl.small_network(256, r=1.0, t2=0.95, seed=31, general_loss=general)
    E, K1 = 64, 4096
    net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, 0, E)
    assert np.min(nS.real) > 150.0
    gbs.gbs_sample(net, net_def.seed_s, 0, E, E, K1)
    _, _, acc, _ = gbs.gbs_get_accumulators(net)
    small = 0
    for e in range(E):
        gm, gp = oracle.gf_sample(n[e], nS[e], K1)
        small += int(np.sum((np.abs(gp) < 2.0 ** -27) & (np.abs(gp) > 2.0 ** -60)))
        for got, want in ((acc[0, e], gm), (acc[1, e], gp)):
            err = np.abs(got - want)
            assert np.all(err <= 1e-11 * np.abs(want) + GF_TERM_FLOOR), (general, e, err.max())
    assert small > 1000  # the FP32 small-term path was exercised
    gbs.gbs_free_network(net)


def test_fp64_distribution_matches_oracle(gbs, stream):
    w = wl.SMALL16
    net_def = w.network()
    net = gbs.gbs_make_network(net_def.T, net_def.r, "fp64", stream)
    gbs.gbs_sample(net, net_def.seed_s, 0, w.E, w.n_sub, w.K1)
    P_mP, s_mP, P_pP, s_pP = gbs.gbs_binned_counts(net, 0, w.K1)
    Po, so, _ = oracle.run(net_def.T, net_def.r, net_def.seed_s, 0, w.E, w.n_sub, w.K1)
    np.testing.assert_allclose(P_mP, Po[0], rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(P_pP, Po[1], rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(s_mP, so[0], rtol=1e-7, atol=1e-12)
    np.testing.assert_allclose(s_pP, so[1], rtol=1e-7, atol=1e-12)
    # and against the exact (aliased) distribution within sampling error
    Pex = ex.exact_distribution(ex.eigenvalues_uniform_loss(net_def.r, w.t2), w.K1).real
    res = agreement(P_mP, s_mP, Pex)
    assert res["ok"], res
    gbs.gbs_free_network(net)


@pytest.mark.parametrize("prec,p", [("bf16x3", 14), ("bf16x6", 20)])
@pytest.mark.parametrize("shape", [(16, 16), (7, 9), (100, 130), (300, 257)])
def test_bf16_per_sample_totals(gbs, stream, prec, p, shape):
    N, M = shape
    net_def = wl.small_network(N, M=M, r=0.9, t2=0.95, seed=7 + N)
    net = gbs.gbs_make_network(net_def.T, net_def.r, prec, stream)
    E = 200  # spans two 128-trajectory tiles with a ragged tail
    e0 = 777
    n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, e0, E)
    no, nSo = oracle.samples(net_def.T, net_def.r, net_def.seed_s, e0, E)
    S = _amp_scale(net_def, range(e0, e0 + E))
    err = np.abs(nS - nSo)
    assert np.all(err <= 2.0 ** -p * S + 1e-12), (err / S).max()
    # n: FP32 sampler arithmetic with a compensated sum
    assert np.max(np.abs(n - no) / np.maximum(np.abs(no), 1.0)) < 1e-5
    gbs.gbs_free_network(net)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_bf16_distribution_within_sigma_of_fp64(gbs, stream, prec):
    """The accuracy gate |dP|/sigma <= 1 between precisions on the same trajectories."""
    for net_def, E, n_sub, K1 in (
            (wl.SMALL16.network(), 2 ** 14, 16, 64),
            (wl.small_network(200, r=0.5, t2=0.99, seed=11), 2 ** 14, 32, 256)):
        res = {}
        for pr in ("fp64", prec):
            net = gbs.gbs_make_network(net_def.T, net_def.r, pr, stream)
            gbs.gbs_sample(net, net_def.seed_s, 0, E, n_sub, K1)
            res[pr] = gbs.gbs_binned_counts(net, 0, K1)
            gbs.gbs_free_network(net)
        for est in (0, 2):
            P64, s64 = res["fp64"][est], res["fp64"][est + 1]
            Pb = res[prec][est]
            ratio = np.abs(Pb - P64) / np.maximum(s64, 1e-13)
            assert ratio.max() <= 1.0, (prec, est, ratio.max())


def test_uniform_loss_identity_gpu(gbs, stream):
    """n_S = t^2 n for T = t U on the device, relative to the amplitude scale
    S = sum_i |alpha'_i||beta'_i| (T is rounded to FP32 on the BF16 paths, so
    T^T T* = t^2 I holds there only to ~2^-24 sqrt(N))."""
    net_def = wl.small_network(64, r=0.9, t2=0.93, seed=21)
    E = 300
    S = _amp_scale(net_def, range(E))
    for prec, tol in (("fp64", 1e-13), ("bf16x3", 2.0 ** -14), ("bf16x6", 2.0 ** -20)):
        net = gbs.gbs_make_network(net_def.T, net_def.r, prec, stream)
        n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, 0, E)
        assert np.max(np.abs(nS - 0.93 * n) / S) < tol, prec
        gbs.gbs_free_network(net)


# ---------------------------------------------------------------------------
# edge cases and API behaviour
# ---------------------------------------------------------------------------
def test_split_calls_equal_one_call(gbs, stream):
    """Calls continue the counter stream; splitting a call at its own chunk
    boundaries (a call of E cuts the fewest chunks of at most the network's
    chunk size: the even split rounded up to a multiple of 128, the last
    chunk shorter) is bitwise identical, any split agrees to rounding;
    get/set round-trips."""
    net_def = wl.small_network(40, r=0.8, t2=0.9, seed=5)
    for prec in ("fp64", "bf16x3"):
        net = gbs.gbs_make_network(net_def.T, net_def.r, prec, stream)
        chunk = gbs.gbs_network_info(net)[3]
        E = 2 * chunk + 77
        nch = -(-E // chunk)
        step = min(chunk, -(-(-(-E // nch)) // 128) * 128)
        assert step % 128 == 0 and -(-E // step) == nch
        gbs.gbs_sample(net, net_def.seed_s, 0, E, 8, 128)
        _, _, acc1, cnt1 = gbs.gbs_get_accumulators(net)
        gbs.gbs_reset(net)
        for f in range(0, E, step):
            gbs.gbs_sample(net, net_def.seed_s, f, min(step, E - f), 8, 128)
        _, _, acc2, cnt2 = gbs.gbs_get_accumulators(net)
        assert np.array_equal(cnt1, cnt2)
        assert np.array_equal(acc1, acc2)
        gbs.gbs_reset(net)
        gbs.gbs_sample(net, net_def.seed_s, 0, 1000, 8, 128)
        gbs.gbs_sample(net, net_def.seed_s, 1000, E - 1000, 8, 128)
        _, _, acc3, cnt3 = gbs.gbs_get_accumulators(net)
        assert np.array_equal(cnt1, cnt3)
        np.testing.assert_allclose(acc3, acc1, rtol=1e-11, atol=1e-9)
        # resume from saved accumulators
        net2 = gbs.gbs_make_network(net_def.T, net_def.r, prec, stream)
        gbs.gbs_set_accumulators(net2, acc1, cnt1)
        r1 = gbs.gbs_binned_counts(net, 0, 128)
        r2 = gbs.gbs_binned_counts(net2, 0, 128)
        gbs.gbs_reset(net)
        gbs.gbs_set_accumulators(net, acc1, cnt1)
        r3 = gbs.gbs_binned_counts(net, 0, 128)
        for a, b in zip(r2, r3):
            assert np.array_equal(a, b)
        gbs.gbs_free_network(net)
        gbs.gbs_free_network(net2)


def test_edge_cases(gbs, stream):
    net_def = wl.small_network(5, r=0.6, t2=0.8, seed=9)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "fp64", stream)
    gbs.gbs_sample(net, net_def.seed_s, 0, 0, 4, 16)     # E = 0 is a no-op
    with pytest.raises(gbs.GbsError):                     # sub-ensembles still empty
        gbs.gbs_binned_counts(net, 0, 16)
    gbs.gbs_sample(net, net_def.seed_s, 0, 3, 4, 16)     # fewer samples than sub-ensembles
    with pytest.raises(gbs.GbsError):
        gbs.gbs_binned_counts(net, 0, 16)
    gbs.gbs_sample(net, net_def.seed_s, 3, 1, 4, 16)
    P = gbs.gbs_binned_counts(net, 0, 16)
    assert abs(P[0].sum() - 1.0) < 1e-12
    with pytest.raises(gbs.GbsError):                     # K1 must stay fixed
        gbs.gbs_sample(net, net_def.seed_s, 4, 10, 4, 32)
    gbs.gbs_free_network(net)
    # K1 = 2, one mode, window offset
    net_def = wl.small_network(1, r=0.4, t2=1.0, seed=10)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "fp64", stream)
    gbs.gbs_sample(net, net_def.seed_s, 0, 1000, 10, 2)
    P = gbs.gbs_binned_counts(net, 5, 2)
    Po, _, _ = oracle.run(net_def.T, net_def.r, net_def.seed_s, 0, 1000, 10, 2, 5)
    np.testing.assert_allclose(P[0], Po[0], atol=1e-12)
    gbs.gbs_free_network(net)


def test_invalid_arguments_are_rejected(gbs, stream):
    T = wl.small_network(4, r=0.5, seed=1).T
    for args in ((T, np.array([0.5, -0.1, 0.2, 0.3])),        # r < 0
                 (T, np.array([0.5, np.nan, 0.2, 0.3]))):     # non-finite r
        with pytest.raises(gbs.GbsError) as ei:
            gbs.gbs_make_network(*args, "fp64", stream)
        assert ei.value.code == gbs.GBS_EINVAL
    with pytest.raises(gbs.GbsError):
        gbs.gbs_make_network(T, np.full(4, 0.5), 7, stream)  # unknown precision
    net = gbs.gbs_make_network(T, np.full(4, 0.5), "fp64", stream)
    for n_sub, K1 in ((4, 24), (0, 16), (4, 1), (70000, 16)):
        with pytest.raises(gbs.GbsError) as ei:
            gbs.gbs_sample(net, 1, 0, 10, n_sub, K1)
        assert ei.value.code == gbs.GBS_EINVAL
    with pytest.raises(gbs.GbsError):
        gbs.gbs_sample(net, 1, 0, -5, 4, 16)
    gbs.gbs_free_network(net)


def test_lossless_odd_bins_vanish(gbs, stream):
    """Lossless, all modes counted: odd-count probabilities vanish per
    trajectory (text after Eq. c-number-variable), here to rounding."""
    net_def = wl.small_network(24, r=0.6, t2=1.0, seed=12)
    for prec, tol in (("fp64", 1e-13), ("bf16x3", 1e-4)):
        net = gbs.gbs_make_network(net_def.T, net_def.r, prec, stream)
        gbs.gbs_sample(net, net_def.seed_s, 0, 2 ** 13, 16, 128)
        P = gbs.gbs_binned_counts(net, 0, 128)[0]
        assert np.max(np.abs(P[1::2])) < tol, prec
        gbs.gbs_free_network(net)
