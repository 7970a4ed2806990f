"""Normally-ordered moments and single-mode marginals on the GPU
(gbs_moments, gbs_debug_occupations) against the oracle (oracle/moments.py).

Tolerances:
  * per-mode occupations n'_j: FP64 path within 1e-10 of the amplitude
    scale A_j B_j, A_j = sum_k |T_jk| |alpha_k|, B_j = sum_k |T_jk| |beta_k|;
    BF16 split paths within 2^-14 (3 products) / 2^-20 (6 products) of it,
    the bounds of the per-trajectory totals applied to one mode;
  * FP64 path: moments, marginals and their errors within 1e-9 relative
    (FP64 throughout; only the order of the sums differs);
  * BF16 paths: within one sampling error of the FP64 result on the same
    trajectories (|d| <= sigma, sigma floored at 1e-13), the gate used for
    the count distribution.
"""
import numpy as np
import pytest

import oracle
import oracle.moments as mo
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


def _amp_scale(net_def, e_list):
    """[M][len(e_list)]: A_j B_j per trajectory."""
    absT = np.abs(net_def.T)
    out = []
    for e in e_list:
        a, b, _, _ = oracle.sample_amplitudes(net_def.T, net_def.r, net_def.seed_s, int(e))
        out.append((absT @ np.abs(a)) * (absT @ np.abs(b)))
    return np.array(out).T


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16x3", 2.0 ** -14),
                                      ("bf16x6", 2.0 ** -20), ("fp32", None)])
@pytest.mark.parametrize("shape", [(16, 16), (7, 9), (9, 7), (100, 130)])
def test_occupations_per_element(gbs, stream, prec, tol, shape):
    N, M = shape
    if tol is None:
        # FP32 GEMM: |d n'_j| <= 2 (N + 2) 2^-24 (1 + 2^-10) A_j B_j (rounding
        # of T and the samples to FP32, N fused multiply-adds)
        tol = 2.0 * (N + 2) * 2.0 ** -24 * (1.0 + 2.0 ** -10)
    net_def = wl.small_network(N, M=M, r=0.9, t2=0.95, seed=40 + N)
    net = gbs.gbs_make_network(net_def.T, net_def.r, prec, stream)
    E, e0 = 200, 777  # two 128-trajectory tiles, ragged tail
    occ = gbs.gbs_debug_occupations(net, net_def.seed_s, e0, E)
    _, occo = mo.mode_samples(net_def.T, net_def.r, net_def.seed_s, e0, E)
    S = _amp_scale(net_def, range(e0, e0 + E))
    err = np.abs(occ - occo.T)
    assert np.all(err <= tol * S + 1e-300), (err / S).max()
    gbs.gbs_free_network(net)


def _compare_fp64(got, want):
    for g_, w_ in zip(got, want):
        scale = max(np.max(np.abs(w_)), 1e-300)
        np.testing.assert_allclose(g_, w_, rtol=1e-9, atol=1e-12 * scale)


@pytest.mark.parametrize("shape,E,e0,n_sub,mmax,cmax", [
    ((16, 16), 3000, 5, 7, 5, 9),      # replicas of every sub-ensemble, (8, 15) tables
    ((9, 7), 1200, 123, 300, 4, 7),    # n_sub > 256: whole sub-ensembles per thread
    ((16, 16), 640, 0, 160, 2, 3),     # 128 < n_sub <= 256
    ((1, 1), 257, 3, 1, 8, 15),        # one sub-ensemble, zero errors
])
def test_fp64_matches_oracle(gbs, stream, shape, E, e0, n_sub, mmax, cmax):
    N, M = shape
    net_def = wl.small_network(N, M=M, r=0.8, t2=0.9, seed=50 + N + M)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "fp64", stream)
    got = gbs.gbs_moments(net, net_def.seed_s, e0, E, n_sub, mmax, cmax)
    want = mo.run(net_def.T, net_def.r, net_def.seed_s, e0, E, n_sub, mmax, cmax)
    _compare_fp64(got, want)
    if n_sub == 1:
        assert np.all(got[1] == 0.0) and np.all(got[3] == 0.0)
    gbs.gbs_free_network(net)


def test_one_trajectory_per_sub_ensemble(gbs, stream):
    net_def = wl.small_network(16, r=0.7, t2=0.9, seed=60)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "fp64", stream)
    got = gbs.gbs_moments(net, net_def.seed_s, 9, 37, 37, 3, 4)
    want = mo.run(net_def.T, net_def.r, net_def.seed_s, 9, 37, 37, 3, 4)
    _compare_fp64(got, want)
    gbs.gbs_free_network(net)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6", "fp32"])
def test_reduced_precision_within_sigma_of_fp64(gbs, stream, prec):
    for net_def, E, n_sub in ((wl.SMALL16.network(), 2 ** 14, 16),
                              (wl.small_network(200, r=0.5, t2=0.99, seed=11), 2 ** 14, 32)):
        res = {}
        for pr in ("fp64", prec):
            net = gbs.gbs_make_network(net_def.T, net_def.r, pr, stream)
            res[pr] = gbs.gbs_moments(net, net_def.seed_s, 0, E, n_sub, 4, 7)
            gbs.gbs_free_network(net)
        for k in (0, 2):
            d = np.abs(res[prec][k] - res["fp64"][k])
            ratio = d / np.maximum(res["fp64"][k + 1], 1e-13)
            assert ratio.max() <= 1.0, (prec, k, ratio.max())


def test_large_occupations_take_the_fp64_route(gbs, stream):
    # r = 2.4: |n'_j| > 40 in a good fraction of trajectories
    net_def = wl.small_network(4, r=2.4, t2=0.95, seed=70)
    E, n_sub = 2048, 16
    net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    occ = gbs.gbs_debug_occupations(net, net_def.seed_s, 0, E)
    assert np.mean(np.abs(occ) > 40.0) > 0.02
    got = gbs.gbs_moments(net, net_def.seed_s, 0, E, n_sub, 3, 6)
    gbs.gbs_free_network(net)
    want = mo.run(net_def.T, net_def.r, net_def.seed_s, 0, E, n_sub, 3, 6)
    for k in (0, 2):
        assert np.all(np.isfinite(got[k]))
        ratio = np.abs(got[k] - want[k]) / np.maximum(want[k + 1], 1e-13)
        assert ratio.max() <= 1.0, (k, ratio.max())


def test_sums_over_modes_are_the_total_count_moment(gbs, stream):
    """sum_j <n'_j> over the same trajectories = the mean of Re n_S (gbs_debug_samples)."""
    net_def = wl.small_network(100, M=130, r=0.9, t2=0.95, seed=80)
    E, n_sub = 1000, 10
    for prec, tol in (("fp64", 1e-12), ("bf16x3", 1e-5)):
        net = gbs.gbs_make_network(net_def.T, net_def.r, prec, stream)
        mom, _, _, _ = gbs.gbs_moments(net, net_def.seed_s, 0, E, n_sub, 1, 0)
        n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, 0, E)
        gbs.gbs_free_network(net)
        sub = np.arange(E) % n_sub
        want_p = np.mean([nS[sub == q].real.mean() for q in range(n_sub)])
        want_m = np.mean([(np.tanh(n[sub == q]) * nS[sub == q].real).mean() for q in range(n_sub)])
        assert abs(mom[1, :, 0].sum() - want_p) <= tol * abs(want_p), prec
        assert abs(mom[0, :, 0].sum() - want_m) <= tol * max(abs(want_m), abs(want_p)), prec


def test_single_lossless_mode(gbs, stream):
    net_def = wl.small_network(1, r=0.7, t2=1.0, seed=3)
    for prec, tol in (("fp64", 1e-14), ("bf16x3", 1e-5)):
        net = gbs.gbs_make_network(net_def.T, net_def.r, prec, stream)
        _, _, marg, _ = gbs.gbs_moments(net, net_def.seed_s, 0, 4096, 8, 2, 7)
        gbs.gbs_free_network(net)
        assert np.max(np.abs(marg[0, 0, 1::2])) < tol, prec     # odd counts vanish exactly
        assert abs(marg[0, 0, 0::2].sum() - 1.0) < 0.05        # mass in c <= 7


def test_repeatable_and_independent_of_the_sums(gbs, stream):
    net_def = wl.small_network(16, r=0.7, t2=0.9, seed=61)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    a = gbs.gbs_moments(net, net_def.seed_s, 0, 5000, 10, 4, 7)
    gbs.gbs_sample(net, net_def.seed_s, 0, 3000, 10, 64)
    b = gbs.gbs_moments(net, net_def.seed_s, 0, 5000, 10, 4, 7)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    gbs.gbs_free_network(net)


def test_invalid_arguments_are_rejected(gbs, stream):
    net_def = wl.small_network(8, r=0.5, t2=0.9, seed=62)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", stream)
    for args in ((100, 4, 0, 4), (100, 4, 9, 4), (100, 4, 2, -1), (100, 4, 2, 16), (100, 0, 2, 2),
                 (3, 4, 2, 2)):
        E, n_sub, mmax, cmax = args
        with pytest.raises(gbs.GbsError) as ei:
            gbs.gbs_moments(net, 1, 0, E, n_sub, mmax, cmax)
        assert ei.value.code == gbs.GBS_EINVAL
    gbs.gbs_free_network(net)
    bins = [0, 0, 0, 0, 1, 1, 1, 1]
    netb = gbs.gbs_make_network_binned(net_def.T, net_def.r, bins, "fp64", stream)
    with pytest.raises(gbs.GbsError) as ei:
        gbs.gbs_moments(netb, 1, 0, 100, 4, 2, 2)
    assert ei.value.code == gbs.GBS_EINVAL
    gbs.gbs_free_network(netb)


@pytest.mark.slow
def test_full_size_m1000(gbs):
    """The bench workload (N = M = 1000, BF16x3, 10^6 trajectories, N_R = 100):
    sampled trajectories element by element against the oracle, and every
    mode's moments and marginals within sampling error of the exact Gaussian
    values."""
    import torch
    w = wl.M1000
    net_def = w.network()
    s = torch.cuda.Stream()
    net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", s.cuda_stream)
    for e in (0, 131071, 131072, w.E - 1):
        occ = gbs.gbs_debug_occupations(net, net_def.seed_s, e, 1)
        _, occo = mo.mode_samples(net_def.T, net_def.r, net_def.seed_s, e, 1)
        S = _amp_scale(net_def, [e])
        assert np.all(np.abs(occ - occo.T) <= 2.0 ** -14 * S), e
    mmax, cmax = 4, 7
    mom, smom, marg, smarg = gbs.gbs_moments(net, net_def.seed_s, 0, w.E, w.n_sub, mmax, cmax)
    gbs.gbs_free_network(net)
    emom = mo.exact_moments(net_def.T, net_def.r, mmax)
    emarg = mo.exact_marginals(net_def.T, net_def.r, cmax)
    res = agreement(mom[0].ravel(), smom[0].ravel(), emom.ravel(), bulk=0.0)
    assert res["ok"], res
    res = agreement(marg[0].ravel(), smarg[0].ravel(), emarg.ravel(), bulk=1e-4)
    assert res["ok"], res
