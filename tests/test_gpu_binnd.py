"""Binning into d = 3 and 4 output bins on the GPU (gbs_make_network_binned,
gbs_sample_nd, gbs_binned_counts_nd) against the oracle (oracle/binnd.py) and
against fewer bins on the same trajectories.

Tolerances: FP64 path within 1e-9 of the oracle (FP64 throughout; only the
order of the sums differs); sums over a bin equal the runs with fewer bins on
the same trajectories within 1e-11 (1e-8 for merged bins on the BF16 path,
whose n_S are then summed in a different FP32 order); the BF16 path lies
within one sampling error of the FP64 path (|d| <= sigma, sigma floored at
1e-13).
"""
import numpy as np
import pytest

import oracle.binnd as bn
import workloads as wl

pytestmark = pytest.mark.gpu

BINS6 = [0, 0, 1, 1, 2, 2]


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


def _run(gbs, stream, net_def, bins, prec, E, n_sub, K, m_off=None, e0=0):
    net = gbs.gbs_make_network_binned(net_def.T, net_def.r, bins, prec, stream)
    gbs.gbs_sample_nd(net, net_def.seed_s, e0, E, n_sub, K)
    out = gbs.gbs_binned_counts_nd(net, K, m_off)
    gbs.gbs_free_network(net)
    return out


@pytest.mark.parametrize("bins,K,m_off", [
    (BINS6, (16, 16, 16), (1, 2, 0)),
    ([0, 1, 2, 0, 1, 2, 0, 1], (8, 16, 8), (0, 0, 3)),
    ([0, 0, 1, 1, 2, 2, 3, 3], (8, 8, 8, 8), (0, 1, 0, 2)),
])
def test_fp64_matches_oracle(orc, gbs, stream, bins, K, m_off):
    M = len(bins)
    net_def = wl.small_network(M, r=0.6, t2=0.9, seed=70 + M + len(K))
    E, n_sub, e0 = 1200, 5, 37
    P = _run(gbs, stream, net_def, bins, "fp64", E, n_sub, K, m_off, e0)
    Po, so = bn.run(net_def.T, net_def.r, net_def.seed_s, e0, E, n_sub, K, bins, m_off)
    for est in (0, 1):
        np.testing.assert_allclose(P[2 * est], Po[est], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(P[2 * est + 1], so[est], rtol=1e-7, atol=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_sums_over_a_bin_equal_fewer_bins(gbs, stream, prec):
    net_def = wl.small_network(6, r=0.7, t2=0.95, seed=81)
    E, n_sub, K = 4096, 8, 16
    P3 = _run(gbs, stream, net_def, BINS6, prec, E, n_sub, (K, K, K))
    # summing out bin 3 = bins 1 and 2 with bin 3's modes unobserved
    keep = [i for i, b in enumerate(BINS6) if b < 2]
    sub = wl.Network(T=np.ascontiguousarray(net_def.T[keep]), r=net_def.r, t2=-1.0,
                     seed_s=net_def.seed_s)
    P2 = _run(gbs, stream, sub, [BINS6[i] for i in keep], prec, E, n_sub, (K, K))
    for est in (0, 2):
        np.testing.assert_allclose(P3[est].sum(axis=2), P2[est], rtol=0, atol=1e-11)
    # merging bins 2 and 3: anti-diagonal sums.  On the BF16 path the merged
    # bin's n_S is summed over its modes within one GEMM tile in FP32, the
    # two bins' over two tiles whose partials are added in FP64, so the two
    # runs differ at FP32 rounding of n_S (~1e-7 relative), not at 1e-11
    merged = [0 if b == 0 else 1 for b in BINS6]
    Pm = _run(gbs, stream, net_def, merged, prec, E, n_sub, (K, K))
    tol = 1e-11 if prec == "fp64" else 1e-8
    for est in (0, 2):
        got = np.zeros((K, K))
        for m2 in range(K):
            for m3 in range(K):
                got[:, (m2 + m3) % K] += P3[est][:, m2, m3]
        np.testing.assert_allclose(got, Pm[est], rtol=0, atol=tol)


def test_bf16_within_sigma_of_fp64(gbs, stream):
    net_def = wl.small_network(12, r=0.6, t2=0.97, seed=82)
    bins = [0, 1, 2] * 4
    E, n_sub, K = 2 ** 14, 16, (16, 16, 16)
    P64 = _run(gbs, stream, net_def, bins, "fp64", E, n_sub, K)
    Pb = _run(gbs, stream, net_def, bins, "bf16x3", E, n_sub, K)
    for est in (0, 2):
        ratio = np.abs(Pb[est] - P64[est]) / np.maximum(P64[est + 1], 1e-13)
        assert ratio.max() <= 1.0, (est, ratio.max())
    assert abs(Pb[0].sum() - 1.0) < 1e-9


def test_two_bins_through_either_entry_point(gbs, stream):
    net_def = wl.small_network(8, r=0.5, t2=0.9, seed=83)
    bins = [0, 1, 1, 0, 1, 0, 0, 1]
    a = _run(gbs, stream, net_def, bins, "bf16x3", 3000, 6, (32, 16), (2, 1))
    net = gbs.gbs_make_network_binned(net_def.T, net_def.r, bins, "bf16x3", stream)
    gbs.gbs_sample_2d(net, net_def.seed_s, 0, 3000, 6, 32, 16)
    b = gbs.gbs_binned_counts_2d(net, 32, 16, 2, 1)
    gbs.gbs_free_network(net)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_lossless_odd_totals_vanish(gbs, stream):
    net_def = wl.small_network(6, r=0.5, t2=1.0, seed=84)
    for prec, tol in (("fp64", 1e-12), ("bf16x3", 1e-4)):
        P = _run(gbs, stream, net_def, BINS6, prec, 2000, 8, (16, 16, 16))
        m = np.indices((16, 16, 16))
        odd = m.sum(axis=0) % 2 == 1
        assert np.max(np.abs(P[0][odd])) < tol, prec


def test_invalid_calls(gbs, stream):
    net_def = wl.small_network(6, r=0.5, t2=0.9, seed=85)
    for bins in ([0, 0, 1, 1, 2, 4], [0, 0, 2, 2, 2, 0], [0] * 6):
        with pytest.raises(gbs.GbsError) as ei:
            gbs.gbs_make_network_binned(net_def.T, net_def.r, bins, "fp64", stream)
        assert ei.value.code == gbs.GBS_EINVAL
    net = gbs.gbs_make_network_binned(net_def.T, net_def.r, BINS6, "bf16x3", stream)
    for K in ((16, 12, 16), (1, 16, 16), (256, 256, 128)):
        with pytest.raises(gbs.GbsError) as ei:
            gbs.gbs_sample_nd(net, 1, 0, 100, 4, K)
        assert ei.value.code == gbs.GBS_EINVAL
    with pytest.raises(gbs.GbsError) as ei:
        gbs.gbs_sample_2d(net, 1, 0, 100, 4, 16, 16)    # three bins
    assert ei.value.code == gbs.GBS_EINVAL
    gbs.gbs_free_network(net)
    plain = gbs.gbs_make_network(net_def.T, net_def.r, "fp64", stream)
    with pytest.raises(gbs.GbsError) as ei:
        gbs.gbs_sample_nd(plain, 1, 0, 100, 4, (16, 16))
    assert ei.value.code == gbs.GBS_EINVAL
    gbs.gbs_free_network(plain)
