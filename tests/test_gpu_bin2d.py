"""Two-bin (d = 2) distributions on the GPU against the oracle
(oracle/bin2d.py) on the same seeded inputs, and the identities that tie them
to the one-bin estimator; the paper's 200-mode example ("Higher-dimensional
binning", Fig. 3: lossless, r = 0.5, bins of 100 modes, 1.2e6 samples,
sampling errors < 3e-5) at full size."""
import numpy as np
import pytest

import oracle.bin2d as b2
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


@pytest.mark.parametrize("bins", [[0] * 6 + [1] * 6, [0, 1] * 6, [1, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 0]])
def test_fp64_matches_oracle(orc, gbs, stream, bins):
    net_def = wl.small_network(12, r=0.7, t2=0.9, seed=14)
    E, n_sub, K = 4000, 8, 32
    net = gbs.gbs_make_network_binned(net_def.T, net_def.r, bins, "fp64", stream)
    gbs.gbs_sample_2d(net, net_def.seed_s, 5, E, n_sub, K, K)
    P = gbs.gbs_binned_counts_2d(net, K, K)
    gbs.gbs_free_network(net)
    Po, so = b2.run(net_def.T, net_def.r, net_def.seed_s, 5, E, n_sub, K, K, bins)
    for est in (0, 1):
        np.testing.assert_allclose(P[2 * est], Po[est], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(P[2 * est + 1], so[est], rtol=1e-7, atol=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "fp32"])
def test_antidiagonal_sums_equal_the_total_count(gbs, stream, prec):
    """Sum over m_1 + m_2 = m (mod K) of the two-bin P equals the one-bin P of
    the same trajectories (gbs_sample on the same binned network)."""
    net_def = wl.small_network(100, M=90, r=0.6, t2=0.93, seed=15)
    bins = [i % 3 == 0 for i in range(90)]
    E, n_sub, K = 20000, 16, 128
    net = gbs.gbs_make_network_binned(net_def.T, net_def.r, np.array(bins, dtype=int), prec,
                                      stream)
    gbs.gbs_sample_2d(net, net_def.seed_s, 0, E, n_sub, K, K)
    gbs.gbs_sample(net, net_def.seed_s, 0, E, n_sub, K)
    P2 = gbs.gbs_binned_counts_2d(net, K, K)
    P1 = gbs.gbs_binned_counts(net, 0, K)
    gbs.gbs_free_network(net)
    m1, m2 = np.meshgrid(np.arange(K), np.arange(K), indexing="ij")
    for est in (0, 1):
        diag = np.bincount(((m1 + m2) % K).ravel(), weights=P2[2 * est].ravel(), minlength=K)
        np.testing.assert_allclose(diag, P1[2 * est], rtol=0, atol=1e-11)


def test_invalid_calls(gbs, stream):
    net_def = wl.small_network(8, r=0.5, t2=0.9, seed=16)
    with pytest.raises(gbs.GbsError):
        gbs.gbs_make_network_binned(net_def.T, net_def.r, [0] * 8, "fp64", stream)  # one bin
    with pytest.raises(gbs.GbsError):
        gbs.gbs_make_network_binned(net_def.T, net_def.r, [0, 2] * 4, "fp64", stream)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "fp64", stream)
    with pytest.raises(gbs.GbsError):
        gbs.gbs_sample_2d(net, 1, 0, 100, 4, 16, 16)  # not a binned network
    gbs.gbs_free_network(net)
    net = gbs.gbs_make_network_binned(net_def.T, net_def.r, [0, 1] * 4, "fp64", stream)
    with pytest.raises(gbs.GbsError):
        gbs.gbs_sample_2d(net, 1, 0, 100, 4, 16, 24)  # K2 not a power of two
    with pytest.raises(gbs.GbsError):
        gbs.gbs_binned_counts_2d(net, 16, 16)         # nothing sampled yet
    gbs.gbs_free_network(net)


@pytest.mark.slow
def test_paper_200_mode_example(gbs, stream):
    """Lossless 200-mode Haar network, r = 0.5, bins {1..100}, {101..200},
    1.2e6 samples: max sampling error below the paper's 3e-5, odd totals
    vanish, and the anti-diagonal sums match the exact negative binomial."""
    M, r, E, n_sub, K = 200, 0.5, 1_200_000, 100, 128
    U = wl.haar_unitary(M, wl.SEED_U_BASE + 200)
    bins = [0] * 100 + [1] * 100
    net = gbs.gbs_make_network_binned(U, np.full(M, r), bins, "bf16x3", stream)
    gbs.gbs_sample_2d(net, wl.SEED_S_BASE + 200, 0, E, n_sub, K, K)
    gbs.gbs_sample(net, wl.SEED_S_BASE + 200, 0, E, n_sub, K)
    P, s, _, _ = gbs.gbs_binned_counts_2d(net, K, K)
    P1, s1, _, _ = gbs.gbs_binned_counts(net, 0, K)
    gbs.gbs_free_network(net)
    assert s.max() < 3e-5, s.max()
    m1, m2 = np.meshgrid(np.arange(K), np.arange(K), indexing="ij")
    odd = (m1 + m2) % 2 == 1
    assert np.max(np.abs(P[odd])) < 1e-4
    assert abs(P.sum() - 1.0) < 1e-9
    # the total count of the same trajectories, and it against the exact
    # lossless distribution (Eq. Exact_multi_mode_squeezed_state)
    diag = np.bincount(((m1 + m2) % K).ravel(), weights=P.ravel(), minlength=K)
    np.testing.assert_allclose(diag, P1, rtol=0, atol=1e-11)
    res = agreement(P1, s1, ex.negative_binomial(M, r, K))
    assert res["ok"], res
