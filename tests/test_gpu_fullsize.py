"""Full-size checks of the named workloads in the launch configuration the
bench times (BF16x3 tcgen05 path, chunks of up to 2^17 trajectories).

At these sizes the oracle cannot run the whole ensemble, so:
  * sampled trajectories are compared one by one with the oracle (n_S within
    2^-14 of the amplitude scale, the 3-product split's bound);
  * P(m) over the full ensemble is compared with the exact uniform-loss
    distribution (determinant generating function, E2) within sampling error;
  * the split precision is compared with the FP64 path on the same
    trajectories (|dP| <= sigma_FP64 on every bin) at the full N;
  * sum_m P(m) = 1 and the uniform-loss identity n_S = t^2 n per trajectory.
"""
import math

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


def _sampled_parity(gbs, net, net_def, picks):
    for e in picks:
        n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, int(e), 1)
        no, nSo = oracle.samples(net_def.T, net_def.r, net_def.seed_s, int(e), 1)
        _, _, ap, bp = oracle.sample_amplitudes(net_def.T, net_def.r, net_def.seed_s, int(e))
        S = float(np.sum(np.abs(ap) * np.abs(bp)))
        assert abs(nS[0] - nSo[0]) <= 2.0 ** -14 * S, (e, nS[0], nSo[0])
        assert abs(n[0] - no[0]) <= 1e-5 * max(abs(no[0]), 1.0)


def _chunk_parity(gbs, net, T, r, seed, e0):
    """One chunk of the network's size (less 77, so that its last trajectory
    tile is ragged) through the GEMM in the tile configuration the network's
    launches use; trajectories at both ends, across a tile boundary and in
    the middle against the oracle one by one."""
    count = gbs.gbs_network_info(net)[3] - 77
    n, nS = gbs.gbs_debug_samples(net, seed, e0, count)
    for q in (0, 127, 128, count // 2 + 7, count - 1):
        no, nSo = oracle.samples(T, r, seed, e0 + q, 1)
        _, _, ap, bp = oracle.sample_amplitudes(T, r, seed, e0 + q)
        S = float(np.sum(np.abs(ap) * np.abs(bp)))
        assert abs(nS[q] - nSo[0]) <= 2.0 ** -14 * S, (q, nS[q], nSo[0])
        assert abs(n[q] - no[0]) <= 1e-5 * max(abs(no[0]), 1.0)
    assert np.all(np.isfinite(nS))


@pytest.mark.parametrize("name", ["m1000", "m4000"])
def test_full_workload(gbs, name):
    import torch
    w = wl.NAMED[name]
    net_def = w.network()
    s = torch.cuda.Stream()
    net = gbs.gbs_make_network(net_def.T, net_def.r, "bf16x3", s.cuda_stream)
    # sampled trajectories, including both ends of the range
    _sampled_parity(gbs, net, net_def, [0, 1, 77777, w.E // 2, w.E - 1])
    # identity n_S = t^2 n on a full chunk
    n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, 0, 4096)
    assert np.max(np.abs(nS - w.t2 * n) / np.abs(n)) < 1e-4
    # the whole ensemble against the exact distribution
    gbs.gbs_sample(net, net_def.seed_s, 0, w.E, w.n_sub, w.K1)
    P = gbs.gbs_binned_counts(net, 0, w.K1)
    mu = ex.eigenvalues_uniform_loss(net_def.r, w.t2)
    Pex = ex.exact_distribution(mu, w.K1).real
    res = agreement(P[0], P[1], Pex)
    assert res["ok"], res
    assert abs(P[0].sum() - 1.0) < 1e-9
    # a whole chunk in the configuration the ensemble's launches were tuned to
    _chunk_parity(gbs, net, net_def.T, net_def.r, net_def.seed_s, w.E // 3)
    gbs.gbs_free_network(net)


@pytest.mark.parametrize("name", ["m1000", "m4000"])
def test_split_precision_gate_at_full_N(gbs, name):
    """|dP| <= sigma between BF16x3 and FP64 on the same trajectories, full N."""
    import torch
    w = wl.NAMED[name]
    net_def = w.network()
    s = torch.cuda.Stream()
    E = 2 ** 13
    res = {}
    for prec in ("fp64", "bf16x3"):
        net = gbs.gbs_make_network(net_def.T, net_def.r, prec, s.cuda_stream)
        gbs.gbs_sample(net, net_def.seed_s, 0, E, 16, w.K1)
        res[prec] = gbs.gbs_binned_counts(net, 0, w.K1)
        gbs.gbs_free_network(net)
    for est in (0, 2):
        ratio = np.abs(res["bf16x3"][est] - res["fp64"][est]) / np.maximum(res["fp64"][est + 1],
                                                                            1e-13)
        assert ratio.max() <= 1.0, (name, est, ratio.max())


@pytest.mark.slow
def test_m8000_workload(gbs):
    """N = M = 8000, r = 1, t^2 = 0.99, E = 2^20, K1 = 16384: sampled
    trajectories against the oracle, the whole ensemble against the exact
    distribution.  The Haar matrix is the QR of the workload's seeded Ginibre
    draw computed on the GPU (equal to the host QR up to rounding); both sides
    use the same T."""
    import torch
    w = wl.NAMED["m8000"]
    T = (math.sqrt(w.t2) * wl.haar_unitary_device(w.N, wl.SEED_U_BASE + w.index)).cpu().numpy()
    T = np.ascontiguousarray(T)
    r = np.full(w.N, 1.0)
    seed = wl.SEED_S_BASE + w.index
    s = torch.cuda.Stream()
    net = gbs.gbs_make_network(T, r, "bf16x3", s.cuda_stream)
    for e in (0, 123457, w.E - 1):
        n, nS = gbs.gbs_debug_samples(net, seed, e, 1)
        no, nSo = oracle.samples(T, r, seed, e, 1)
        _, _, ap, bp = oracle.sample_amplitudes(T, r, seed, e)
        S = float(np.sum(np.abs(ap) * np.abs(bp)))
        assert abs(nS[0] - nSo[0]) <= 2.0 ** -14 * S, (e, nS[0], nSo[0])
        assert abs(n[0] - no[0]) <= 1e-5 * max(abs(no[0]), 1.0)
    gbs.gbs_sample(net, seed, 0, w.E, w.n_sub, w.K1)
    P = gbs.gbs_binned_counts(net, 0, w.K1)
    # a whole chunk through the configuration the bench's launches use: a
    # banded tile order with aligned waves (A does not fit in L2)
    pair, band, keep = gbs.gbs_gemm_config(net)
    assert band > 0 and keep & 8, (pair, band, keep)
    _chunk_parity(gbs, net, T, r, seed, w.E // 2 + 5)
    gbs.gbs_free_network(net)
    mu = ex.eigenvalues_uniform_loss(r, w.t2)
    z = ex.roots_of_unity(w.K1)
    G = np.concatenate([ex.gf_from_eigenvalues(mu, z[a:a + 256]) for a in range(0, w.K1, 256)])
    Pex = ex.distribution_from_gf(G).real
    res = agreement(P[0], P[1], Pex)
    assert res["ok"], res
    assert abs(P[0].sum() - 1.0) < 1e-9
