"""Per-trajectory observable densities (Appendix A) on the GPU against the
oracle's projectors of the same trajectories, and the paper's diagnostic:
for lossless GBS (M = 20, r = 0.5) the +P projectors G_+(4) and G_+(3) have
long positive and negative tails, the matrix-P G_0(4) stays in (0, 0.4] and
G_0(3) vanishes."""
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


def _oracle_hist(orc, n, nS, ms, lo, hi, nbins):
    out = np.zeros((2, len(ms), nbins + 2), dtype=np.int64)
    inv = nbins / (hi - lo)
    for i in range(n.shape[0]):
        for q, m in enumerate(ms):
            gm, gp = orc.projector_direct(n[i], nS[i], m, 1)
            for est, v in enumerate((gm[0].real, gp[0].real)):
                x = (v - lo) * inv
                b = 0 if not (x >= 0) else (nbins + 1 if x >= nbins else 1 + int(x))
                out[est, q, b] += 1
    return out


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_histogram_matches_oracle(orc, gbs, prec):
    import torch
    net_def = wl.small_network(10, r=0.6, t2=0.85, seed=33)
    ms, lo, hi, nbins, E = [0, 3, 4], -1.0, 1.0, 400, 6000
    net = gbs.gbs_make_network(net_def.T, net_def.r, prec, torch.cuda.current_stream().cuda_stream)
    got = gbs.gbs_histogram(net, net_def.seed_s, 17, E, ms, lo, hi, nbins)
    n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, 17, E)
    gbs.gbs_free_network(net)
    want = _oracle_hist(orc, n, nS, ms, lo, hi, nbins)   # the device's own n, n_S
    assert got.sum() == 2 * len(ms) * E
    assert np.abs(got - want).sum() <= 4      # values within rounding of a bin edge
    if prec == "fp64":
        no, nSo = orc.samples(net_def.T, net_def.r, net_def.seed_s, 17, E)
        want_o = _oracle_hist(orc, no, nSo, ms, lo, hi, nbins)
        assert np.abs(got - want_o).sum() <= 4


def test_invalid_histograms(gbs):
    import torch
    net_def = wl.small_network(6, r=0.5, t2=0.9, seed=34)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "fp64", torch.cuda.current_stream().cuda_stream)
    for args in (([3], 1.0, -1.0, 10),         # lo >= hi
                 ([3], -1.0, 1.0, 0),          # no bins
                 ([3, 4], -1.0, 1.0, 4000)):   # counts beyond shared memory
        with pytest.raises(gbs.GbsError):
            gbs.gbs_histogram(net, 1, 0, 100, *args)
    gbs.gbs_free_network(net)


@pytest.mark.slow
def test_appendix_a_tails(gbs):
    import torch
    M, r = 20, 0.5
    U = wl.haar_unitary(M, wl.SEED_U_BASE + 20)
    net = gbs.gbs_make_network(U, np.full(M, r), "fp64", torch.cuda.current_stream().cuda_stream)
    lo, hi, nbins, E = -3.75, 3.75, 3000, 2 ** 21      # bins of 0.0025
    h = gbs.gbs_histogram(net, wl.SEED_S_BASE + 20, 0, E, [3, 4], lo, hi, nbins)
    gbs.gbs_free_network(net)
    edges = lo + (hi - lo) * np.arange(nbins + 1) / nbins
    lower = np.concatenate([[-np.inf], edges[:-1], [hi]])   # lower edge of each bin
    upper = np.concatenate([[lo], edges[1:], [np.inf]])
    mp3, mp4 = h[0, 0], h[0, 1]
    pp3, pp4 = h[1, 0], h[1, 1]
    # matrix-P: G_0(4) in (0, 0.4], G_0(3) within one bin of zero
    assert mp4[(upper <= 0.0) | (lower > 0.4)].sum() == 0
    assert mp3[(lower < -0.0025) | (upper > 0.0025)].sum() == 0
    # +P: the bulk in [-0.5, 0.5], with tails beyond it, positive for m = 4
    # and negative for m = 3
    assert pp4[(lower >= -0.5) & (upper <= 0.5)].sum() > 0.9 * E
    assert pp4[lower >= 0.5].sum() > 0 and pp4[upper <= -0.5].sum() == 0
    assert pp3[upper <= -0.5].sum() > 0 and pp3[lower >= 0.5].sum() == 0
