"""The generating-function windows and the FP64 rate probe.

Per trajectory the finalize kernel bounds the k at which each term of the
generating functions can exceed the skip threshold (2^-60 on the FP64
path, 2^-47 on the BF16 split paths, whose double-float evaluation rounds
terms of order one to 2^-46).  Outside the windows the oracle's terms, at
the device's own n and n_S, must lie below that threshold: the e^{(z-1) n_S}
term (the +P generating function) outside w1, matrix-P's second term
outside w2, so G_mP below twice the threshold outside both.
"""
import numpy as np
import pytest

import oracle
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
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("prec,thresh", [("fp64", 2.0 ** -60), ("bf16x3", 2.0 ** -47)])
@pytest.mark.parametrize("general", [False, True])
def test_terms_outside_windows_below_threshold(gbs, stream, prec, thresh, general):
    net_def = wl.small_network(48, r=0.9, t2=0.9, seed=77, general_loss=general)
    E, K1 = 128, 1024
    net = gbs.gbs_make_network(net_def.T, net_def.r, prec, stream)
    gbs.gbs_sample(net, net_def.seed_s, 0, E, 4, K1)
    n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, 0, E)
    w = gbs.gbs_debug_windows(net, net_def.seed_s, 0, E)
    gbs.gbs_free_network(net)
    k = np.arange(K1)
    d0 = np.minimum(k, K1 - k)
    dpi = np.abs(k - K1 // 2)
    inside = 0
    for e in range(E):
        gm, gp = oracle.gf_sample(n[e], nS[e], K1)
        out1 = d0 > w[e, 0]
        out2 = dpi > w[e, 1]
        assert np.all(np.abs(gp[out1]) < thresh), (e, np.abs(gp[out1]).max())
        both = out1 & out2
        assert np.all(np.abs(gm[both]) < 2.0 * thresh), (e, np.abs(gm[both]).max())
        inside += int(np.sum(~out1))
    # the windows leave part of the circle out (the skip does something)
    assert inside < 0.95 * E * K1


def test_fp64_rate_probe(gbs, stream):
    """CUDA-event FMA-chain probe: a plausible FP64 rate (GB300's FP64 pipe
    is rated at about 1.2 TFLOP/s), positive and finite."""
    rate = gbs.gbs_measure_fp64_rate(stream)
    assert np.isfinite(rate) and 0.1 < rate < 10.0, rate
