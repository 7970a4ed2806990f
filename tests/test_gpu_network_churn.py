"""Networks created and freed in a loop.

Every buffer a network owns comes from the device's stream-ordered memory
pool on the network's stream, and a freed network's memory is handed to the
next one.  The results of each pass must equal the first pass bit for bit
(nothing read before it is written), across precisions, binned networks and
two streams, and the device's free memory must not shrink from pass to pass
(the pool reuses what it holds instead of growing).
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_12749_gb300 as g
    g.build()
    return g, torch


def _pass(g, streams, defs):
    out = []
    for i, (nd, prec) in enumerate(defs):
        s = streams[i % len(streams)]
        net = g.gbs_make_network(nd.T, nd.r, prec, s)
        chunk = g.gbs_network_info(net)[3]
        # two chunks and a ragged tail
        g.gbs_sample(net, nd.seed_s, 3, 2 * chunk + 777, 8, 128)
        out.append(g.gbs_binned_counts(net, 0, 128))
        g.gbs_free_network(net)
        bins = [b % 2 for b in range(nd.T.shape[0])]
        net = g.gbs_make_network_binned(nd.T, nd.r, bins, prec, s)
        g.gbs_sample_nd(net, nd.seed_s, 9, 5000, 6, (32, 32))
        out.append(g.gbs_binned_counts_nd(net, (32, 32), (0, 0)))
        g.gbs_free_network(net)
    return out


def test_results_and_memory_stable_over_network_churn(env):
    g, torch = env
    streams = [torch.cuda.Stream().cuda_stream, torch.cuda.Stream().cuda_stream]
    defs = [(wl.small_network(48, 56, r=0.6, t2=0.9, seed=130), "bf16x3"),
            (wl.small_network(20, 20, r=0.8, t2=0.95, seed=131), "fp64"),
            (wl.small_network(130, 120, r=0.5, t2=0.9, seed=132), "bf16x6")]
    first = _pass(g, streams, defs)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        again = _pass(g, streams, defs)
        for a, b in zip(first, again):
            for x, y in zip(a, b):
                assert np.array_equal(np.asarray(x), np.asarray(y))
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # a little slack for the driver's own bookkeeping
    assert free1 >= free0 - (64 << 20), (free0, free1)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_pinned_host_T_read_in_place_equals_staged_upload(env, prec):
    """gbs_make_network reads T in place when it lies in page-locked host
    memory the device can address, and stages it through a device buffer
    otherwise; both give bitwise the same network (per-trajectory n, n_S and
    the sub-ensemble sums)."""
    g, torch = env
    nd = wl.small_network(300, M=260, r=0.8, t2=0.9, seed=5, general_loss=True)
    s = torch.cuda.current_stream().cuda_stream
    pinned = torch.empty(2 * nd.T.size, dtype=torch.float64, pin_memory=True)
    Tp = pinned.numpy().view(np.complex128).reshape(nd.T.shape)
    Tp[:] = nd.T
    res = []
    for T in (np.array(nd.T, copy=True), Tp):
        net = g.gbs_make_network(T, nd.r, prec, s)
        n, nS = g.gbs_debug_samples(net, nd.seed_s, 11, 1000)
        g.gbs_sample(net, nd.seed_s, 0, 5000, 10, 256)
        _, _, acc, cnt = g.gbs_get_accumulators(net)
        g.gbs_free_network(net)
        res.append((n, nS, acc, cnt))
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)
