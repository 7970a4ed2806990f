"""Failure detection without a GPU fault.

Each failure is caused on the host and reported through the C ABI, and the
network stays usable afterwards:
  * GBS_ETIMEOUT: a wait limit of 0 (gbs_set_wait_limit) makes every GEMM
    launch first wait on a barrier that nothing arrives on; the wait gives
    up, raises the network's timeout flag, the kernel issues no MMA, lets the
    loads it already issued land and returns.  The next synchronous read
    reports the timeout and clears the flag.
  * GBS_ENONFINITE: sub-ensemble sums holding NaN and infinity are uploaded
    with gbs_set_accumulators.
  * GBS_ENOMEM: sub-ensemble sums of 2 x 65535 x 2^20 complex doubles (about
    2.2 TB, beyond the device) are asked for; the allocation fails at once
    without taking memory.
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


def _sums(gbs, net, seed, E, n_sub, K1):
    gbs.gbs_sample(net, seed, 0, E, n_sub, K1)
    P = gbs.gbs_binned_counts(net, 0, K1)
    _, _, acc, counts = gbs.gbs_get_accumulators(net)
    return P, acc, counts


@pytest.mark.parametrize("precision", ["bf16x3", "bf16x6"])
def test_gemm_wait_timeout_is_reported_and_recoverable(gbs, stream, precision):
    net_def = wl.small_network(96, M=160, r=0.7, t2=0.9, seed=41)
    E, n_sub, K1 = 6000, 8, 128
    ref = gbs.gbs_make_network(net_def.T, net_def.r, precision, stream)
    gbs.gbs_set_gemm_config(ref, 1, 0, 0)
    P_ref, acc_ref, cnt_ref = _sums(gbs, ref, net_def.seed_s, E, n_sub, K1)
    gbs.gbs_free_network(ref)

    net = gbs.gbs_make_network(net_def.T, net_def.r, precision, stream)
    gbs.gbs_set_gemm_config(net, 1, 0, 0)
    gbs.gbs_set_wait_limit(net, 0)
    gbs.gbs_sample(net, net_def.seed_s, 0, E, n_sub, K1)  # asynchronous: no error yet
    with pytest.raises(gbs.GbsError) as ei:
        gbs.gbs_binned_counts(net, 0, K1)
    assert ei.value.code == gbs.GBS_ETIMEOUT
    # the report cleared the flag; with the default limit back and the sums
    # cleared, the network gives bitwise the results of a fresh one
    gbs.gbs_set_wait_limit(net, 2_000_000_000)
    gbs.gbs_reset(net)
    P, acc, cnt = _sums(gbs, net, net_def.seed_s, E, n_sub, K1)
    gbs.gbs_free_network(net)
    assert np.array_equal(cnt, cnt_ref)
    assert np.array_equal(acc.view(np.float64), acc_ref.view(np.float64))
    for x, y in zip(P, P_ref):
        assert np.array_equal(x, y)


def test_timeout_of_one_network_leaves_another_untouched(gbs, stream):
    """The flag is per network: a timed-out launch on one network does not
    make another network's read fail."""
    d = wl.small_network(64, r=0.6, t2=0.95, seed=43)
    a = gbs.gbs_make_network(d.T, d.r, "bf16x3", stream)
    b = gbs.gbs_make_network(d.T, d.r, "bf16x3", stream)
    gbs.gbs_set_gemm_config(a, 1, 0, 0)
    gbs.gbs_set_gemm_config(b, 1, 0, 0)
    gbs.gbs_set_wait_limit(a, 0)
    gbs.gbs_sample(a, d.seed_s, 0, 2048, 4, 64)
    gbs.gbs_sample(b, d.seed_s, 0, 2048, 4, 64)
    P = gbs.gbs_binned_counts(b, 0, 64)
    assert abs(P[0].sum() - 1.0) < 1e-9
    with pytest.raises(gbs.GbsError) as ei:
        gbs.gbs_binned_counts(a, 0, 64)
    assert ei.value.code == gbs.GBS_ETIMEOUT
    gbs.gbs_free_network(a)
    gbs.gbs_free_network(b)


def test_nonfinite_sums_are_counted(gbs, stream):
    d = wl.small_network(32, r=0.5, t2=0.9, seed=44)
    net = gbs.gbs_make_network(d.T, d.r, "fp64", stream)
    n_sub, K1 = 4, 64
    gbs.gbs_sample(net, d.seed_s, 0, 4096, n_sub, K1)
    _, _, acc, counts = gbs.gbs_get_accumulators(net)
    assert gbs.gbs_check_finite(net) == 0
    bad = acc.copy()
    bad[0, 1, 3] = complex(np.nan, 0.0)            # the count is of complex entries
    bad[1, 2, 7] = complex(np.inf, -np.inf)
    bad[1, 3, 0] = complex(1.0, np.nan)
    gbs.gbs_set_accumulators(net, bad, counts)
    assert gbs.gbs_check_finite(net) == 3
    with pytest.raises(gbs.GbsError) as ei:
        gbs.gbs_binned_counts(net, 0, K1)
    assert ei.value.code == gbs.GBS_ENONFINITE
    # finite sums uploaded again: the original result
    gbs.gbs_set_accumulators(net, acc, counts)
    assert gbs.gbs_check_finite(net) == 0
    P = gbs.gbs_binned_counts(net, 0, K1)
    assert abs(P[0].sum() - 1.0) < 1e-9
    gbs.gbs_free_network(net)


def test_allocation_failure_is_reported_and_recoverable(gbs, stream):
    d = wl.small_network(32, r=0.5, t2=0.9, seed=45)
    net = gbs.gbs_make_network(d.T, d.r, "bf16x3", stream)
    with pytest.raises(gbs.GbsError) as ei:
        gbs.gbs_sample(net, d.seed_s, 0, 1024, 65535, 1 << 20)
    assert ei.value.code == gbs.GBS_ENOMEM
    # nothing was fixed: a normal call on the same network works
    P, _, counts = _sums(gbs, net, d.seed_s, 4096, 4, 64)
    assert counts.sum() == 4096
    assert abs(P[0].sum() - 1.0) < 1e-9
    gbs.gbs_free_network(net)
