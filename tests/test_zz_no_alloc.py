"""The allocation-free inversion entry point (gbs_binned_counts_noalloc).

Callers that cannot allocate device memory (a process whose device memory
belongs to another allocator, or a loop that must not synchronise the device
through cudaMalloc/cudaFree) pass their own device buffers and the library
uses a fixed internal work array.  Its results must equal those of the
allocating entry point, gbs_binned_counts_device, on the same sums, on two
calls in a row (the second call reuses the array the first one left behind).
This file is named to be collected last.
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


def _reference(g, torch, net, m_off, K1, stream):
    out = torch.zeros(4 * K1, dtype=torch.float64, device="cuda")
    g.gbs_binned_counts_device(net, m_off, out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_allocating_inversion_twice(env):
    g, torch = env
    stream = torch.cuda.current_stream().cuda_stream
    cases = []
    for net_def, prec, E, n_sub, K1, m_off in (
            (wl.SMALL16.network(), "fp64", 4096, 16, 64, 0),
            (wl.small_network(200, r=0.5, t2=0.99, seed=11), "bf16x3", 20000, 50, 256, 7)):
        net = g.gbs_make_network(net_def.T, net_def.r, prec, stream)
        g.gbs_sample(net, net_def.seed_s, 0, E, n_sub, K1)
        _, _, acc, cnt = g.gbs_get_accumulators(net)
        ref = _reference(g, torch, net, m_off, K1, stream)
        acc_d = torch.from_numpy(np.ascontiguousarray(acc).view(np.float64).ravel().copy()).cuda()
        cnt_d = torch.from_numpy(cnt.copy()).cuda()
        cases.append((net, acc_d, cnt_d, n_sub, K1, m_off, ref))
    # two calls in a row per case, the cases interleaved
    for rep in range(2):
        for net, acc_d, cnt_d, n_sub, K1, m_off, ref in cases:
            out = torch.full((4 * K1,), float("nan"), dtype=torch.float64, device="cuda")
            g.gbs_binned_counts_noalloc(acc_d.data_ptr(), cnt_d.data_ptr(), n_sub, K1, m_off,
                                        out.data_ptr(), stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15)
    for net, *_ in cases:
        g.gbs_free_network(net)


def test_noalloc_rejects_sizes_beyond_its_work_space(env):
    g, torch = env
    stream = torch.cuda.current_stream().cuda_stream
    acc_d = torch.zeros(8, dtype=torch.float64, device="cuda")
    cnt_d = torch.ones(2, dtype=torch.int64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    for n_sub, K1 in ((1024, 1024), (1, 1 << 17), (4, 24)):
        with pytest.raises(g.GbsError) as ei:
            g.gbs_binned_counts_noalloc(acc_d.data_ptr(), cnt_d.data_ptr(), n_sub, K1, 0,
                                        out.data_ptr(), stream)
        assert ei.value.code == g.GBS_EINVAL
