"""GBS_FP32: the FP64 path with the propagation GEMM in FP32 arithmetic.

The sampler, the occupation epilogue, the generating functions and the
inversion are those of GBS_FP64; only alpha' = T alpha and beta' = T* beta
are formed from FP32-rounded operands with FP32 products accumulated in FP32
along the N input modes.

Tolerance of n_S (derived from the arithmetic, u = 2^-24): rounding T and
alpha to FP32 and N fused multiply-adds give
|d alpha'_i| <= (N + 2) u A_i with A_i = sum_j |T_ij| |alpha_j| (likewise
B_i for beta'); the epilogue's FP64 products and sums add nothing at this
scale, so |d n_S| <= 2 (N + 2) u (1 + 2^-10) sum_i A_i B_i.  The errors must
also be visibly above FP64 rounding, which shows that the FP32 arithmetic
ran.  P(m) must agree with the FP64 path on the same trajectories within one
sampling error, and with the exact distribution within sampling error
(pooled over independent ensembles).
"""

import numpy as np
import pytest

import oracle
import oracle.exact as ex
import workloads as wl
from stats import pooled_z2

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


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


def _bound_scale(net_def, e_list):
    """sum_i A_i B_i per trajectory, A_i = sum_j |T_ij| |alpha_j|."""
    absT = np.abs(net_def.T)
    out = []
    for e in e_list:
        a, b, _, _ = oracle.sample_amplitudes(net_def.T, net_def.r, net_def.seed_s, int(e))
        out.append(float(np.sum((absT @ np.abs(a)) * (absT @ np.abs(b)))))
    return np.array(out)


@pytest.mark.parametrize("shape", [(16, 16), (7, 9), (9, 7), (1, 1), (100, 130), (257, 200),
                                   (1000, 64)])
@pytest.mark.parametrize("general", [False, True])
def test_fp32_per_sample_totals(gbs, stream, shape, general):
    N, M = shape
    net_def = wl.small_network(N, M=M, r=0.7, t2=0.9, seed=N + 2 * M, general_loss=general)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "fp32", stream)
    assert gbs.gbs_network_info(net)[2] == gbs.GBS_FP32
    E, e0 = 200, 777
    n, nS = gbs.gbs_debug_samples(net, net_def.seed_s, e0, E)
    gbs.gbs_free_network(net)
    no, nSo = oracle.samples(net_def.T, net_def.r, net_def.seed_s, e0, E)
    # the sampler is the FP64 one
    assert np.max(np.abs(n - no) / np.maximum(np.abs(no), 1.0)) < 1e-10
    scale = _bound_scale(net_def, range(e0, e0 + E))
    err = np.abs(nS - nSo)
    bound = 2.0 * (N + 2) * U32 * (1.0 + 2.0 ** -10) * scale
    assert np.all(err <= bound), float(np.max(err / bound))
    # FP32 arithmetic, not FP64: errors well above FP64 rounding
    if N * M > 1:
        assert np.max(err / scale) > 2.0 ** -40


def test_fp32_distribution_matches_fp64_and_exact(gbs, stream):
    """Same trajectories on both SIMT precisions: |dP| <= sigma_FP64 per bin,
    for 12 independent ensembles; and P(m) against the exact uniform-loss
    distribution by the pooled (dP / sigma)^2 of the 12 (one ensemble's bins
    share its trajectories, so one run's chi^2 has few degrees of freedom:
    the first seed here gives 2.96 on the FP64 oracle as well)."""
    net_def = wl.small_network(257, r=0.6, t2=0.95, seed=5)
    E, n_sub, K1 = 1 << 15, 64, 512
    Pex = ex.exact_distribution(ex.eigenvalues_uniform_loss(net_def.r, 0.95), K1).real
    runs = []
    for k in range(12):
        seed = net_def.seed_s + 1000 * k
        res = {}
        for prec in ("fp64", "fp32"):
            net = gbs.gbs_make_network(net_def.T, net_def.r, prec, stream)
            gbs.gbs_sample(net, seed, 0, E, n_sub, K1)
            res[prec] = gbs.gbs_binned_counts(net, 0, K1)
            gbs.gbs_free_network(net)
        P64, s64 = res["fp64"][0], res["fp64"][1]
        P32, s32 = res["fp32"][0], res["fp32"][1]
        assert np.all(np.abs(P32 - P64) <= np.maximum(s64, 1e-13)), k
        assert abs(P32.sum() - 1.0) < 1e-9
        runs.append((P32, s32, Pex))
    pooled = pooled_z2(runs)
    assert 0.5 <= pooled["mean_z2"] <= 2.0, pooled
    assert 0.5 <= pooled["frac_within_1sigma"] <= 0.85, pooled


def test_fp32_is_rejected_where_only_split_precisions_run(gbs, stream):
    """Batches and the tcgen05 configuration calls need a BF16 split
    precision; an FP32 network is refused with EINVAL like an FP64 one."""
    net_def = wl.small_network(16, r=0.5, t2=0.9, seed=1)
    net = gbs.gbs_make_network(net_def.T, net_def.r, "fp32", stream)
    with pytest.raises(gbs.GbsError) as e1:
        gbs.gbs_set_gemm_config(net, 1, 0, 0)
    with pytest.raises(gbs.GbsError) as e2:
        gbs.gbs_make_batch([net])
    assert e1.value.code == gbs.GBS_EINVAL and e2.value.code == gbs.GBS_EINVAL
    gbs.gbs_free_network(net)
