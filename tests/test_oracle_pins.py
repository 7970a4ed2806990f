"""Pins of the CPU oracle against things other than itself.

Each test ties an oracle function to a value the paper prints, a closed form,
an invariant, a textbook/library special case, or a brute-force computation,
so that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.  No GPU needed.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle.exact as ex
import workloads as wl
from stats import agreement, pooled_z2

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _paper():
    with open(os.path.join(GOLD, "paper_values.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# Random numbers
# ---------------------------------------------------------------------------
def test_philox_known_answers(orc):
    """Philox-4x32-10 against the Random123 known-answer vectors (Salmon et al. SC'11)."""
    rows = []
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for row in rows:
        out = orc.philox4x32_10(row[:4], row[4:6])
        assert list(out) == row[6:]


def test_box_muller_moments(orc):
    """Box-Muller normals: mean 0, variance 1, kurtosis 3, uncorrelated pair."""
    w = np.array([orc.normals(7, e, j) for e in range(4000) for j in range(10)])
    n = w.size
    x = w.ravel()
    assert abs(x.mean()) < 5.0 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs(np.mean(x ** 4) - 3.0) < 5.0 * math.sqrt(96.0 / n)
    assert abs(np.mean(w[:, 0] * w[:, 1])) < 5.0 / math.sqrt(n / 2)


def test_sampler_covariance_matches_squeezed_plusP_density(orc):
    """'Applications to GBS': the +P density of a squeezed vacuum on the real
    plane is xi(a) xi(b) e^{ab}, xi(a) ~ exp(-a^2 coth(r)/2).  Its covariance
    is the inverse of the precision matrix [[coth r, -1], [-1, coth r]]
    (inverted here by numpy, independently of the sampler's own formula)."""
    for r in (0.3, 1.0):
        ab = np.array([orc.sample_inputs(np.array([r]), 11, e)[:2] for e in range(30000)])[:, :, 0]
        cov = ab.T @ ab / ab.shape[0]
        prec = np.array([[1.0 / math.tanh(r), -1.0], [-1.0, 1.0 / math.tanh(r)]])
        want = np.linalg.inv(prec)
        # standard errors of second moments of a Gaussian pair
        se = np.sqrt((want ** 2 + np.outer(np.diag(want), np.diag(want))) / ab.shape[0])
        assert np.all(np.abs(cov - want) < 5 * se), (r, cov, want)
        assert abs(np.mean(ab[:, 0])) < 5 * math.sqrt(want[0, 0] / ab.shape[0])


# ---------------------------------------------------------------------------
# Propagation
# ---------------------------------------------------------------------------
def test_propagation_matches_matmul(orc):
    """alpha' = t alpha and beta' = t* beta ('Applications to GBS') against
    numpy's matrix product on the oracle's own input amplitudes."""
    net = wl.small_network(7, M=9, r=0.6, t2=0.9, seed=3)
    a, b, ap, bp = orc.sample_amplitudes(net.T, net.r, net.seed_s, 5)
    np.testing.assert_allclose(ap, net.T @ a, rtol=0, atol=1e-13)
    np.testing.assert_allclose(bp, net.T.conj() @ b, rtol=0, atol=1e-13)
    n, nS = orc.samples(net.T, net.r, net.seed_s, 5, 1)
    assert abs(nS[0] - np.sum(ap * bp)) < 1e-12
    assert abs(n[0] - np.dot(a, b)) < 1e-12


def test_uniform_loss_identity(orc):
    """For T = t U with U unitary, T^T T* = t^2 I, so n_S = t^2 n exactly."""
    net = wl.small_network(12, r=0.8, t2=0.93, seed=4)
    n, nS = orc.samples(net.T, net.r, net.seed_s, 0, 300)
    assert np.max(np.abs(nS - 0.93 * n)) < 1e-12 * max(1.0, np.max(np.abs(n)))


def test_matmul_pin_detects_transposed_network(orc):
    """Planted mistake: propagating with T^T instead of T.  U^T is unitary
    too, so the identity above cannot see it, but the element-wise matmul
    pin does (for square networks as well as non-square ones)."""
    net = wl.small_network(12, r=0.8, t2=0.93, seed=4)
    a, b, ap, bp = orc.sample_amplitudes(np.ascontiguousarray(net.T.T), net.r, net.seed_s, 3)
    assert np.max(np.abs(ap - net.T @ a)) > 1e-3
    assert np.max(np.abs(bp - net.T.conj() @ b)) > 1e-3


def test_identity_detects_non_unitary_network(orc):
    """The identity is a real constraint: with non-uniform loss it fails."""
    net = wl.small_network(12, r=0.8, t2=0.93, seed=4, general_loss=True)
    n, nS = orc.samples(net.T, net.r, net.seed_s, 0, 50)
    assert np.max(np.abs(nS - 0.93 * n)) > 1e-2


# ---------------------------------------------------------------------------
# Projectors and generating functions
# ---------------------------------------------------------------------------
def _some_samples():
    # positive, negative, small and large n; real and complex n_S
    return [(3.0, 2.7 + 0.0j), (0.4, 0.35 - 0.1j), (-2.0, -1.8 + 0.3j), (25.0, 24.5 + 0.2j),
            (8.0, 8.0 + 0.0j), (-0.3, 0.2 + 0.05j)]


def test_gf_at_one_is_one(orc):
    """G(z = 1) = sum_m G(m) = 1 per sample for both estimators (normalisation)."""
    for n, nS in _some_samples():
        gm, gp = orc.gf_sample(n, nS, 16)
        assert abs(gm[0] - 1.0) < 1e-14 and abs(gp[0] - 1.0) < 1e-14


def test_gf_sign_flip_symmetries(orc):
    """Changing the sign of every alpha_j maps (n, n_S) to (-n, -n_S).  The
    matrix-P GF cosh(n + (z-1) n_S) / cosh n is unchanged (cosh is even); the
    +P GF e^{(z-1) n_S} goes to its reciprocal, so the product of the two
    +P values is 1 at every z_k."""
    K1 = 64
    for n, nS in _some_samples():
        gm1, gp1 = orc.gf_sample(n, nS, K1)
        gm2, gp2 = orc.gf_sample(-n, -nS, K1)
        assert np.max(np.abs(gm1 - gm2)) < 1e-12 * max(1.0, np.max(np.abs(gm1))), (n, nS)
        assert np.max(np.abs(gp1 * gp2 - 1.0)) < 1e-12, (n, nS)


def test_matrixP_gf_bounded_for_uniform_loss(orc):
    """For T = t U, n_S = t^2 n is real and, on |z| = 1,
    Re(n + (z-1) n_S) = n (1 - t^2 (1 - cos theta)) has modulus at most |n|;
    since |cosh(x + iy)| <= cosh x, |G_mP(z_k)| <= 1 for every sample and k.
    With the sign of (z - 1) flipped the bound fails on the same samples."""
    net = wl.small_network(10, r=0.9, t2=0.7, seed=6)
    n, nS = orc.samples(net.T, net.r, net.seed_s, 0, 200)
    K1 = 128
    z = np.exp(2j * np.pi * np.arange(K1) / K1)
    worst, flipped = 0.0, 0.0
    for a, b in zip(n, nS):
        gm, _ = orc.gf_sample(a, b, K1)
        worst = max(worst, float(np.max(np.abs(gm))))
        flipped = max(flipped, float(np.max(np.abs(np.cosh(a + (1 - z) * b) / np.cosh(a)))))
    assert worst <= 1.0 + 1e-12
    assert flipped > 1.5


def test_gf_taylor_coefficients_equal_direct_projector(orc):
    """The GF's Taylor coefficients (read off by an FFT at K1 far beyond the
    support) equal the per-bin projector of Eq. c-number-variable, for both
    parities of m and both estimators."""
    K1 = 512
    for n, nS in _some_samples():
        gm, gp = orc.gf_sample(n, nS, K1)
        cm = np.fft.fft(gm) / K1
        cp = np.fft.fft(gp) / K1
        dm, dp = orc.projector_direct(n, nS, 0, 80)
        scale = max(1.0, np.max(np.abs(dm)))
        assert np.max(np.abs(cm[:80] - dm)) < 1e-12 * scale, (n, nS)
        assert np.max(np.abs(cp[:80] - dp)) < 1e-12 * max(1.0, np.max(np.abs(dp))), (n, nS)


def test_lossless_parity_projector_special_case(orc):
    """All channels counted (n_S = n): odd projectors vanish and
    g0(2m) = n^{2m} / [cosh(n) (2m)!] (text after Eq. c-number-variable)."""
    for n in (0.5, 3.0, 9.0):
        dm, _ = orc.projector_direct(n, n + 0j, 0, 24)
        for m in range(24):
            if m % 2:
                assert abs(dm[m]) < 1e-15
            else:
                want = n ** m / (math.cosh(n) * math.factorial(m))
                assert abs(dm[m] - want) <= 1e-13 * max(want, 1e-300) + 1e-300


def test_plusP_projector_is_poisson(orc):
    """+P uses g0 = 1 (Eq. phase_space_projector): G_+(m) = n^m e^{-n} / m!."""
    for nS in (0.7, 4.0, 12.0):
        _, dp = orc.projector_direct(1.0, nS + 0j, 0, 30)
        want = np.array([nS ** m * math.exp(-nS) / math.factorial(m) for m in range(30)])
        np.testing.assert_allclose(dp.real, want, rtol=1e-12, atol=1e-300)


def test_matrixP_G0_4_range_and_plusP_tails(orc):
    """Appendix A / Fig. 5, lossless M = 20, r = 0.5: the matrix-P projector
    G0(4) stays in (0, 0.4) with its upper peak near 0.39, while the +P
    observables G+(4), G+(3) have long positive / negative tails."""
    p = _paper()["matrixP_G0_4"]
    U = wl.haar_unitary(p["M"], 20)
    n, nS = orc.samples(U, np.full(p["M"], p["r"]), 99, 0, 20000)
    g4 = np.array([orc.projector_direct(a, b, 4, 1)[0][0].real for a, b in zip(n, nS)])
    assert g4.min() > -1e-10 and g4.max() < p["range"][1]
    assert abs(g4.max() - p["upper_mode"]) < 0.01
    gp4 = np.array([orc.projector_direct(a, b, 4, 1)[1][0].real for a, b in zip(n, nS)])
    gp3 = np.array([orc.projector_direct(a, b, 3, 1)[1][0].real for a, b in zip(n, nS)])
    assert gp4.max() > 2.0 and gp3.min() < -2.0


# ---------------------------------------------------------------------------
# Exact references (E1-E4)
# ---------------------------------------------------------------------------
def test_exact_E2_equals_E1_for_uniform_loss():
    net = wl.small_network(6, r=[0.3, 0.5, 0.7, 0.4, 0.6, 0.2], t2=0.8, seed=1)
    mu1 = np.sort(ex.eigenvalues_general(net.T, net.r))
    mu2 = np.sort(ex.eigenvalues_uniform_loss(net.r, 0.8))
    np.testing.assert_allclose(mu1, mu2, atol=1e-13)


def test_exact_E2_reduces_to_negative_binomial():
    """Eq. Exact_multi_mode_squeezed_state (lossless, uniform r)."""
    for M, r in ((20, 0.5), (200, 0.5), (64, 1.0)):
        P3 = ex.negative_binomial(M, r, 200)
        P2 = ex.exact_unaliased(ex.eigenvalues_uniform_loss(np.full(M, r), 1.0), 200)
        np.testing.assert_allclose(P2, P3, rtol=0, atol=1e-13)
        assert np.all(P3[1::2] == 0.0)


def test_exact_E1_matches_bruteforce_hafnians():
    """Pattern probabilities from Hafnians (pure and mixed-state formulas),
    summed over patterns, reproduce the determinant generating function."""
    U = wl.haar_unitary(3, 5)
    r = np.array([0.3, 0.5, 0.4])
    Pb = ex.total_count_bruteforce(U, r, 7, pure_U=U)
    P1 = ex.exact_unaliased(ex.eigenvalues_general(U, r), 7)
    np.testing.assert_allclose(Pb, P1, atol=1e-12)
    assert np.all(np.abs(Pb[1::2]) < 1e-15)
    net = wl.small_network(3, r=[0.3, 0.4, 0.35], t2=0.9, seed=2, general_loss=True)
    Pb = ex.total_count_bruteforce(net.T, net.r, 6)
    P1 = ex.exact_unaliased(ex.eigenvalues_general(net.T, net.r), 6)
    np.testing.assert_allclose(Pb, P1, atol=1e-12)


def test_exact_cutoffs_match_paper_table():
    """Appendix B prints m_min / m_max (1e-7 cut-offs) for r = 0.89; the
    negative binomial gives them to within a few counts (the paper's exact
    threshold convention is not stated)."""
    p = _paper()
    c = p["cutoffs_r089"]
    for M, lo_p, hi_p in zip(c["M"], c["m_min"], c["m_max"]):
        P = ex.negative_binomial(M, c["r"], hi_p + 200)
        lo, hi = ex.cutoffs(P, c["threshold"])
        assert abs(hi - hi_p) <= 5 and abs(lo - lo_p) <= 5, (M, lo, hi, lo_p, hi_p)
    c2 = p["cutoffs_right_panel"]
    for M, hi_p in zip(c2["M"], c2["m_max"]):
        P = ex.negative_binomial(M, c2["r"], hi_p + 200)
        assert abs(ex.cutoffs(P)[1] - hi_p) <= 5


# ---------------------------------------------------------------------------
# The Monte-Carlo estimator against the exact distribution
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["small16", "lossless", "general_loss"])
def test_matrixP_estimator_unbiased(orc, case):
    """Matrix-P P(m) from the whole oracle pipeline agrees with the exact
    (aliased) distribution within its own sampling errors."""
    if case == "small16":
        w = wl.SMALL16
        net = w.network()
        E, n_sub, K1 = w.E, w.n_sub, w.K1
        mu = ex.eigenvalues_uniform_loss(net.r, w.t2)
    elif case == "lossless":
        net = wl.small_network(10, r=0.7, t2=1.0, seed=6)
        E, n_sub, K1 = 2 ** 17, 64, 64
        mu = ex.eigenvalues_uniform_loss(net.r, 1.0)
    else:
        net = wl.small_network(8, r=[0.5, 0.9, 0.7, 0.6, 1.0, 0.4, 0.8, 0.55], t2=0.85, seed=7,
                               general_loss=True)
        E, n_sub, K1 = 2 ** 17, 64, 64
        mu = ex.eigenvalues_general(net.T, net.r)
    P, s, im = orc.run(net.T, net.r, net.seed_s, 0, E, n_sub, K1)
    Pex = ex.exact_distribution(mu, K1).real
    res = agreement(P[0], s[0], Pex)
    assert res["ok"], res
    assert abs(P[0].sum() - 1.0) < 1e-12  # G(1) = 1 per sample
    assert im[0] < 1e-3
    if case == "lossless":
        assert np.max(np.abs(P[0][1::2])) < 1e-12  # odd counts vanish (Eq. c-number-variable)


def test_sigma_scale_pooled_over_seeds(orc):
    """The reported sigma is the standard error of P(m), from both sides:
    over 16 independent ensembles (seeds) of a lossy 6-mode network, the
    pooled mean (dP / sigma)^2 against the exact distribution lies in
    [0.5, 2] and about two thirds of the bulk bins lie within one sigma.  The
    same check fails for sigma scaled by 2 or by 1/2."""
    net = wl.small_network(6, r=0.6, t2=0.9, seed=9)
    E, n_sub, K1 = 2 ** 13, 16, 64
    Pex = ex.exact_distribution(ex.eigenvalues_uniform_loss(net.r, 0.9), K1).real
    runs = []
    for k in range(16):
        P, s, _ = orc.run(net.T, net.r, net.seed_s + 1000 * k, 0, E, n_sub, K1)
        runs.append((P[0], s[0], Pex))
    res = pooled_z2(runs)
    assert 0.5 <= res["mean_z2"] <= 2.0, res
    assert 0.5 <= res["frac_within_1sigma"] <= 0.85, res
    assert pooled_z2([(P, 2.0 * s, R) for P, s, R in runs])["mean_z2"] < 0.5
    assert pooled_z2([(P, 0.5 * s, R) for P, s, R in runs])["mean_z2"] > 2.0


def test_direct_route_equals_gf_route(orc):
    """Direct per-bin sums and GF + inverse DFT give the same sub-ensemble
    statistics when K1 exceeds the support."""
    w = wl.SMALL16
    net = w.network()
    n, nS = orc.samples(net.T, net.r, net.seed_s, 0, 3000)
    Pd, sd = orc.direct_bins(n, nS, 0, 16, 0, 64)
    acc, cnt = orc.accumulate_gf(n, nS, 0, 16, 256)
    Pg, sg, _ = orc.invert(acc, cnt)
    np.testing.assert_allclose(Pg[:, :64], Pd, atol=1e-13)
    np.testing.assert_allclose(sg[:, :64], sd, atol=1e-13)


def test_windowed_dft_offset(orc):
    """A DFT window starting at m_off returns the same aliased bins shifted."""
    w = wl.SMALL16
    net = w.network()
    n, nS = orc.samples(net.T, net.r, net.seed_s, 0, 500)
    acc, cnt = orc.accumulate_gf(n, nS, 0, 4, 64)
    P0, s0, _ = orc.invert(acc, cnt, 0)
    P1, s1, _ = orc.invert(acc, cnt, 20)
    np.testing.assert_allclose(P1, np.roll(P0, -20, axis=1), atol=1e-14)


@pytest.mark.slow
def test_sampling_error_scale_matches_paper(orc):
    """Fig. 1 / Appendix A: lossless M = 200, r = 0.5 with 1.2e6 samples gives
    max errors < 6e-5.  Errors scale as 1/sqrt(E), so a 100x smaller ensemble
    must give max sigma below 10 x 6e-5.  The +P estimate on the same
    trajectories is far from converged: its actual error against the exact
    distribution is orders of magnitude larger (the paper: up to ~1000x)."""
    p = _paper()["matrixP_error_M200"]
    U = wl.haar_unitary(p["M"], 200)
    E = p["E"] // 100
    P, s, _ = orc.run(U, np.full(p["M"], p["r"]), 123, 0, E, p["n_sub"], 256)
    scaled = s[0].max() * math.sqrt(E / p["E"])
    assert 1e-6 < scaled < p["max_sigma"], scaled
    Pex = ex.negative_binomial(p["M"], p["r"], 256)
    err_mp = np.max(np.abs(P[0] - Pex))
    err_pp = np.max(np.abs(P[1] - Pex))
    assert err_mp < 6 * s[0].max()
    assert err_pp > 30 * err_mp, (err_pp, err_mp)
