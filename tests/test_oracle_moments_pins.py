"""Pins of the moments / marginals oracle (oracle/moments.py) to facts fixed
outside it: the generating-function identity that ties the per-trajectory
projectors to the per-trajectory moments, the exact vanishing of odd counts
for a single lossless squeezed mode, Wick's and Isserlis' theorems, the
textbook squeezed-vacuum distribution, and Monte-Carlo agreement with the
exact Gaussian moments and marginals."""
import math

import numpy as np
import pytest

import oracle.exact as ex
import oracle.moments as mo
import workloads as wl
from stats import agreement


def _falling(c, m):
    out = np.ones_like(c, dtype=np.float64)
    for q in range(m):
        out = out * (c - q)
    return out


def test_projector_factorial_moments_are_the_moment_samples():
    # sum_c z^c G_mP(c) = cosh(n + (z - 1) n') / cosh(n): its m-th derivative
    # at z = 1 is n'^m tanh(n)^(m mod 2); for +P, exp((z - 1) n') gives n'^m.
    rng = np.random.default_rng(3)
    E, M, cmax, mmax = 40, 3, 90, 5
    n = rng.uniform(-4.0, 4.0, size=E)
    n[:3] = [0.0, 1e-3, -25.0]
    occ = rng.normal(scale=1.5, size=(E, M)) + 1j * rng.normal(scale=1.5, size=(E, M))
    occ[0, 0] = 0.0
    G = mo.marginal_samples(n, occ, cmax)
    S = mo.moment_samples(n, occ, mmax)
    c = np.arange(cmax + 1)
    np.testing.assert_allclose(G.sum(axis=3), np.ones((2, E, M)), rtol=0, atol=1e-12)
    for m in range(1, mmax + 1):
        fm = (G * _falling(c, m)).sum(axis=3)
        np.testing.assert_allclose(fm, S[..., m - 1], rtol=1e-10, atol=1e-10)
    # even orders carry no weight: matrix-P equals +P per trajectory
    np.testing.assert_array_equal(S[0][..., 1::2], S[1][..., 1::2])
    assert np.max(np.abs(S[0][..., 0::2] - S[1][..., 0::2])) > 1e-3


def test_single_lossless_mode_has_no_odd_counts_per_trajectory(orc):
    T = np.array([[1.0 + 0j]])
    n, occ = mo.mode_samples(T, np.array([0.7]), 11, 0, 200)
    np.testing.assert_allclose(occ[:, 0], n, rtol=1e-15, atol=0)   # n' = n
    G = mo.marginal_samples(n, occ, 9)
    assert np.max(np.abs(G[0][..., 1::2])) < 1e-14
    assert np.max(np.abs(G[1][..., 1::2])) > 1e-2                    # +P is not exact here


def test_wick_and_isserlis():
    rng = np.random.default_rng(4)
    for _ in range(5):
        nb = rng.uniform(0.1, 2.0)
        mb = complex(rng.normal(), rng.normal())
        assert abs(mo.isserlis_moment(nb, mb, 1) - nb) < 1e-15
        # Wick: <a^dag a^dag a a> = 2 <a^dag a>^2 + |<a a>|^2
        assert abs(mo.isserlis_moment(nb, mb, 2) - (2 * nb ** 2 + abs(mb) ** 2)) < 1e-12
        # pairings grouped by the number k of (a, a) pairs
        for m in (3, 4, 5):
            closed = sum((math.comb(m, 2 * k) * math.prod(range(2 * k - 1, 0, -2))) ** 2
                         * math.factorial(m - 2 * k) * abs(mb) ** (2 * k) * nb ** (m - 2 * k)
                         for k in range(m // 2 + 1))
            assert abs(mo.isserlis_moment(nb, mb, m) - closed) < 1e-10 * closed


def test_squeezed_vacuum_textbook_distribution():
    r = np.array([0.3, 0.8, 1.1])
    T = np.eye(3, dtype=np.complex128)
    nbar, mbar = mo.mode_covariances(T, r)
    np.testing.assert_allclose(nbar, np.sinh(r) ** 2, rtol=1e-14)
    np.testing.assert_allclose(mbar, np.sinh(r) * np.cosh(r), rtol=1e-14)
    P = mo.exact_marginals(T, r, 20)
    for j, rj in enumerate(r):
        for c in range(21):
            if c % 2:
                ref = 0.0
            else:
                k = c // 2
                ref = (math.tanh(rj) ** c * math.factorial(c) / (2 ** k * math.factorial(k)) ** 2
                       / math.cosh(rj))
            assert abs(P[j, c] - ref) < 1e-13


def test_exact_marginals_and_moments_agree_and_sum_to_the_mean_count():
    net = wl.small_network(5, r=[0.4, 0.7, 0.5, 0.9, 0.3], t2=0.85, seed=21)
    mom = mo.exact_moments(net.T, net.r, 4)
    P = mo.exact_marginals(net.T, net.r, 400)   # geometric tails: ratio <= 0.8
    c = np.arange(401)
    for m in range(1, 5):
        np.testing.assert_allclose((P * _falling(c, m)).sum(axis=1), mom[:, m - 1], rtol=1e-10)
    assert abs(mom[:, 0].sum() - ex.mean_total_count(net.T, net.r)) < 1e-12
    # the series route against E1's DFT route for each mode's 2 x 2 block
    nbar, mbar = mo.mode_covariances(net.T, net.r)
    for j in range(5):
        mu = np.array([nbar[j] + abs(mbar[j]), nbar[j] - abs(mbar[j])])
        np.testing.assert_allclose(P[j, :60], ex.exact_unaliased(mu, 60), rtol=0, atol=1e-14)


@pytest.mark.parametrize("t2", [1.0, 0.8])
def test_monte_carlo_agrees_with_the_exact_gaussian_values(orc, t2):
    net = wl.small_network(4, r=[0.35, 0.5, 0.45, 0.3], t2=t2, seed=17)
    mmax, cmax = 4, 6
    mom, smom, marg, smarg = mo.run(net.T, net.r, net.seed_s, 0, 2 ** 15, 32, mmax, cmax)
    emom = mo.exact_moments(net.T, net.r, mmax)
    emarg = mo.exact_marginals(net.T, net.r, cmax)
    for est in (0, 1):
        res = agreement(mom[est].ravel(), smom[est].ravel(), emom.ravel(), bulk=0.0)
        assert res["ok"], (est, res)
        res = agreement(marg[est].ravel(), smarg[est].ravel(), emarg.ravel(), bulk=1e-4)
        assert res["ok"], (est, res)
    # the marginals of the parity estimator are the better ones (Appendix A)
    assert np.median(smarg[0][:, 2:]) < np.median(smarg[1][:, 2:])
