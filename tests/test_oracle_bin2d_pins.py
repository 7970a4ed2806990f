"""Pins of the two-dimensional binning oracle (oracle/bin2d.py): the joint
distribution against brute-force Hafnian pattern sums, and the identities
that tie it to the one-dimensional estimator on the same trajectories
(marginal = the distribution of one bin, anti-diagonal sums = the total
count), the lossless parity selection of "Higher-dimensional binning", and
the per-trajectory generating function at z_2 = 1 against the C oracle."""
import numpy as np
import pytest

import oracle.bin2d as b2
import workloads as wl
from stats import agreement

BINS4 = [0, 0, 1, 1]


def _tiny(t2, seed):
    net = wl.small_network(4, r=[0.3, 0.4, 0.35, 0.25], t2=t2, seed=seed)
    U = wl.haar_unitary(4, wl.SEED_U_BASE + 500 + seed)
    return net, U


@pytest.mark.parametrize("t2", [1.0, 0.8])
def test_joint_distribution_matches_hafnian_pattern_sums(orc, t2):
    net, U = _tiny(t2, 31)
    K = 16
    P, sig = b2.run(net.T, net.r, net.seed_s, 0, 2 ** 15, 16, K, K, BINS4)
    # complete pattern sums up to total 8 (pure-state Hafnians of order <= 8)
    # or 6 (mixed-state Hafnians of order <= 12)
    tmax = 8 if t2 == 1.0 else 6
    exact = b2.exact_bruteforce(net.T, net.r, BINS4, K, K, total_max=tmax,
                                pure_U=U if t2 == 1.0 else None)
    assert exact.sum() > 1.0 - 1e-3     # mass beyond tmax
    m1, m2 = np.meshgrid(np.arange(K), np.arange(K), indexing="ij")
    sel = (m1 + m2) <= tmax              # bins where the pattern sum is complete
    # the matrix-P estimate (as in the one-dimensional pins; the +P estimate's
    # heavy tails make its sample sigma an unreliable error bar, the paper's
    # point, and the identity pins below cover both estimators)
    res = agreement(P[0][sel], sig[0][sel], exact[sel], bulk=1e-3)
    assert res["ok"], res
    assert abs(P[0].sum() - 1.0) < 1e-12


def test_marginal_is_the_one_bin_distribution(orc):
    net = wl.small_network(6, r=0.6, t2=0.9, seed=8)
    bins = [0, 1, 0, 1, 1, 0]
    E, n_sub, K = 3000, 5, 32
    P2, _ = b2.run(net.T, net.r, net.seed_s, 7, E, n_sub, K, K, bins)
    rows0 = [i for i, b in enumerate(bins) if b == 0]
    P1, _, _ = orc.run(net.T[rows0], net.r, net.seed_s, 7, E, n_sub, K)
    np.testing.assert_allclose(P2.sum(axis=2), P1, rtol=0, atol=1e-12)


def test_antidiagonal_sums_are_the_total_count(orc):
    net = wl.small_network(6, r=0.6, t2=0.9, seed=9)
    bins = [1, 1, 0, 0, 1, 0]
    E, n_sub, K = 3000, 5, 32
    P2, _ = b2.run(net.T, net.r, net.seed_s, 3, E, n_sub, K, K, bins)
    Pt, _, _ = orc.run(net.T, net.r, net.seed_s, 3, E, n_sub, K)
    diag = np.zeros((2, K))
    for m1 in range(K):
        for m2 in range(K):
            diag[:, (m1 + m2) % K] += P2[:, m1, m2]
    np.testing.assert_allclose(diag, Pt, rtol=0, atol=1e-12)


def test_lossless_odd_totals_vanish(orc):
    net = wl.small_network(8, r=0.5, t2=1.0, seed=10)
    bins = [0, 0, 0, 0, 1, 1, 1, 1]
    P2, _ = b2.run(net.T, net.r, net.seed_s, 0, 500, 4, 32, 32, bins)
    m1, m2 = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    odd = (m1 + m2) % 2 == 1
    assert np.max(np.abs(P2[0][odd])) < 1e-12
    assert np.max(np.abs(P2[0][~odd])) > 1e-3


def test_generating_function_at_z2_equal_1_is_the_one_dimensional_one(orc):
    for n, s1, s2 in ((3.2, 2.5 + 0.3j, 0.4 - 0.1j), (-1.1, 0.7 - 0.2j, 1.9 + 0.5j)):
        gm, gp = b2.gf2_sample(n, s1, s2, 32, 16)
        gm1, gp1 = orc.gf_sample(n, s1, 32)
        np.testing.assert_allclose(gm[:, 0], gm1, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(gp[:, 0], gp1, rtol=1e-12, atol=1e-14)
