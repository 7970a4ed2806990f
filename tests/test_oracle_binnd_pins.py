"""Pins of the d-dimensional binning oracle (oracle/binnd.py): the joint
distribution of three bins against brute-force Hafnian pattern sums, and the
identities that tie it to fewer bins on the same trajectories (summing out a
bin = leaving its modes unobserved, merging two bins = summing along their
anti-diagonals), the lossless parity selection, and d = 2 against the
two-bin oracle."""
import numpy as np
import pytest

import oracle.bin2d as b2
import oracle.binnd as bn
import workloads as wl
from stats import agreement

BINS6 = [0, 0, 1, 1, 2, 2]


def _tiny(t2, seed):
    net = wl.small_network(6, r=[0.3, 0.4, 0.35, 0.25, 0.3, 0.2], t2=t2, seed=seed)
    U = wl.haar_unitary(6, wl.SEED_U_BASE + 500 + seed)
    return net, U


@pytest.mark.parametrize("t2", [1.0, 0.8])
def test_three_bins_match_hafnian_pattern_sums(orc, t2):
    net, U = _tiny(t2, 41)
    K = (8, 8, 8)
    P, sig = bn.run(net.T, net.r, net.seed_s, 0, 2 ** 14, 16, K, BINS6)
    # complete pattern sums up to total 6 (pure-state Hafnians of order <= 6)
    # or 4 (mixed-state Hafnians of order <= 8)
    tmax = 6 if t2 == 1.0 else 4
    exact = bn.exact_bruteforce(net.T, net.r, BINS6, K, total_max=tmax,
                                pure_U=U if t2 == 1.0 else None)
    assert exact.sum() > 1.0 - 2e-2
    m = np.indices(K)
    sel = m.sum(axis=0) <= tmax
    res = agreement(P[0][sel], sig[0][sel], exact[sel], bulk=1e-3)
    assert res["ok"], res
    assert abs(P[0].sum() - 1.0) < 1e-12


def test_summing_out_a_bin_leaves_its_modes_unobserved(orc):
    net = wl.small_network(6, r=0.6, t2=0.9, seed=12)
    E, n_sub, K = 1500, 5, (16, 16, 16)
    P3, _ = bn.run(net.T, net.r, net.seed_s, 7, E, n_sub, K, BINS6)
    keep = [i for i, b in enumerate(BINS6) if b < 2]
    P2, _ = b2.run(net.T[keep], net.r, net.seed_s, 7, E, n_sub, 16, 16,
                   [BINS6[i] for i in keep])
    np.testing.assert_allclose(P3.sum(axis=3), P2, rtol=0, atol=1e-12)


def test_merging_two_bins_sums_their_antidiagonals(orc):
    net = wl.small_network(6, r=0.6, t2=0.9, seed=13)
    E, n_sub, K = 1500, 5, 16
    P3, _ = bn.run(net.T, net.r, net.seed_s, 3, E, n_sub, (K, K, K), BINS6)
    merged = [0 if b == 0 else 1 for b in BINS6]
    P2, _ = b2.run(net.T, net.r, net.seed_s, 3, E, n_sub, K, K, merged)
    got = np.zeros((2, K, K))
    for m2 in range(K):
        for m3 in range(K):
            got[:, :, (m2 + m3) % K] += P3[:, :, m2, m3]
    np.testing.assert_allclose(got, P2, rtol=0, atol=1e-12)


def test_lossless_odd_totals_vanish(orc):
    net = wl.small_network(6, r=0.5, t2=1.0, seed=14)
    P3, _ = bn.run(net.T, net.r, net.seed_s, 0, 400, 4, (16, 16, 16), BINS6)
    m = np.indices((16, 16, 16))
    odd = m.sum(axis=0) % 2 == 1
    assert np.max(np.abs(P3[0][odd])) < 1e-12
    assert np.max(np.abs(P3[0][~odd])) > 1e-3


def test_two_bins_are_the_two_bin_oracle(orc):
    net = wl.small_network(6, r=0.6, t2=0.9, seed=15)
    bins = [0, 1, 1, 0, 1, 0]
    Pn, sn = bn.run(net.T, net.r, net.seed_s, 5, 800, 4, (16, 32), bins, m_off=(3, 1))
    P2, s2 = b2.run(net.T, net.r, net.seed_s, 5, 800, 4, 16, 32, bins, m_off=(3, 1))
    np.testing.assert_allclose(Pn, P2, rtol=0, atol=1e-13)
    np.testing.assert_allclose(sn, s2, rtol=0, atol=1e-13)
