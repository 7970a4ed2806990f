"""The synthetic input recipe (workloads/): Haar unitaries, the batched
networks' parameter draws, and the DFT windows they are run with.

The window check uses the exact total-count distribution of a uniform-loss
network (its generating function depends on r and t^2 only), so it needs no
unitary: the mass the window leaves out must be at rounding level, and a
window a quarter as wide must visibly miss mass.  No GPU needed.
"""
import math

import numpy as np

import oracle.exact as ex
import workloads as wl


def test_haar_unitary_is_unitary_and_seeded():
    U = wl.haar_unitary(64, 5)
    assert np.max(np.abs(U.conj().T @ U - np.eye(64))) < 1e-12
    assert np.array_equal(U, wl.haar_unitary(64, 5))
    assert not np.array_equal(U, wl.haar_unitary(64, 6))
    # unit columns: the mean of |U_ij|^2 is exactly 1/m
    assert abs(np.mean(np.abs(U) ** 2) - 1.0 / 64) < 1e-12
    # phase-fixed QR: the diagonal phases are not all trivial (no R-sign bias)
    assert np.std(np.angle(np.diagonal(U))) > 0.5


def test_batched_networks_follow_the_recipe():
    ws = wl.batched_networks()
    assert len(ws) == 64
    Ns = np.array([w.N for w in ws])
    assert np.all(Ns == np.array([w.M for w in ws]))
    assert Ns.min() >= 100 and Ns.max() <= 2000
    # log-uniform: about half the networks below the geometric midpoint
    assert 20 <= np.sum(Ns < math.sqrt(100 * 2000)) <= 44
    t2 = np.array([w.t2 for w in ws])
    assert t2.min() >= 0.25 and t2.max() <= 0.995 ** 2
    assert all(w.E == 2 ** 18 and w.n_sub == 64 for w in ws)
    for w in ws[:4]:
        r = w.squeezing()
        assert r.shape == (w.N,) and r.min() >= 0.5 and r.max() <= 1.5
        assert np.array_equal(r, w.squeezing())
        assert np.array_equal(r, w.network().r)


def _window(w):
    r = w.squeezing()
    K1, off = wl.dft_window(w.N, float(r.max()), w.t2, float(np.mean(np.sinh(r) ** 2)))
    return ex.eigenvalues_uniform_loss(r, w.t2), K1, off


def _mass_outside(mu, K1, a, width):
    """Exact probability of counts outside [a, a + width), from the
    distribution on 2 K1 points (aliasing negligible when K1 covers it)."""
    lo = max(0, a - K1 // 2)
    P = ex.exact_distribution(mu, 2 * K1, lo).real
    m = lo + np.arange(2 * K1)
    return float(P[(m < a) | (m >= a + width)].sum())


def test_dft_windows_cover_the_batched_networks_support():
    ws = sorted(wl.batched_networks(), key=lambda w: w.N)
    # the smallest and largest networks and some between (every K1 that occurs)
    for w in [ws[0], ws[9], ws[21], ws[33], ws[45], ws[-1]]:
        mu, K1, off = _window(w)
        assert abs(_mass_outside(mu, K1, off, K1)) < 1e-11, w.name
    # the check sees missing mass: +-3 standard deviations around the mean
    # leave out about 3e-3
    mu, K1, _ = _window(ws[-1])
    mean = 0.5 * float(np.sum(mu))
    sd = math.sqrt(0.5 * float(np.sum(mu + mu ** 2)))
    assert _mass_outside(mu, K1, int(mean - 3 * sd), int(6 * sd)) > 1e-3


def test_count_windows_cover_the_batched_networks_support():
    """count_window (the batch bench's windows, from the count's own mean and
    variance) is tighter than dft_window yet leaves out no mass above
    rounding."""
    ws = sorted(wl.batched_networks(), key=lambda w: w.N)
    for w in ws[::8] + [ws[-1]]:
        r = w.squeezing()
        K1, off = wl.count_window(r, w.t2)
        K0, _ = _window(w)[1:]
        assert K1 <= K0
        mu = ex.eigenvalues_uniform_loss(r, w.t2)
        assert abs(_mass_outside(mu, K1, off, K1)) < 1e-11, w.name
