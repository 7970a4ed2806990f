"""Oracle of the d-dimensional binned count distribution (2 <= d <= 4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

"Higher-dimensional binning" and Eq. General_GCP for general d: the output
modes are split into d bins S_1 .. S_d (every mode in one of them) and the
observable is the joint probability G(m_1, .., m_d) of m_b photons counted
in bin b.  Per trajectory the c-number projectors of Eq. projection_op,
summed over the patterns with bin totals (m_1, .., m_d), have the
generating function

    sum_m prod_b z_b^{m_b} P_e(m) = cosh(n + sum_b (z_b - 1) n_Sb) / cosh(n)   (matrix-P)
                                  = exp(sum_b (z_b - 1) n_Sb)                 (+P),

n = sum_j alpha_j beta_j, n_Sb = sum_{i in S_b} alpha'_i beta'_i (the
one-dimensional form of Eq. c-number-variable with the exponent summed over
the bins).  It is evaluated at z_b = exp(2 pi i k_b / K_b) and inverted by a
d-dimensional DFT; sub-ensembles e mod N_R give the errors (Appendix A).
For d = 2 this is ``oracle.bin2d``.

Plain numpy, FP64; the trajectories come from the C oracle
(``oracle.sample_amplitudes``).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

import oracle
import oracle.exact as ex


def bin_totals(T: np.ndarray, r: np.ndarray, seed: int, e0: int, E: int, bins: Sequence[int]):
    """n[E] and n_S[E, d] (complex) of trajectories e0..e0+E-1; bins[i] in
    0..d-1 is the bin of output mode i (d = max(bins) + 1)."""
    bins = np.asarray(bins)
    d = int(bins.max()) + 1
    n = np.zeros(E)
    nS = np.zeros((E, d), dtype=np.complex128)
    for q in range(E):
        a, b, ap, bp = oracle.sample_amplitudes(T, r, seed, e0 + q)
        n[q] = float(np.dot(a, b))
        occ = ap * bp
        for k in range(d):
            nS[q, k] = occ[bins == k].sum()
    return n, nS


def gf_sample(n: float, nS: Sequence[complex], K: Sequence[int]):
    """(G_mP, G_+P), each of shape K, at z_b = exp(2 pi i k_b / K_b).  The
    cosh is written as [e^{L + c1} + e^{-L + c2}] / (1 + e^{-2|n|}) with
    c1 = min(0, 2n), c2 = -2 max(n, 0) (numerator and denominator times
    e^{-|n|}), L = sum_b (z_b - 1) n_Sb."""
    d = len(K)
    L = np.zeros(tuple(K), dtype=np.complex128)
    for b in range(d):
        z = np.exp(2j * np.pi * np.arange(K[b]) / K[b])
        shape = [1] * d
        shape[b] = K[b]
        L = L + ((z - 1.0) * nS[b]).reshape(shape)
    c1 = min(0.0, 2.0 * n)
    c2 = -2.0 * max(n, 0.0)
    gp = np.exp(L)
    gm = (np.exp(L + c1) + np.exp(-L + c2)) / (1.0 + np.exp(-2.0 * abs(n)))
    return gm, gp


def accumulate(n: np.ndarray, nS: np.ndarray, e0: int, n_sub: int, K: Sequence[int]):
    """Sub-ensemble sums acc[2][n_sub][K...] and counts[n_sub]; trajectory
    e0 + q belongs to sub-ensemble (e0 + q) mod n_sub."""
    acc = np.zeros((2, n_sub) + tuple(K), dtype=np.complex128)
    cnt = np.zeros(n_sub, dtype=np.int64)
    for q in range(n.shape[0]):
        rr = (e0 + q) % n_sub
        gm, gp = gf_sample(n[q], nS[q], K)
        acc[0, rr] += gm
        acc[1, rr] += gp
        cnt[rr] += 1
    return acc, cnt


def invert(acc: np.ndarray, cnt: np.ndarray, m_off: Sequence[int]):
    """P[2][K...] (mean over sub-ensembles of the real part) and sigma
    (sample standard deviation / sqrt(N_R)) for m_b = m_off_b .. + K_b - 1:
    P_r(m) = (1/prod K_b) sum_k <G>_r(z) prod_b z_b^{-m_b}."""
    n_sub = acc.shape[1]
    K = acc.shape[2:]
    d = len(K)
    mean = acc / cnt.reshape((1, n_sub) + (1,) * d)
    Pr = np.fft.fftn(mean, axes=tuple(range(2, 2 + d))) / float(np.prod(K))
    for b in range(d):
        idx = (m_off[b] + np.arange(K[b])) % K[b]
        Pr = np.take(Pr, idx, axis=2 + b)
    Pr = Pr.real
    P = Pr.mean(axis=1)
    sig = Pr.std(axis=1, ddof=1) / np.sqrt(n_sub) if n_sub > 1 else np.zeros_like(P)
    return P, sig


def run(T, r, seed, e0, E, n_sub, K, bins, m_off=None):
    K = list(K)
    m_off = [0] * len(K) if m_off is None else list(m_off)
    n, nS = bin_totals(T, r, seed, e0, E, bins)
    acc, cnt = accumulate(n, nS, e0, n_sub, K)
    return invert(acc, cnt, m_off)


def exact_bruteforce(T: np.ndarray, r: np.ndarray, bins: Sequence[int], K: Sequence[int],
                     total_max: int, pure_U=None) -> np.ndarray:
    """Exact G(m) for m_b < K_b by summing Hafnian pattern probabilities
    (oracle.exact) over every pattern with total <= total_max (tiny M only)."""
    bins = np.asarray(bins)
    d = len(K)
    M = T.shape[0]
    out = np.zeros(tuple(K))
    for tot in range(total_max + 1):
        for c in ex._compositions(tot, M):
            c = np.asarray(c)
            m = tuple(int(c[bins == b].sum()) for b in range(d))
            if any(m[b] >= K[b] for b in range(d)):
                continue
            if pure_U is not None:
                p = ex.pattern_probability_pure(pure_U, r, c)
            else:
                p = ex.pattern_probability(T, r, c)
            out[m] += p
    return out
