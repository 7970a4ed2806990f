"""Oracle of the two-dimensional binned count distribution.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

"Higher-dimensional binning" and Eq. General_GCP with d = 2: the output modes
are split into two bins S_1, S_2 (every mode in one of them, n~ = M) and the
observable is the joint probability G(m_1, m_2) of m_b photons counted in bin
b.  Per trajectory the c-number projectors of Eq. projection_op, summed over
the patterns with bin totals (m_1, m_2), have the generating function

    sum_{m_1, m_2} z_1^{m_1} z_2^{m_2} P_e(m_1, m_2)
        = cosh(n + (z_1 - 1) n_S1 + (z_2 - 1) n_S2) / cosh(n)     (matrix-P, M = 2)
        = exp((z_1 - 1) n_S1 + (z_2 - 1) n_S2)                     (+P),

n = sum_j alpha_j beta_j and n_Sb = sum_{i in S_b} alpha'_i beta'_i: the
one-dimensional form of Eq. c-number-variable with the exponent summed over
the bins (the parity weight depends on the total count m_1 + m_2).  The
generating function is evaluated at z_b = exp(2 pi i k_b / K_b) and inverted
by a two-dimensional DFT; sub-ensembles e mod N_R give the errors (Appendix A).

Plain numpy, FP64; the trajectories come from the C oracle
(``oracle.sample_amplitudes``).
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np

import oracle
import oracle.exact as ex


def bin_totals(T: np.ndarray, r: np.ndarray, seed: int, e0: int, E: int,
               bins: Sequence[int]) -> Tuple[np.ndarray, np.ndarray]:
    """n[E] and n_S[E, 2] (complex) of trajectories e0..e0+E-1; bins[i] in
    {0, 1} is the bin of output mode i."""
    bins = np.asarray(bins)
    n = np.zeros(E)
    nS = np.zeros((E, 2), dtype=np.complex128)
    for q in range(E):
        a, b, ap, bp = oracle.sample_amplitudes(T, r, seed, e0 + q)
        n[q] = float(np.dot(a, b))
        occ = ap * bp
        nS[q, 0] = occ[bins == 0].sum()
        nS[q, 1] = occ[bins == 1].sum()
    return n, nS


def gf2_sample(n: float, nS1: complex, nS2: complex, K1: int, K2: int):
    """(G_mP, G_+P), each [K1, K2], at z_b = exp(2 pi i k_b / K_b).  The
    cosh is written as [e^{L + c1} + e^{-L + c2}] / (1 + e^{-2|n|}) with
    c1 = min(0, 2n), c2 = -2 max(n, 0) (numerator and denominator times
    e^{-|n|}), L = (z_1 - 1) n_S1 + (z_2 - 1) n_S2."""
    z1 = np.exp(2j * np.pi * np.arange(K1) / K1)
    z2 = np.exp(2j * np.pi * np.arange(K2) / K2)
    L = (z1[:, None] - 1.0) * nS1 + (z2[None, :] - 1.0) * nS2
    c1 = min(0.0, 2.0 * n)
    c2 = -2.0 * max(n, 0.0)
    gp = np.exp(L)
    gm = (np.exp(L + c1) + np.exp(-L + c2)) / (1.0 + np.exp(-2.0 * abs(n)))
    return gm, gp


def accumulate(n: np.ndarray, nS: np.ndarray, e0: int, n_sub: int, K1: int, K2: int):
    """Sub-ensemble sums acc[2][n_sub][K1][K2] and counts[n_sub]; trajectory
    e0 + q belongs to sub-ensemble (e0 + q) mod n_sub."""
    acc = np.zeros((2, n_sub, K1, K2), dtype=np.complex128)
    cnt = np.zeros(n_sub, dtype=np.int64)
    for q in range(n.shape[0]):
        rr = (e0 + q) % n_sub
        gm, gp = gf2_sample(n[q], nS[q, 0], nS[q, 1], K1, K2)
        acc[0, rr] += gm
        acc[1, rr] += gp
        cnt[rr] += 1
    return acc, cnt


def invert(acc: np.ndarray, cnt: np.ndarray, m_off=(0, 0)):
    """P[2][K1][K2] (mean over sub-ensembles of the real part) and sigma
    (sample standard deviation / sqrt(N_R)) for m_b = m_off_b .. + K_b - 1:
    P_r(m_1, m_2) = (1/(K1 K2)) sum_k <G>_r(z) z_1^{-m_1} z_2^{-m_2}."""
    _, n_sub, K1, K2 = acc.shape
    mean = acc / cnt[None, :, None, None]
    Pr = np.fft.fft2(mean, axes=(2, 3)) / (K1 * K2)       # sum_k x_k e^{-2 pi i k m / K}
    i1 = (m_off[0] + np.arange(K1)) % K1
    i2 = (m_off[1] + np.arange(K2)) % K2
    Pr = Pr[:, :, i1][:, :, :, i2].real
    P = Pr.mean(axis=1)
    sig = Pr.std(axis=1, ddof=1) / np.sqrt(n_sub) if n_sub > 1 else np.zeros_like(P)
    return P, sig


def run(T, r, seed, e0, E, n_sub, K1, K2, bins, m_off=(0, 0)):
    n, nS = bin_totals(T, r, seed, e0, E, bins)
    acc, cnt = accumulate(n, nS, e0, n_sub, K1, K2)
    return invert(acc, cnt, m_off)


def exact_bruteforce(T: np.ndarray, r: np.ndarray, bins: Sequence[int], K1: int, K2: int,
                     total_max: int, pure_U=None) -> np.ndarray:
    """Exact G(m_1, m_2) for m_b < K_b by summing Hafnian pattern
    probabilities (oracle.exact) over every pattern with total <= total_max
    (tiny M only)."""
    bins = np.asarray(bins)
    M = T.shape[0]
    out = np.zeros((K1, K2))
    for tot in range(total_max + 1):
        for c in ex._compositions(tot, M):
            c = np.asarray(c)
            m1 = int(c[bins == 0].sum())
            m2 = int(c[bins == 1].sum())
            if m1 >= K1 or m2 >= K2:
                continue
            if pure_U is not None:
                p = ex.pattern_probability_pure(pure_U, r, c)
            else:
                p = ex.pattern_probability(T, r, c)
            out[m1, m2] += p
    return out
