"""Exact (sampling-free) total-count references for Gaussian boson sampling.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

E1  General Gaussian determinant.  For squeezed vacua r_j through a linear
    network T (M x N), the normally-ordered moments of the outputs are those
    of a complex Gaussian field zeta = (alpha, alpha*) with covariance
        C = [[T Dn T^H, T Dm T^T], [T* Dm T^H, T* Dn T^T]],
    Dn = diag(sinh^2 r), Dm = diag(sinh r cosh r).  The total-count
    generating function <z^{n_hat}> = <:exp((z-1) n_hat):> is the Gaussian
    integral det(I + (1-z) C)^{-1/2} = prod_k (1 + (1-z) mu_k)^{-1/2}, mu_k the
    (real) eigenvalues of the Hermitian C.  On |z| = 1 every factor has a
    positive real part (mu_k > -1/2), so the principal square root of each
    factor is the continuous branch from z = 1.
E2  Uniform loss T = t U: C = t^2 W [[Dn, Dm], [Dm, Dn]] W^H with W unitary,
    so mu = {t^2 sinh r_j e^{r_j}, -t^2 sinh r_j e^{-r_j}} (independent of U).
    This is the uniform-loss exact distribution the paper cites after Eq.
    Exact_multi_mode_squeezed_state.
E3  Lossless, uniform squeezing: Eq. Exact_multi_mode_squeezed_state, the
    negative binomial in m/2 with p_S = 1/(1 + sinh^2 r), zero for odd m.
E4  Brute-force Hafnian probabilities of single output patterns (Hamilton et
    al., PRL 119, 170501 (2017); Kruse et al., PRA 100, 032326 (2019)):
    Pr(c) = Haf(A_c) / (c! sqrt(det sigma_Q)), sigma_Q = sigma + I/2,
    A = X (I - sigma_Q^{-1}); summed over patterns with sum c = m.

P(m) from a generating function: P(m) = (1/K1) sum_k G(z_k) z_k^{-m}, the
aliased distribution sum_j P(m + j K1); with K1 beyond the support it is P(m).
"""
from __future__ import annotations

import itertools
import math
from typing import Iterable

import numpy as np
from scipy.special import gammaln


# ----------------------------------------------------------------------------
# E1 / E2 eigenvalues and generating functions
# ----------------------------------------------------------------------------
def covariance_normal_ordered(T: np.ndarray, r: np.ndarray) -> np.ndarray:
    """C of E1 (2M x 2M Hermitian)."""
    T = np.asarray(T, dtype=np.complex128)
    r = np.asarray(r, dtype=np.float64)
    Dn = np.diag(np.sinh(r) ** 2)
    Dm = np.diag(np.sinh(r) * np.cosh(r))
    Tc = T.conj()
    top = np.hstack([T @ Dn @ Tc.T, T @ Dm @ T.T])
    bot = np.hstack([Tc @ Dm @ Tc.T, Tc @ Dn @ T.T])
    return np.vstack([top, bot])


def eigenvalues_general(T: np.ndarray, r: np.ndarray) -> np.ndarray:
    """mu_k of E1 via a Hermitian eigensolver."""
    C = covariance_normal_ordered(T, r)
    return np.linalg.eigvalsh(C)


def eigenvalues_uniform_loss(r: np.ndarray, t2: float) -> np.ndarray:
    """mu_k of E2 for T = t U."""
    r = np.asarray(r, dtype=np.float64)
    s = np.sinh(r)
    return np.concatenate([t2 * s * np.exp(r), -t2 * s * np.exp(-r)])


def gf_from_eigenvalues(mu: np.ndarray, z: np.ndarray) -> np.ndarray:
    """G(z) = prod_k (1 + (1-z) mu_k)^{-1/2}, summed in log space."""
    z = np.asarray(z, dtype=np.complex128)
    w = (1.0 - z)[:, None] * np.asarray(mu, dtype=np.float64)[None, :]
    logG = -0.5 * np.log(1.0 + w).sum(axis=1)  # principal Log of each factor
    return np.exp(logG)


def roots_of_unity(K1: int) -> np.ndarray:
    k = np.arange(K1)
    th = 2.0 * np.pi * k / K1
    return np.cos(th) + 1j * np.sin(th)


def distribution_from_gf(G: np.ndarray, m_off: int = 0) -> np.ndarray:
    """P(m), m = m_off..m_off+K1-1, from G at the K1 roots of unity (aliased)."""
    K1 = G.shape[0]
    # (1/K1) sum_k G_k z_k^{-m} is numpy's forward FFT divided by K1
    p = np.fft.fft(G) / K1
    idx = (m_off + np.arange(K1)) % K1
    return p[idx]


def exact_distribution(mu: np.ndarray, K1: int, m_off: int = 0) -> np.ndarray:
    """Aliased exact P(m) (complex; imaginary part is rounding) on K1 points."""
    return distribution_from_gf(gf_from_eigenvalues(mu, roots_of_unity(K1)), m_off)


def exact_unaliased(mu: np.ndarray, mmax: int) -> np.ndarray:
    """Exact P(m), m = 0..mmax-1, with K1 large enough that aliasing is below
    double rounding (K1 = power of two >= 8 * max(mmax, mean + 40 sd))."""
    # cumulants of the total count from log G(e^s): mean = sum(mu)/2,
    # variance = sum(mu + mu^2)/2
    mean = 0.5 * float(np.sum(mu))
    var = 0.5 * float(np.sum(mu + mu ** 2))
    hi = max(mmax, int(mean + 40.0 * math.sqrt(max(var, 1.0))) + 64)
    K1 = 1 << int(math.ceil(math.log2(8 * hi)))
    return exact_distribution(mu, K1)[:mmax].real


# ----------------------------------------------------------------------------
# E3 negative binomial (Eq. Exact_multi_mode_squeezed_state)
# ----------------------------------------------------------------------------
def negative_binomial(M: int, r: float, mmax: int) -> np.ndarray:
    """P(m) for m = 0..mmax-1, lossless, M modes of squeezing r."""
    nbar = math.sinh(r) ** 2
    p = 1.0 / (1.0 + nbar)
    out = np.zeros(mmax)
    for m in range(0, mmax, 2):
        k = m // 2
        logc = gammaln(M / 2.0 + k) - gammaln(k + 1.0) - gammaln(M / 2.0)
        out[m] = math.exp(logc + (M / 2.0) * math.log(p) + k * math.log1p(-p))
    return out


def cutoffs(P: np.ndarray, thresh: float = 1e-7):
    """(m_min, m_max): first and last m with P(m) >= thresh."""
    idx = np.nonzero(P >= thresh)[0]
    return int(idx[0]), int(idx[-1])


# ----------------------------------------------------------------------------
# E4 brute-force Hafnians
# ----------------------------------------------------------------------------
def hafnian(A: np.ndarray) -> complex:
    """Sum over perfect matchings of prod A[i, j] (recursive expansion on the
    first index).  Exponential: for matrices up to ~12 x 12."""
    n = A.shape[0]
    if n == 0:
        return 1.0
    if n % 2:
        return 0.0
    total = 0.0
    rest = list(range(1, n))
    for pos, j in enumerate(rest):
        others = rest[:pos] + rest[pos + 1:]
        sub = A[np.ix_(others, others)]
        total = total + A[0, j] * hafnian(sub)
    return total


def gaussian_sigma(T: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Complex covariance sigma in the basis (a_1..a_M, a_1^+..a_M^+), vacuum
    = I/2: sigma = C + I/2 with C the normally-ordered covariance of E1."""
    C = covariance_normal_ordered(T, r)
    return C + 0.5 * np.eye(C.shape[0])


def pattern_probability(T: np.ndarray, r: np.ndarray, c: Iterable[int]) -> float:
    """Pr(c) of a photon-number pattern c (length M) by the mixed-state
    Hafnian formula of Kruse et al. (2019)."""
    c = list(c)
    M = len(c)
    sigma = gaussian_sigma(T, r)
    sQ = sigma + 0.5 * np.eye(2 * M)
    X = np.block([[np.zeros((M, M)), np.eye(M)], [np.eye(M), np.zeros((M, M))]])
    A = X @ (np.eye(2 * M) - np.linalg.inv(sQ))
    rows = []
    for i, ci in enumerate(c):
        rows += [i] * ci
    rows = rows + [i + M for i in rows]
    Ac = A[np.ix_(rows, rows)]
    fact = 1.0
    for ci in c:
        fact *= math.factorial(ci)
    val = hafnian(Ac) / (fact * np.sqrt(np.linalg.det(sQ)))
    return float(np.real(val))


def pattern_probability_pure(U: np.ndarray, r: np.ndarray, c: Iterable[int]) -> float:
    """Lossless pure-state formula (Hamilton et al. 2017):
    Pr(c) = |Haf(B_c)|^2 / (c! prod_j cosh r_j), B = U diag(tanh r) U^T."""
    c = list(c)
    B = U @ np.diag(np.tanh(r)) @ U.T
    rows = []
    for i, ci in enumerate(c):
        rows += [i] * ci
    Bc = B[np.ix_(rows, rows)]
    fact = 1.0
    for ci in c:
        fact *= math.factorial(ci)
    return float(abs(hafnian(Bc)) ** 2 / (fact * np.prod(np.cosh(r))))


def total_count_bruteforce(T: np.ndarray, r: np.ndarray, mmax: int, pure_U=None) -> np.ndarray:
    """P(m) for m = 0..mmax-1 by summing pattern probabilities over all
    patterns with total m (tiny M only)."""
    M = T.shape[0]
    out = np.zeros(mmax)
    for m in range(mmax):
        s = 0.0
        for c in _compositions(m, M):
            if pure_U is not None:
                s += pattern_probability_pure(pure_U, r, c)
            else:
                s += pattern_probability(T, r, c)
        out[m] = s
    return out


def _compositions(m: int, parts: int):
    """All tuples of `parts` non-negative ints summing to m."""
    for bars in itertools.combinations(range(m + parts - 1), parts - 1):
        prev = -1
        out = []
        for b in bars:
            out.append(b - prev - 1)
            prev = b
        out.append(m + parts - 1 - prev - 1)
        yield tuple(out)


def mean_total_count(T: np.ndarray, r: np.ndarray) -> float:
    """<n_hat> = tr(T Dn T^H) for squeezed vacua through T."""
    T = np.asarray(T, dtype=np.complex128)
    return float(np.real(np.trace(T @ np.diag(np.sinh(r) ** 2) @ T.conj().T)))
