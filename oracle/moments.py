"""Oracle of the normally-ordered photon-count moments and the single-mode
count marginals.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Moments, Eq. moment ("Photon-counting observables"): for output mode j,

    <:n_j^m:> = < (alpha'_j beta'_j)^m  tr[T^{p_m} Omega] >,   p_m = m mod 2,

with the averaging over the phase-space trajectories.  In the parity case
(M = 2) used for squeezed inputs ("Applications to GBS") Omega_00 = 1 and
T_0 = tanh(n), n = sum_k alpha_k beta_k, so a trajectory contributes

    matrix-P:  (n'_j)^m tanh(n)^{p_m},     +P:  (n'_j)^m,

n'_j = alpha'_j beta'_j.  Even orders carry no weight, so they coincide with
+P trajectory by trajectory.

Marginals: the single-mode count probability P_j(c) = <G(c)> with the
projector of Eq. projection_op for the set S = {j}.  Per trajectory it is the
c-number projector of Eq. c-number-variable with n_S = n'_j:

    matrix-P:  g_0(n'_j, c) (n'_j)^c e^{-n'_j} / c!,
               g_0 = (1 + (-1)^c e^{2(n'_j - n)}) / (1 + e^{-2n}),
    +P:        (n'_j)^c e^{-n'_j} / c!          (Eq. phase_space_projector).

Statistics (Appendix A): trajectory e belongs to sub-ensemble e mod N_R; the
estimate is the mean over sub-ensembles of the real part of the sub-ensemble
mean, its error the sample standard deviation over sub-ensembles divided by
sqrt(N_R).

Exact references for a Gaussian state (E1 of ``oracle.exact``): the output
modes' normally-ordered covariances nbar_j = <a_j^dag a_j> = (T Dn T^H)_jj and
mbar_j = <a_j a_j> = (T Dm T^T)_jj; the moments follow from Isserlis' theorem
(sum over all pairings of m conjugate and m plain amplitudes), the marginal
from the single-mode determinant formula with eigenvalues nbar_j +- |mbar_j|.

Plain numpy, FP64; the trajectories come from the C oracle
(``oracle.sample_amplitudes``).
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np
from scipy.special import gammaln

import oracle
import oracle.exact as ex


# ----------------------------------------------------------------------------
# Trajectories
# ----------------------------------------------------------------------------
def mode_samples(T: np.ndarray, r: np.ndarray, seed: int, e0: int, E: int):
    """n[E] (input totals) and occ[E, M] = alpha'_j beta'_j of trajectories
    e0 .. e0+E-1."""
    M = T.shape[0]
    n = np.zeros(E)
    occ = np.zeros((E, M), dtype=np.complex128)
    for q in range(E):
        a, b, ap, bp = oracle.sample_amplitudes(T, r, seed, e0 + q)
        n[q] = float(np.dot(a, b))
        occ[q] = ap * bp
    return n, occ


# ----------------------------------------------------------------------------
# Per-trajectory values
# ----------------------------------------------------------------------------
def moment_samples(n: np.ndarray, occ: np.ndarray, mmax: int) -> np.ndarray:
    """[2][E][M][mmax] complex: the trajectories' contributions to
    <:n_j^m:>, m = 1..mmax (matrix-P, +P)."""
    E, M = occ.shape
    out = np.zeros((2, E, M, mmax), dtype=np.complex128)
    w = np.tanh(n)[:, None]
    for m in range(1, mmax + 1):
        pw = occ ** m
        p_m = m % 2
        out[0, :, :, m - 1] = pw * (w ** p_m)
        out[1, :, :, m - 1] = pw
    return out


def marginal_samples(n: np.ndarray, occ: np.ndarray, cmax: int) -> np.ndarray:
    """[2][E][M][cmax+1] complex: per-trajectory projectors G(c), c = 0..cmax
    (matrix-P, +P).  The g_0 factor is applied as written, with numerator and
    denominator multiplied by e^{n - |n|} so that no exponential overflows:
    G_mP(c) = [e^{L - n'} e^{n - |n|} + (-1)^c e^{L + n' - 2n} e^{n - |n|}]
              / (1 + e^{-2|n|}),  L = c Log(n') - log c!."""
    E, M = occ.shape
    out = np.zeros((2, E, M, cmax + 1), dtype=np.complex128)
    nn = n[:, None]
    shift = nn - np.abs(nn)
    den = 1.0 + np.exp(-2.0 * np.abs(nn))
    zero = occ == 0
    logocc = np.log(np.where(zero, 1.0, occ))
    for c in range(cmax + 1):
        L = c * logocc - gammaln(c + 1.0)
        sign = 1.0 if c % 2 == 0 else -1.0
        gm = (np.exp(L - occ + shift) + sign * np.exp(L + occ - 2.0 * nn + shift)) / den
        gp = np.exp(L - occ)
        if c > 0:  # n'^c = 0 at n' = 0
            gm = np.where(zero, 0.0, gm)
            gp = np.where(zero, 0.0, gp)
        out[0, :, :, c] = gm
        out[1, :, :, c] = gp
    return out


# ----------------------------------------------------------------------------
# Sub-ensemble statistics
# ----------------------------------------------------------------------------
def estimate(samples: np.ndarray, e0: int, n_sub: int) -> Tuple[np.ndarray, np.ndarray]:
    """(mean, sigma) over axis 1 (trajectories e0 + q, sub-ensemble
    (e0 + q) mod n_sub) of the real part of ``samples`` [2][E][...]."""
    E = samples.shape[1]
    sub = (e0 + np.arange(E)) % n_sub
    means = []
    for rr in range(n_sub):
        sel = sub == rr
        if not sel.any():
            raise ValueError("empty sub-ensemble")
        means.append(samples[:, sel].mean(axis=1).real)
    means = np.stack(means, axis=1)        # [2][n_sub][...]
    mean = means.mean(axis=1)
    sig = means.std(axis=1, ddof=1) / math.sqrt(n_sub) if n_sub > 1 else np.zeros_like(mean)
    return mean, sig


def run(T: np.ndarray, r: np.ndarray, seed: int, e0: int, E: int, n_sub: int, mmax: int,
        cmax: int):
    """(mom[2][M][mmax], sig_mom, marg[2][M][cmax+1], sig_marg); index 0 is
    matrix-P, 1 is +P; moments for m = 1..mmax, marginals for c = 0..cmax."""
    n, occ = mode_samples(T, r, seed, e0, E)
    mom, smom = estimate(moment_samples(n, occ, mmax), e0, n_sub)
    marg, smarg = estimate(marginal_samples(n, occ, cmax), e0, n_sub)
    return mom, smom, marg, smarg


# ----------------------------------------------------------------------------
# Exact references (Gaussian state, E1)
# ----------------------------------------------------------------------------
def mode_covariances(T: np.ndarray, r: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(nbar[M], mbar[M]): the diagonal blocks' diagonals of the
    normally-ordered covariance C of E1."""
    M = T.shape[0]
    C = ex.covariance_normal_ordered(T, r)
    return np.real(np.diag(C)[:M]).copy(), np.diag(C[:M, M:]).copy()


def _pairings(items: List[int]):
    if not items:
        yield []
        return
    first = items[0]
    for q in range(1, len(items)):
        rest = items[1:q] + items[q + 1:]
        for p in _pairings(rest):
            yield [(first, items[q])] + p


def isserlis_moment(nbar: float, mbar: complex, m: int) -> complex:
    """<(a^dag)^m a^m> of a zero-mean Gaussian state by brute force over all
    (2m - 1)!! pairings of m conjugate (label 1) and m plain (label 0)
    amplitudes: <a^dag a> = nbar, <a a> = mbar, <a^dag a^dag> = conj(mbar)."""
    labels = [1] * m + [0] * m
    total = 0.0 + 0.0j
    for p in _pairings(list(range(2 * m))):
        v = 1.0 + 0.0j
        for i, j in p:
            li, lj = labels[i], labels[j]
            if li != lj:
                v *= nbar
            elif li == 0:
                v *= mbar
            else:
                v *= np.conj(mbar)
        total += v
    return total


def exact_moments(T: np.ndarray, r: np.ndarray, mmax: int) -> np.ndarray:
    """[M][mmax]: <:n_j^m:>, m = 1..mmax."""
    nbar, mbar = mode_covariances(T, r)
    out = np.zeros((T.shape[0], mmax))
    for j in range(T.shape[0]):
        for m in range(1, mmax + 1):
            out[j, m - 1] = isserlis_moment(nbar[j], mbar[j], m).real
    return out


def exact_marginals(T: np.ndarray, r: np.ndarray, cmax: int) -> np.ndarray:
    """[M][cmax+1]: P_j(c) from the single-mode form of E1.  The 2 x 2 block
    [[nbar, mbar], [conj mbar, nbar]] of C has eigenvalues mu = nbar +- |mbar|,
    so G(z) = prod_mu (1 + (1 - z) mu)^{-1/2}
            = prod_mu (1 + mu)^{-1/2} (1 - q_mu z)^{-1/2},  q_mu = mu / (1 + mu),
    and (1 - q z)^{-1/2} = sum_c binom(2c, c) (q / 4)^c z^c: P_j is the
    convolution of the two binomial series (no DFT, so no aliasing or
    rounding floor in the tails)."""
    nbar, mbar = mode_covariances(T, r)
    out = np.zeros((T.shape[0], cmax + 1))
    c = np.arange(cmax + 1)
    # log binom(2c, c) - c log 4
    lb = gammaln(2 * c + 1.0) - 2.0 * gammaln(c + 1.0) - c * math.log(4.0)
    for j in range(T.shape[0]):
        series = []
        for mu in (nbar[j] + abs(mbar[j]), nbar[j] - abs(mbar[j])):
            q = mu / (1.0 + mu)
            with np.errstate(divide="ignore"):
                mag = np.exp(lb + c * np.log(abs(q))) if q != 0.0 else (c == 0).astype(float)
            sgn = np.where((q < 0) & (c % 2 == 1), -1.0, 1.0)
            series.append(sgn * mag / math.sqrt(1.0 + mu))
        out[j] = np.convolve(series[0], series[1])[:cmax + 1]
    return out
