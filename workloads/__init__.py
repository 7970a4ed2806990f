"""Seeded synthetic inputs for the matrix-P total-count estimator.

This module is shared by the CUDA path (tests, bench) and by the CPU oracle.
It generates *inputs only* -- Haar-random networks, squeezing vectors and the
named workload definitions -- and contains none of the estimator's arithmetic
(no sampling of phase-space amplitudes, no propagation, no projectors).

Paper context (arXiv:2503.12749):
  * networks are Haar-random unitaries U_H, optionally with uniform amplitude
    loss t, i.e. T = t * U_H ("Applications to GBS" and Appendix B, Fig. 6);
  * inputs are single-mode squeezed vacua with squeezing r_j >= 0.

Haar sampling follows the published recipe of F. Mezzadri, "How to generate
random matrices from the classical compact groups", Notices AMS 54 (2007):
QR of a complex Ginibre matrix, then multiply column k of Q by
R_kk / |R_kk| so the distribution is exactly Haar.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Seed conventions for network i of a workload.
SEED_U_BASE = 12749            # Haar matrix of network i: SEED_U_BASE + i
SEED_S_BASE = 2503 * 10**6     # Philox key of network i: SEED_S_BASE + i
SEED_R_OFFSET = 10**6          # squeezing draws: default_rng(seed_U + SEED_R_OFFSET)


def haar_unitary(m: int, seed: int) -> np.ndarray:
    """Haar-random m x m complex unitary (Mezzadri 2007), complex128."""
    if m <= 0:
        raise ValueError("m must be positive")
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return q * ph[np.newaxis, :]


@dataclasses.dataclass
class Network:
    """One network instance: transmission matrix T (M x N complex) and squeezing r (N)."""
    T: np.ndarray          # complex128, shape (M, N), C-contiguous
    r: np.ndarray          # float64, shape (N,)
    t2: float              # uniform intensity transmission if T = t*U, else -1
    seed_s: int            # Philox key for this network's samples

    @property
    def N(self) -> int:
        return self.T.shape[1]

    @property
    def M(self) -> int:
        return self.T.shape[0]


@dataclasses.dataclass
class Workload:
    """A named workload: network recipe plus ensemble sizes."""
    name: str
    N: int                 # input modes (== M for every named workload)
    M: int                 # output modes
    r_lo: float            # r_j ~ U[r_lo, r_hi] (r_lo == r_hi: uniform squeezing)
    r_hi: float
    t2: float              # intensity transmission, T = sqrt(t2) * U
    E: int                 # samples
    n_sub: int             # number of sub-ensembles N_R
    K1: int                # number of DFT points K+1 (power of two)
    precision: str         # default precision of the GPU run
    index: int = 0         # network index i (selects the seeds)

    def squeezing(self) -> np.ndarray:
        """The N squeezing parameters r_j of network() (no unitary drawn)."""
        if self.r_lo == self.r_hi:
            r = np.full(self.N, float(self.r_lo))
        else:
            rng = np.random.default_rng(SEED_U_BASE + self.index + SEED_R_OFFSET)
            r = rng.uniform(self.r_lo, self.r_hi, size=self.N)
        return np.ascontiguousarray(r, dtype=np.float64)

    def network(self, device: bool = False) -> Network:
        """T = sqrt(t2) U and r.  device=True draws the same Ginibre matrix
        but takes its QR on the GPU (haar_unitary_device; equal up to
        rounding, much faster for thousands of modes) and returns T on the
        host."""
        if device:
            U = haar_unitary_device(self.M, SEED_U_BASE + self.index).cpu().numpy()
        else:
            U = haar_unitary(self.M, SEED_U_BASE + self.index)
        if self.N != self.M:
            U = U[:, : self.N]
        T = np.ascontiguousarray(math.sqrt(self.t2) * U, dtype=np.complex128)
        return Network(T=T, r=self.squeezing(), t2=self.t2, seed_s=SEED_S_BASE + self.index)


# The named workloads.  Sizes follow the paper's regimes (M up to 8000 modes,
# sub-ensembles of 10^4 trajectories, Appendix A) at the shapes used for the
# GB300 measurements.
SMALL16 = Workload("small16: N=M=16 r=1 t2=0.9 E=2^14 K+1=64", 16, 16, 1.0, 1.0, 0.9,
                   2**14, 16, 64, "fp64")
M1000 = Workload("m1000: N=M=1000 r=1 t2=0.98 E=10^6 K+1=4096 N_R=100", 1000, 1000, 1.0, 1.0,
                 0.98, 10**6, 100, 4096, "bf16x3")
M4000 = Workload("m4000: N=M=4000 r~U[0.8,1.2] t2=0.99 E=2^21 K+1=8192 N_R=128", 4000, 4000,
                 0.8, 1.2, 0.99, 2**21, 128, 8192, "bf16x3")
M8000 = Workload("m8000: N=M=8000 r=1 t2=0.99 E=2^20 K+1=16384 N_R=64", 8000, 8000, 1.0, 1.0,
                 0.99, 2**20, 64, 16384, "bf16x3")

NAMED = {"small16": SMALL16, "m1000": M1000, "m4000": M4000, "m8000": M8000}


def batched_networks(count: int = 64, n_lo: int = 100, n_hi: int = 2000,
                     seed: int = SEED_U_BASE + 777) -> List[Workload]:
    """Uneven batch: N=M log-uniform in [n_lo, n_hi], r_j ~ U[0.5, 1.5],
    amplitude transmission t ~ U[0.5, 0.995] (T = t U), one Workload each."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        t = float(rng.uniform(0.5, 0.995))
        out.append(Workload(f"batch[{i}]: N=M={n}", n, n, 0.5, 1.5, t * t, 2**18, 64, 0,
                            "bf16x3", index=1000 + i))
    return out


def dft_window(N: int, r_max: float, t2: float, r_mean2: float):
    """(K1, m_offset) of a DFT window covering the total-count support of a
    network of N squeezed inputs with squeezing up to r_max and intensity
    transmission t2: centred on the mean count t2 * N * <sinh^2 r> (mean
    photon number sinh^2 r per squeezed mode, as stated with the lossless
    exact distribution), half-width 12 x the largest per-mode standard
    deviation sqrt(2 nbar (nbar + 1)) times sqrt(N), rounded up to a power of
    two.  r_mean2 = <sinh^2 r_j>."""
    nbar = math.sinh(r_max) ** 2
    half = 12.0 * math.sqrt(2.0 * nbar * (nbar + 1.0) * N) + 64.0
    K1 = 1 << int(math.ceil(math.log2(2.0 * half)))
    mean = t2 * N * r_mean2
    m_off = max(0, int(round(mean)) - K1 // 2)
    return K1, m_off


def count_window(r: np.ndarray, t2: float):
    """(K1, m_offset) of a DFT window from the total count's own mean and
    variance under uniform loss T = t U: per squeezed mode the count has mean
    t2 sinh^2 r and variance t2 (1 - t2) sinh^2 r + 2 t2^2 sinh^2 r cosh^2 r
    (the lossless squeezed-vacuum variance 2 sinh^2 r cosh^2 r, thinned by
    the loss), and modes add.  Half-width 12 standard deviations + 64 around
    the mean, rounded up to a power of two: tighter than dft_window's bound
    for lossy networks or spread squeezing."""
    r = np.asarray(r, dtype=np.float64)
    s2 = np.sinh(r) ** 2
    mean = float(t2 * np.sum(s2))
    var = float(np.sum(t2 * (1.0 - t2) * s2 + 2.0 * t2 * t2 * s2 * np.cosh(r) ** 2))
    half = 12.0 * math.sqrt(var) + 64.0
    K1 = 1 << int(math.ceil(math.log2(2.0 * half)))
    m_off = max(0, int(round(mean)) - K1 // 2)
    return K1, m_off


def small_network(N: int, M: Optional[int] = None, r=0.5, t2: float = 1.0, seed: int = 0,
                  general_loss: bool = False) -> Network:
    """A small test network.  r may be a scalar or a length-N sequence.
    general_loss=True applies a non-uniform diagonal loss after U so that
    T^T T* is not a multiple of the identity (general, non-Gram case)."""
    M = N if M is None else M
    U = haar_unitary(max(M, N), SEED_U_BASE + 500 + seed)[:M, :N]
    rr = np.full(N, float(r)) if np.isscalar(r) else np.asarray(r, dtype=np.float64)
    if general_loss:
        rng = np.random.default_rng(SEED_U_BASE + 900 + seed)
        amp = rng.uniform(0.6, 1.0, size=M)
        T = (amp[:, None] * U) * math.sqrt(t2)
        t2_hint = -1.0
    else:
        T = math.sqrt(t2) * U
        t2_hint = t2 if M == N else -1.0
    return Network(T=np.ascontiguousarray(T, dtype=np.complex128),
                   r=np.ascontiguousarray(rr, dtype=np.float64), t2=t2_hint,
                   seed_s=SEED_S_BASE + 500 + seed)


# ----------------------------------------------------------------------------
# Networks of the learned surrogate's training and held-out sets
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class SurrogateNet:
    """One network of the surrogate workload: N = M modes, squeezing r (N),
    amplitude transmission t (T = t U), DFT window (K1, m_off), seeds."""
    N: int
    r: np.ndarray
    t: float
    K1: int
    m_off: int
    seed_u: int
    seed_s: int

    @property
    def M(self) -> int:
        return self.N


SUR_TRAIN_SEED = SEED_U_BASE + 5000
SUR_HELDOUT_SEED = SEED_U_BASE + 6000


def surrogate_networks(count: int, seed: int = SUR_TRAIN_SEED, n_lo: int = 500,
                       n_hi: int = 8000) -> List[SurrogateNet]:
    """N log-uniform in [n_lo, n_hi]; per network c ~ U[0.5, 1.5],
    delta ~ U[0, 0.3], r_j ~ U[c - delta, c + delta]; t ~ U[0.9, 0.999];
    window from dft_window.  Network i uses seeds (seed + i, SEED_S_BASE +
    seed + i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        c = float(rng.uniform(0.5, 1.5))
        d = float(rng.uniform(0.0, 0.3))
        t = float(rng.uniform(0.9, 0.999))
        r = np.random.default_rng(seed + i + SEED_R_OFFSET).uniform(c - d, c + d, size=n)
        K1, m_off = dft_window(n, float(r.max()), t * t, float(np.mean(np.sinh(r) ** 2)))
        out.append(SurrogateNet(n, r, t, K1, m_off, seed + i, SEED_S_BASE + seed + i))
    return out


def fourier_unitary_device(N: int, seed: int, device="cuda"):
    """U = F diag(e^{i phi}) as a torch complex128 (N, N) tensor on `device`:
    F_jk = e^{-2 pi i jk / N} / sqrt(N) (the unitary DFT matrix, built from a
    table of the N roots of unity indexed by jk mod N), phases phi_k ~ U[0, 2pi)
    from numpy's default_rng(seed).  Exactly unitary up to rounding; its
    |U_jk|^2 = 1/N like the average of a Haar matrix."""
    import torch
    ph = np.random.default_rng(seed).uniform(0.0, 2.0 * math.pi, size=N)
    roots = np.exp(-2j * math.pi * np.arange(N) / N) / math.sqrt(N)
    roots_d = torch.from_numpy(roots).to(device)
    phase_d = torch.from_numpy(np.exp(1j * ph)).to(device)
    j = torch.arange(N, device=device, dtype=torch.int64)
    idx = torch.remainder(j[:, None] * j[None, :], N)
    return roots_d[idx] * phase_d[None, :]


def haar_unitary_device(N: int, seed: int, device="cuda"):
    """The Haar matrix of haar_unitary(N, seed) (same Ginibre draw and phase
    fix), its QR computed by torch on `device`; equal to it up to rounding."""
    import torch
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / math.sqrt(2.0)
    q, r = torch.linalg.qr(torch.from_numpy(z).to(device))
    d = torch.diagonal(r)
    return q * (d / d.abs())[None, :]
