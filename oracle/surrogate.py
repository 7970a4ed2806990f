"""Oracle of the learned surrogate of the binned total-count distribution.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): plain FP64 numpy,
imported by tests, ``__graft_entry__.smoke()`` and the CPU legs of bench.py,
never by the library.

The surrogate is not part of the paper.  It approximates the quantity the
paper's method estimates -- the binned total-count distribution P(m) of a
Gaussian boson sampler ("Applications to GBS", the multi-mode exact result
and the binned generating function) -- for networks T = t U with squeezed
inputs r_j, and the matrix-P run stays its judge.  The definitions below are
this project's own and the GPU path implements the same ones:

Features (10).  u = [ln N, ln M, mean r, std r (population), min r, max r,
    t, log2 K1, ln mu, ln s], with mu and s the closed-form mean and standard
    deviation of the total count.  From the uniform-loss eigenvalues
    mu_k = {t^2 sinh r_j e^{r_j}, -t^2 sinh r_j e^{-r_j}} of the determinant
    generating function G(z) = prod_k (1 + (1 - z) mu_k)^{-1/2}:
        mean     = (1/2) sum_k mu_k            = t^2 sum_j sinh^2 r_j,
        variance = (1/2) sum_k (mu_k + mu_k^2)
                 = sum_j [t^2 sinh^2 r_j + t^4 sinh^2 r_j cosh 2 r_j].
    The network sees (u - mean_train) / std_train.

Output (512).  Two channels of 256 values: even counts (p = 0) and odd
    counts (p = 1), on the standardised grid x_i = -8 + 16 (i + 1/2) / 256.
    Channel p holds the density of the counts of parity p per unit x,
    f_p(x) = (s / 2) P(m)|_{m = mu + s x, m of parity p}, as the residual
    o_{p,i} = 100 (f_p(x_i) - phi(x_i) / 2) from half a standard normal
    density phi (each parity class carries about half the mass).

Encoding a distribution (targets).  P on the lattice of parity p (spacing 2)
    is interpolated at m* = mu + s x_i by the Catmull-Rom cubic (E. Catmull,
    R. Rom, "A class of local interpolating splines", 1974); counts outside
    the window [m_off, m_off + K1) read as 0.

Decoding an output.  For each m of the window: x = (m - mu) / s,
    f = Catmull-Rom interpolation of channel (m mod 2) on the x grid (0 off the
    grid, clamped at 0), P(m) = 2 f / s, then P is renormalised to sum 1.

MLP.  Layers l = 1..L: y_l = W_l h_{l-1} + b_l, h_l = silu(y_l) for l < L,
    output y_L; silu(y) = y / (1 + e^{-y}) (Elfwing, Uchibe, Doya 2018).  Loss
    L = (1 / (B O)) sum_{b,o} (y_L - target)^2.  Gradients by the chain rule;
    Adam (Kingma & Ba, ICLR 2015, Algorithm 1) with bias correction.  On the
    GPU the weights used by the products are the BF16 rounding (nearest-even)
    of FP32 master weights; ``bf16_round`` gives the same values here.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

GRID = 256
X_LO = -8.0
X_HI = 8.0
OUT_SCALE = 100.0
N_FEATURES = 10
OUT_DIM = 2 * GRID


def grid() -> np.ndarray:
    """x_i = X_LO + (X_HI - X_LO) (i + 1/2) / GRID."""
    return X_LO + (X_HI - X_LO) * (np.arange(GRID) + 0.5) / GRID


def half_normal_density(x: np.ndarray) -> np.ndarray:
    """phi(x) / 2."""
    return 0.5 * np.exp(-0.5 * np.asarray(x, dtype=np.float64) ** 2) / math.sqrt(2.0 * math.pi)


# ----------------------------------------------------------------------------
# closed-form moments and features
# ----------------------------------------------------------------------------
def count_moments(r: Sequence[float], t: float) -> Tuple[float, float]:
    """(mean, standard deviation) of the total count for T = t U (see header)."""
    r = np.asarray(r, dtype=np.float64)
    eta = t * t
    s2 = np.sinh(r) ** 2
    mean = eta * float(np.sum(s2))
    var = float(np.sum(eta * s2 + eta * eta * s2 * np.cosh(2.0 * r)))
    return mean, math.sqrt(var)


def features(N: int, M: int, r: Sequence[float], t: float, K1: int) -> np.ndarray:
    """The 10 raw features u of one network (see header)."""
    r = np.asarray(r, dtype=np.float64)
    mu, s = count_moments(r, t)
    return np.array([math.log(N), math.log(M), float(r.mean()), float(r.std()), float(r.min()),
                     float(r.max()), float(t), math.log2(K1), math.log(mu), math.log(s)])


# ----------------------------------------------------------------------------
# Catmull-Rom interpolation, encoding and decoding
# ----------------------------------------------------------------------------
def catmull_rom(ym1, y0, y1, y2, u):
    """Cubic through (0, y0), (1, y1) with slopes (y1 - ym1) / 2 and
    (y2 - y0) / 2, evaluated at u in [0, 1)."""
    u = np.asarray(u, dtype=np.float64)
    h00 = 2 * u ** 3 - 3 * u ** 2 + 1
    h10 = u ** 3 - 2 * u ** 2 + u
    h01 = -2 * u ** 3 + 3 * u ** 2
    h11 = u ** 3 - u ** 2
    return h00 * y0 + h10 * 0.5 * (y1 - ym1) + h01 * y1 + h11 * 0.5 * (y2 - y0)


def encode(P: np.ndarray, m_off: int, mu: float, s: float) -> np.ndarray:
    """Targets o (512) of a distribution P on the window [m_off, m_off + len(P))."""
    P = np.asarray(P, dtype=np.float64)
    K1 = P.shape[0]
    x = grid()
    out = np.zeros((2, GRID))
    for p in range(2):
        for i in range(GRID):
            mstar = mu + s * x[i]
            q = (mstar - p) / 2.0          # position on the parity-p lattice m = p + 2q
            q0 = math.floor(q)
            u = q - q0
            ys = []
            for dq in (-1, 0, 1, 2):
                m = p + 2 * (q0 + dq)
                ys.append(P[m - m_off] if 0 <= m - m_off < K1 else 0.0)
            f = 0.5 * s * catmull_rom(ys[0], ys[1], ys[2], ys[3], u)
            out[p, i] = OUT_SCALE * (f - half_normal_density(x[i]))
    return out.reshape(-1)


def decode(o: np.ndarray, m_off: int, K1: int, mu: float, s: float) -> np.ndarray:
    """P(m) on the window [m_off, m_off + K1) from an output o (512)."""
    o = np.asarray(o, dtype=np.float64).reshape(2, GRID)
    x = grid()
    f = o / OUT_SCALE + half_normal_density(x)[None, :]
    dx = (X_HI - X_LO) / GRID
    P = np.zeros(K1)
    for j in range(K1):
        m = m_off + j
        p = m % 2
        g = ((m - mu) / s - x[0]) / dx     # position on the grid
        if g < 0.0 or g > GRID - 1:
            continue
        g0 = math.floor(g)
        u = g - g0
        ys = [f[p, i] if 0 <= i < GRID else 0.0 for i in (g0 - 1, g0, g0 + 1, g0 + 2)]
        P[j] = 2.0 / s * max(float(catmull_rom(ys[0], ys[1], ys[2], ys[3], u)), 0.0)
    total = P.sum()
    return P / total if total > 0 else P


# ----------------------------------------------------------------------------
# BF16 rounding
# ----------------------------------------------------------------------------
def bf16_round(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even) of the FP32 rounding of x,
    returned as float64 (finite inputs)."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    rounded = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


# ----------------------------------------------------------------------------
# MLP forward, loss, backward, Adam
# ----------------------------------------------------------------------------
Params = List[Tuple[np.ndarray, np.ndarray]]   # [(W_l [out, in], b_l [out])]


def silu(y):
    return y / (1.0 + np.exp(-y))


def silu_grad(y):
    sg = 1.0 / (1.0 + np.exp(-y))
    return sg * (1.0 + y * (1.0 - sg))


def forward(params: Params, X: np.ndarray):
    """Output [B, O] and the cache (inputs of every layer, pre-activations)."""
    h = np.asarray(X, dtype=np.float64)
    hs, ys = [h], []
    for l, (W, b) in enumerate(params):
        y = h @ W.T + b[None, :]
        ys.append(y)
        if l < len(params) - 1:
            h = silu(y)
            hs.append(h)
        else:
            h = y
    return h, (hs, ys)


def loss(Y: np.ndarray, target: np.ndarray) -> float:
    d = Y - target
    return float(np.sum(d * d) / d.size)


def backward(params: Params, cache, Y: np.ndarray, target: np.ndarray) -> Params:
    """(dL/dW_l, dL/db_l) for every layer."""
    hs, ys = cache
    g = 2.0 * (Y - target) / Y.size              # dL/dy_L
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        grads[l] = (g.T @ hs[l], g.sum(axis=0))
        if l > 0:
            g = (g @ W) * silu_grad(ys[l - 1])   # dL/dy_{l-1}
    return grads


def adam_step(params: Params, grads: Params, m: Params, v: Params, step: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step = 1, 2, ...) in place of copies; returns
    (params, m, v)."""
    c1 = 1.0 - beta1 ** step
    c2 = 1.0 - beta2 ** step
    out_p, out_m, out_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        new = []
        for p_, g_, m_, v_ in ((W, gW, mW, vW), (b, gb, mb, vb)):
            m1 = beta1 * m_ + (1.0 - beta1) * g_
            v1 = beta2 * v_ + (1.0 - beta2) * g_ * g_
            p1 = p_ - lr * (m1 / c1) / (np.sqrt(v1 / c2) + eps)
            new.append((p1, m1, v1))
        out_p.append((new[0][0], new[1][0]))
        out_m.append((new[0][1], new[1][1]))
        out_v.append((new[0][2], new[1][2]))
    return out_p, out_m, out_v
