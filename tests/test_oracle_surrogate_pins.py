"""Pins of the surrogate oracle (oracle/surrogate.py) to facts fixed outside it:
the moments of the exact determinant distribution, closed forms of the
Catmull-Rom cubic, of the normal density and of Adam's first steps, BF16
ties-to-even values, and central finite differences of the oracle's own loss
for its backward pass."""
import math

import numpy as np
import pytest

import oracle.exact as ex
import oracle.surrogate as sur


def _net(N, lo, hi, t, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=N), t


@pytest.mark.parametrize("N,lo,hi,t,seed", [(12, 0.3, 1.2, 0.9, 1), (40, 0.8, 1.0, 1.0, 2),
                                            (25, 0.1, 1.5, 0.7, 3)])
def test_count_moments_equal_those_of_the_exact_distribution(N, lo, hi, t, seed):
    r, t = _net(N, lo, hi, t, seed)
    mu_k = ex.eigenvalues_uniform_loss(r, t * t)
    mean0, sd0 = sur.count_moments(r, t)
    P = ex.exact_unaliased(mu_k, int(mean0 + 60 * sd0) + 64)
    m = np.arange(P.size)
    mean = float(np.sum(m * P))
    var = float(np.sum((m - mean) ** 2 * P))
    assert abs(P.sum() - 1.0) < 1e-10
    assert abs(mean - mean0) < 1e-9 * mean0
    assert abs(math.sqrt(var) - sd0) < 1e-8 * sd0


def test_features_layout():
    r = np.array([0.5, 1.0, 1.5, 0.7])
    u = sur.features(4, 5, r, 0.9, 1024)
    mu, s = sur.count_moments(r, 0.9)
    expect = [math.log(4), math.log(5), r.mean(), r.std(), 0.5, 1.5, 0.9, 10.0, math.log(mu),
              math.log(s)]
    assert np.allclose(u, expect, rtol=0, atol=1e-15)


def test_catmull_rom_interpolates_nodes_and_reproduces_quadratics():
    rng = np.random.default_rng(5)
    a, b, c = rng.normal(size=3)
    q = lambda x: a * x * x + b * x + c
    u = np.linspace(0.0, 1.0, 17)
    got = sur.catmull_rom(q(-1.0), q(0.0), q(1.0), q(2.0), u)
    assert np.allclose(got, q(u), rtol=0, atol=1e-14)
    assert sur.catmull_rom(3.0, -1.0, 2.0, 7.0, 0.0) == -1.0
    assert abs(sur.catmull_rom(3.0, -1.0, 2.0, 7.0, 1.0) - 2.0) < 1e-15
    # x^3 is not reproduced: with central-difference slopes 1 and 4 the
    # Hermite cubic through (0, 0), (1, 1) is u - 3 u^2 + 3 u^3
    got = sur.catmull_rom(-1.0, 0.0, 1.0, 8.0, u)
    assert np.allclose(got, u - 3 * u ** 2 + 3 * u ** 3, rtol=0, atol=1e-14)


def test_grid_and_half_normal():
    x = sur.grid()
    assert x.size == 256 and x[0] == -8.0 + 1.0 / 32 and x[1] - x[0] == 1.0 / 16 and x[-1] == 8.0 - 1.0 / 32
    assert abs(sur.half_normal_density(0.0) - 0.5 / math.sqrt(2 * math.pi)) < 1e-16
    # integral of phi/2 over the grid range: erf(8 / sqrt 2) / 2
    xs = np.linspace(-8, 8, 200001)
    integral = np.trapezoid(sur.half_normal_density(xs), xs)
    assert abs(integral - 0.5 * math.erf(8 / math.sqrt(2))) < 1e-9


def test_encode_of_a_discretised_normal_is_zero():
    # P(m) = phi((m - mu)/s) / s on both parities: each parity channel has the
    # density (s/2) P = phi/2, the baseline, so every output is ~0
    mu, s = 5000.3, 61.7
    m_off, K1 = 4000, 2048
    m = m_off + np.arange(K1)
    P = np.exp(-0.5 * ((m - mu) / s) ** 2) / (math.sqrt(2 * math.pi) * s)
    o = sur.encode(P, m_off, mu, s)
    assert np.max(np.abs(o)) < 2e-3 * sur.OUT_SCALE * 0.2
    # and a wrong factor 2 in the density would give outputs ~ OUT_SCALE * phi / 2
    assert sur.OUT_SCALE * sur.half_normal_density(0.0) > 10.0


def test_decode_of_zero_output_is_the_discretised_normal():
    mu, s = 777.7, 33.3
    m_off, K1 = 512, 1024
    P = sur.decode(np.zeros(512), m_off, K1, mu, s)
    m = m_off + np.arange(K1)
    ref = np.exp(-0.5 * ((m - mu) / s) ** 2)
    ref /= ref.sum()
    assert abs(P.sum() - 1.0) < 1e-12
    assert np.max(np.abs(P - ref)) < 2e-5 * ref.max()


@pytest.mark.parametrize("N,lo,hi,t", [(300, 0.5, 0.9, 0.95), (120, 1.0, 1.4, 0.999)])
def test_decode_inverts_encode_on_exact_distributions(N, lo, hi, t):
    r, t = _net(N, lo, hi, t, 7)
    mu, s = sur.count_moments(r, t)
    K1 = 1 << int(math.ceil(math.log2(mu + 14 * s)))
    mu_k = ex.eigenvalues_uniform_loss(r, t * t)
    P = ex.exact_distribution(mu_k, K1).real
    o = sur.encode(P, 0, mu, s)
    back = sur.decode(o, 0, K1, mu, s)
    assert abs(back.sum() - 1.0) < 1e-12
    assert np.max(np.abs(back - P)) < 1e-4 * P.max()


def test_lossless_distribution_has_an_empty_odd_channel():
    r = np.full(50, 0.8)
    mu, s = sur.count_moments(r, 1.0)
    K1 = 512
    P = ex.negative_binomial(50, 0.8, K1)
    o = sur.encode(P, 0, mu, s).reshape(2, 256)
    odd_baseline = -sur.OUT_SCALE * sur.half_normal_density(sur.grid())
    assert np.max(np.abs(o[1] - odd_baseline)) < 1e-12
    back = sur.decode(o.reshape(-1), 0, K1, mu, s)
    assert np.max(back[1::2]) < 1e-14 * P.max()   # rounding of o/100 + phi/2 only
    assert np.max(np.abs(back - P)) < 2e-4 * P.max()


def test_bf16_round_ties_to_even():
    one = 1.0
    assert sur.bf16_round(one + 2.0 ** -8) == 1.0                     # tie -> even (mantissa 0)
    assert sur.bf16_round(one + 3 * 2.0 ** -8) == one + 2.0 ** -6       # tie -> even (mantissa 2)
    assert sur.bf16_round(one + 2.0 ** -8 + 2.0 ** -20) == one + 2.0 ** -7
    assert sur.bf16_round(-(one + 2.0 ** -8 + 2.0 ** -20)) == -(one + 2.0 ** -7)
    assert sur.bf16_round(3.0) == 3.0
    assert sur.bf16_round(0.0) == 0.0


def test_silu_closed_forms():
    assert sur.silu(0.0) == 0.0
    assert abs(sur.silu(math.log(3.0)) - 0.75 * math.log(3.0)) < 1e-15
    # silu'(0) = 1/2, silu'(ln 3) = 3/4 (1 + ln3 / 4)
    assert abs(sur.silu_grad(0.0) - 0.5) < 1e-16
    assert abs(sur.silu_grad(math.log(3.0)) - 0.75 * (1 + math.log(3.0) / 4)) < 1e-15


def _tiny_params(seed, dims):
    rng = np.random.default_rng(seed)
    return [(rng.normal(size=(dims[i + 1], dims[i])) / math.sqrt(dims[i]),
             0.1 * rng.normal(size=dims[i + 1])) for i in range(len(dims) - 1)]


def test_backward_matches_central_differences():
    dims = [3, 7, 6, 5, 4]
    params = _tiny_params(11, dims)
    rng = np.random.default_rng(12)
    X = rng.normal(size=(5, 3))
    T = rng.normal(size=(5, 4))
    Y, cache = sur.forward(params, X)
    grads = sur.backward(params, cache, Y, T)
    h = 1e-6
    for l in range(len(params)):
        for which in (0, 1):
            arr = params[l][which]
            g = grads[l][which]
            it = np.nditer(arr, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = arr[idx]
                arr[idx] = old + h
                lp = sur.loss(sur.forward(params, X)[0], T)
                arr[idx] = old - h
                lm = sur.loss(sur.forward(params, X)[0], T)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) < 1e-7 * max(1.0, abs(fd)), (l, which, idx, fd, g[idx])


def test_adam_first_steps_closed_form():
    # constant gradient g: m_hat = g and v_hat = g^2 at every step, so each
    # step moves by -lr g / (|g| + eps)
    p = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    g = [(np.array([[0.3, -4.0]]), np.array([1e-3]))]
    m = [(np.zeros((1, 2)), np.zeros(1))]
    v = [(np.zeros((1, 2)), np.zeros(1))]
    lr, eps = 0.01, 1e-8
    cur = p
    for step in (1, 2, 3):
        cur, m, v = sur.adam_step(cur, g, m, v, step, lr)
        for (W0, b0), (W1, b1), (gW, gb) in zip(p, cur, g):
            expW = W0 - step * lr * gW / (np.abs(gW) + eps)
            expb = b0 - step * lr * gb / (np.abs(gb) + eps)
            assert np.allclose(W1, expW, rtol=0, atol=1e-12)
            assert np.allclose(b1, expb, rtol=0, atol=1e-12)
    # first moments after 3 steps: (1 - 0.9^3) g
    assert np.allclose(m[0][0], (1 - 0.9 ** 3) * g[0][0], rtol=1e-14)
    assert np.allclose(v[0][0], (1 - 0.999 ** 3) * g[0][0] ** 2, rtol=1e-12)


def test_loss_is_mean_squared_error():
    Y = np.array([[1.0, 2.0], [3.0, 5.0]])
    T = np.array([[0.0, 2.0], [3.0, 1.0]])
    assert sur.loss(Y, T) == (1.0 + 16.0) / 4.0
