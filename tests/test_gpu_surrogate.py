"""The surrogate's GPU kernels against the FP64 oracle (oracle/surrogate.py).

MLP: the GPU multiplies BF16 weights (the nearest-even rounding of the FP32
master copy) by activations carried as two BF16 planes (hi + lo: the
activation to ~2^-17 relative), accumulating in FP32 on the tensor cores.
The oracle runs the same network in FP64 with the same BF16 weight values
and FP32 biases, so the two differ only by the activation split, FP32
accumulation and FP32 silu: ~1e-5 relative per layer.  Tolerances: outputs
within 1e-4 of their largest magnitude, gradients within 5e-4 (norm of the
difference over the norm) and 2e-3 of the largest entry per tensor.

Representation kernels (features, statistics, encode, decode) run in FP64
like the oracle: 1e-12 relative, except the FP32 outputs of encode (2^-22
of the output scale).
"""
import math

import numpy as np
import pytest

import oracle.exact as ex
import oracle.surrogate as sur
import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gbs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_12749_gb300 as g
    g.build()
    return g


def _init_params(seed, dims, out_scale=0.3):
    rng = np.random.default_rng(seed)
    params = []
    for i in range(len(dims) - 1):
        W = rng.normal(size=(dims[i + 1], dims[i])) * math.sqrt(2.0 / dims[i])
        if i == len(dims) - 2:
            W *= out_scale
        b = 0.1 * rng.normal(size=dims[i + 1])
        params.append((W.astype(np.float32), b.astype(np.float32)))
    return params


def _pack(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def _unpack(vec, dims):
    out, o = [], 0
    for i in range(len(dims) - 1):
        n, k = dims[i + 1], dims[i]
        W = vec[o:o + n * k].reshape(n, k)
        o += n * k
        b = vec[o:o + n]
        o += n
        out.append((W, b))
    return out


def _oracle_params(params):
    """What the GPU multiplies: BF16 weights, FP32 biases, as float64."""
    return [(sur.bf16_round(W), np.asarray(b, dtype=np.float64)) for W, b in params]


@pytest.mark.parametrize("in_dim,width,out_dim,layers,batch", [
    (10, 512, 512, 4, 300),   # the surrogate's shape, ragged batch (3 tiles)
    (3, 256, 256, 2, 128),    # one tile, two layers
    (32, 256, 512, 3, 1),     # a single row
])
def test_mlp_forward_matches_oracle(gbs, in_dim, width, out_dim, layers, batch):
    import torch
    dims = [in_dim] + [width] * (layers - 1) + [out_dim]
    params = _init_params(100 + layers, dims)
    mlp = gbs.gbs_mlp_create(in_dim, width, out_dim, layers, max(batch, 256))
    gbs.gbs_mlp_set_params(mlp, _pack(params))
    assert np.array_equal(gbs.gbs_mlp_get_params(mlp), _pack(params))
    X = np.random.default_rng(7).normal(size=(batch, in_dim)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.zeros(batch, out_dim, dtype=torch.float32, device="cuda")
    gbs.gbs_mlp_forward(mlp, Xd.data_ptr(), batch, Yd.data_ptr())
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().astype(np.float64)
    Yo, _ = sur.forward(_oracle_params(params), X.astype(np.float64))
    err = np.max(np.abs(Y - Yo)) / np.max(np.abs(Yo))
    assert err < 1e-4, err
    gbs.gbs_mlp_free(mlp)


@pytest.mark.parametrize("width,out_dim,layers,batch", [(512, 512, 4, 260), (256, 256, 3, 97)])
def test_mlp_gradients_match_oracle(gbs, width, out_dim, layers, batch):
    import torch
    in_dim = 10
    dims = [in_dim] + [width] * (layers - 1) + [out_dim]
    params = _init_params(200 + batch, dims)
    mlp = gbs.gbs_mlp_create(in_dim, width, out_dim, layers, 512)
    gbs.gbs_mlp_set_params(mlp, _pack(params))
    rng = np.random.default_rng(8)
    X = rng.normal(size=(batch, in_dim)).astype(np.float32)
    T = rng.normal(size=(batch, out_dim)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    loss, grad = gbs.gbs_mlp_gradients(mlp, Xd.data_ptr(), Td.data_ptr(), batch)
    po = _oracle_params(params)
    Yo, cache = sur.forward(po, X.astype(np.float64))
    lo = sur.loss(Yo, T.astype(np.float64))
    go = sur.backward(po, cache, Yo, T.astype(np.float64))
    assert abs(loss - lo) < 1e-5 * lo
    gg = _unpack(grad.astype(np.float64), dims)
    for l in range(layers):
        for w in (0, 1):
            a, b = gg[l][w], go[l][w]
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            mx = np.max(np.abs(a - b)) / np.max(np.abs(b))
            assert rel < 5e-4 and mx < 2e-3, (l, w, rel, mx)
    # planted check of the tolerance: a transposed weight gradient fails it
    W_t = go[1][0].T if go[1][0].shape[0] == go[1][0].shape[1] else None
    if W_t is not None:
        assert np.linalg.norm(gg[1][0] - W_t) / np.linalg.norm(W_t) > 5e-4
    gbs.gbs_mlp_free(mlp)


def test_adam_step_matches_oracle(gbs):
    import torch
    dims = [10, 256, 256, 256, 256]
    params = _init_params(3, dims)
    mlp = gbs.gbs_mlp_create(10, 256, 256, 4, 256)
    gbs.gbs_mlp_set_params(mlp, _pack(params))
    rng = np.random.default_rng(9)
    X = torch.from_numpy(rng.normal(size=(200, 10)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=(200, 256)).astype(np.float32)).cuda()
    _, g = gbs.gbs_mlp_gradients(mlp, X.data_ptr(), T.data_ptr(), 200)
    lr = 2e-3
    gbs.gbs_mlp_train(mlp, X.data_ptr(), T.data_ptr(), 200, [lr])
    m1, m2, step = gbs.gbs_mlp_get_adam_state(mlp)
    assert step == 1
    new = gbs.gbs_mlp_get_params(mlp).astype(np.float64)
    # the oracle's Adam from the same gradient (the GPU's own, so that only the
    # update arithmetic is compared)
    P = [(W.astype(np.float64), b.astype(np.float64)) for W, b in params]
    G = _unpack(g.astype(np.float64), dims)
    Z = [(np.zeros_like(W), np.zeros_like(b)) for W, b in P]
    Po, Mo, Vo = sur.adam_step(P, G, Z, Z, 1, lr)
    assert np.allclose(m1, _pack(Mo), rtol=1e-6, atol=1e-12)
    assert np.allclose(m2, _pack(Vo), rtol=1e-5, atol=1e-20)
    assert np.max(np.abs(new - _pack(Po))) < 1e-6 + 1e-3 * lr
    gbs.gbs_mlp_free(mlp)


def test_training_lowers_the_loss_and_is_deterministic(gbs):
    import torch
    dims = [10, 256, 256, 256, 256]
    rng = np.random.default_rng(10)
    X = torch.from_numpy(rng.normal(size=(384, 10)).astype(np.float32)).cuda()
    W = rng.normal(size=(10, 256))
    T = torch.from_numpy(np.tanh(X.cpu().numpy() @ W * 0.2).astype(np.float32)).cuda()
    out = []
    for _ in range(2):
        mlp = gbs.gbs_mlp_create(10, 256, 256, 4, 384)
        gbs.gbs_mlp_set_params(mlp, _pack(_init_params(4, dims)))
        hist = gbs.gbs_mlp_train(mlp, X.data_ptr(), T.data_ptr(), 384, np.full(300, 1e-3))
        out.append((hist, gbs.gbs_mlp_get_params(mlp)))
        gbs.gbs_mlp_free(mlp)
    hist = out[0][0]
    assert hist[-1] < 0.05 * hist[0], (hist[0], hist[-1])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][0], out[1][0])


def _records(gbs, nets):
    import torch
    feat = torch.zeros(len(nets), gbs.GBS_SUR_RECORD, dtype=torch.float64, device="cuda")
    gbs.gbs_surrogate_features([n.N for n in nets], [n.M for n in nets], [n.t for n in nets],
                               [n.K1 for n in nets], [n.m_off for n in nets],
                               [n.r for n in nets], feat.data_ptr())
    return feat


def test_features_match_oracle(gbs):
    nets = wl.surrogate_networks(6, seed=777) + wl.surrogate_networks(1, seed=778, n_lo=3, n_hi=3)
    feat = _records(gbs, nets).cpu().numpy()
    for i, n in enumerate(nets):
        u = sur.features(n.N, n.M, n.r, n.t, n.K1)
        mu, s = sur.count_moments(n.r, n.t)
        assert np.allclose(feat[i, :10], u, rtol=1e-12, atol=1e-13), (i, feat[i, :10], u)
        assert abs(feat[i, 10] - mu) < 1e-12 * mu and abs(feat[i, 11] - s) < 1e-12 * s
        assert feat[i, 12] == n.m_off and feat[i, 13] == n.K1


def test_feature_stats_and_standardize(gbs):
    import torch
    nets = wl.surrogate_networks(40, seed=779, n_lo=100, n_hi=300)
    feat = _records(gbs, nets)
    stats = torch.zeros(4, 10, dtype=torch.float64, device="cuda")
    gbs.gbs_surrogate_feature_stats(len(nets), feat.data_ptr(), stats.data_ptr())
    U = feat.cpu().numpy()[:, :10]
    st = stats.cpu().numpy()
    assert np.allclose(st[0], U.mean(0), rtol=1e-12, atol=1e-14)
    assert np.allclose(st[1], U.std(0), rtol=1e-10, atol=1e-14)
    assert np.array_equal(st[2], U.min(0)) and np.array_equal(st[3], U.max(0))
    # queries: the training networks (in domain) and a much larger one (not)
    q = nets[:3] + wl.surrogate_networks(1, seed=780, n_lo=5000, n_hi=5000)
    fq = _records(gbs, q)
    X = torch.zeros(len(q), 10, dtype=torch.float32, device="cuda")
    dom = torch.zeros(len(q), dtype=torch.int32, device="cuda")
    gbs.gbs_surrogate_standardize(len(q), fq.data_ptr(), stats.data_ptr(), X.data_ptr(),
                                  dom.data_ptr())
    Uq = fq.cpu().numpy()[:, :10]
    sd = np.where(st[1] > 1e-12, st[1], np.inf)
    expect = ((Uq - st[0]) / sd).astype(np.float32)
    assert np.allclose(X.cpu().numpy(), expect, rtol=1e-6, atol=1e-6)
    assert dom.cpu().numpy().tolist() == [1, 1, 1, 0]


def test_encode_decode_match_oracle(gbs):
    import torch
    rng = np.random.default_rng(12)
    cases = []
    for N, lo, hi, t in [(300, 0.5, 0.9, 0.95), (120, 1.0, 1.4, 0.999), (60, 0.2, 0.4, 0.9)]:
        r = rng.uniform(lo, hi, size=N)
        mu, s = sur.count_moments(r, t)
        K1 = 1 << int(math.ceil(math.log2(mu + 14 * s)))
        m_off = max(0, int(mu - 10 * s)) // 2 * 2 + (1 if N == 60 else 0)
        P = ex.exact_distribution(ex.eigenvalues_uniform_loss(r, t * t), K1, m_off).real
        cases.append((wl.SurrogateNet(N, r, t, K1, m_off, 0, 0), P))
    nets = [c[0] for c in cases]
    ld = max(n.K1 for n in nets)
    Pd = torch.zeros(len(nets), ld, dtype=torch.float64, device="cuda")
    for i, (_, P) in enumerate(cases):
        Pd[i, :P.size] = torch.from_numpy(P)
    feat = _records(gbs, nets)
    Y = torch.zeros(len(nets), 512, dtype=torch.float32, device="cuda")
    gbs.gbs_surrogate_encode(len(nets), feat.data_ptr(), Pd.data_ptr(), ld, Y.data_ptr())
    # decode an output that is not a round trip: the oracle's encoding + noise
    noise = rng.normal(size=(len(nets), 512)).astype(np.float32) * 0.05
    Yn = torch.from_numpy(noise).cuda() + Y
    Pout = torch.zeros_like(Pd)
    gbs.gbs_surrogate_decode(len(nets), feat.data_ptr(), Yn.data_ptr(), Pout.data_ptr(), ld)
    torch.cuda.synchronize()
    Yh = Y.cpu().numpy()
    Yn_h = Yn.cpu().numpy().astype(np.float64)
    for i, (n, P) in enumerate(cases):
        mu, s = sur.count_moments(n.r, n.t)
        o = sur.encode(P, n.m_off, mu, s)
        assert np.max(np.abs(Yh[i] - o)) < 2.0 ** -22 * sur.OUT_SCALE, i
        back = sur.decode(Yn_h[i], n.m_off, n.K1, mu, s)
        got = Pout[i, :n.K1].cpu().numpy()
        assert np.max(np.abs(got - back)) < 1e-12 * back.max(), i
        assert abs(got.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_network_from_device_memory_equals_host_upload(gbs, prec):
    import torch
    net_def = wl.small_network(150, M=130, r=0.9, t2=0.95, seed=41)
    s = torch.cuda.current_stream().cuda_stream
    a = gbs.gbs_make_network(net_def.T, net_def.r, prec, s)
    Td = torch.from_numpy(net_def.T).cuda()
    b = gbs.gbs_make_network_device(Td.data_ptr(), 130, 150, net_def.r, prec, s)
    na, sa = gbs.gbs_debug_samples(a, net_def.seed_s, 5, 700)
    nb, sb = gbs.gbs_debug_samples(b, net_def.seed_s, 5, 700)
    assert np.array_equal(na, nb) and np.array_equal(sa, sb)
    bad = Td.clone()
    bad[3, 4] = float("nan")
    with pytest.raises(gbs.GbsError):
        gbs.gbs_make_network_device(bad.data_ptr(), 130, 150, net_def.r, prec, s)
