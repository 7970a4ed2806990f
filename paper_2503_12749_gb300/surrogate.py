"""The learned surrogate of the binned total-count distribution.

A small MLP (10 features -> 512 outputs, see include/gbs_surrogate.h) maps a
network T = t U with squeezed inputs r_j to its total-count distribution
P(m).  It is trained on distributions that the matrix-P ensemble itself
produced, and the ensemble stays both its fallback (networks outside the
training domain are run by the ensemble) and the judge of its error.  The
surrogate is not part of the paper.

This module is host orchestration only: every arithmetic step runs in the
library's kernels (gbs_make_network_device, gbs_sample,
gbs_binned_counts_device, gbs_surrogate_*, gbs_mlp_*); PyTorch provides
device buffers and streams.
"""
from __future__ import annotations

import math
from typing import Callable, Optional, Sequence

import numpy as np

from . import (GBS_SUR_FEATURES, GBS_SUR_OUT, GBS_SUR_RECORD, gbs_binned_counts_device,
               gbs_free_network, gbs_make_network_device, gbs_mlp_create, gbs_mlp_forward,
               gbs_mlp_free, gbs_mlp_get_params, gbs_mlp_gradients, gbs_mlp_set_params,
               gbs_mlp_train, gbs_sample,
               gbs_surrogate_decode, gbs_surrogate_encode, gbs_surrogate_feature_stats,
               gbs_surrogate_features, gbs_surrogate_standardize)


def method_distributions(nets: Sequence, E: int, n_sub: int, make_T: Callable,
                         precision: str = "bf16x3", stream=None):
    """Run the matrix-P ensemble on every network.

    nets: objects with N, M, r, t, K1, m_off, seed_s (e.g. workloads.SurrogateNet).
    make_T(net): the (M, N) complex128 transmission matrix on the device.
    Returns (P, sigma, ldP): device float64 tensors [count, ldP] holding each
    network's matrix-P P(m) and its sampling error on its window."""
    import torch
    ldP = max(int(n.K1) for n in nets)
    s = stream if stream is not None else torch.cuda.current_stream()
    with torch.cuda.stream(s):
        P = torch.zeros(len(nets), ldP, dtype=torch.float64, device="cuda")
        S = torch.zeros_like(P)
        out = torch.empty(4 * ldP, dtype=torch.float64, device="cuda")
        for i, n in enumerate(nets):
            T = make_T(n)
            net = gbs_make_network_device(T.data_ptr(), n.M, n.N, n.r, precision, s.cuda_stream)
            del T
            gbs_sample(net, n.seed_s, 0, E, n_sub, n.K1)
            gbs_binned_counts_device(net, n.m_off, out.data_ptr())
            K1 = int(n.K1)
            P[i, :K1] = out[:K1]
            S[i, :K1] = out[K1:2 * K1]
            gbs_free_network(net)
    return P, S, ldP


def _loss(mlp, X, Y) -> float:
    """Loss of the MLP on (X, Y) (device tensors), through gbs_mlp_gradients."""
    loss, _ = gbs_mlp_gradients(mlp, X.data_ptr(), Y.data_ptr(), X.shape[0])
    return loss


def init_params(seed: int, width: int = 512, layers: int = 4) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), the last layer scaled by 0.1,
    zero biases; packed in the gbs_mlp_set_params layout."""
    rng = np.random.default_rng(seed)
    dims = [GBS_SUR_FEATURES] + [width] * (layers - 1) + [GBS_SUR_OUT]
    parts = []
    for i in range(layers):
        W = rng.normal(size=(dims[i + 1], dims[i])) * math.sqrt(2.0 / dims[i])
        if i == layers - 1:
            W *= 0.1
        parts += [W.ravel(), np.zeros(dims[i + 1])]
    return np.concatenate(parts).astype(np.float32)


def cosine_schedule(steps: int, lr_max: float, lr_min: float) -> np.ndarray:
    i = np.arange(steps)
    return (lr_min + 0.5 * (lr_max - lr_min) * (1.0 + np.cos(np.pi * i / max(steps, 1)))
            ).astype(np.float32)


class Surrogate:
    """MLP surrogate with its feature statistics (set by fit)."""

    def __init__(self, max_batch: int = 2048, width: int = 512, layers: int = 4, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.width, self.layers, self.max_batch = width, layers, max_batch
        self.mlp = gbs_mlp_create(GBS_SUR_FEATURES, width, GBS_SUR_OUT, layers, max_batch,
                                  self.stream.cuda_stream)
        with torch.cuda.stream(self.stream):
            self.stats = torch.zeros(4, GBS_SUR_FEATURES, dtype=torch.float64, device="cuda")
        self.trained = False

    def close(self):
        if self.mlp is not None:
            gbs_mlp_free(self.mlp)
            self.mlp = None

    def records(self, nets: Sequence):
        """Feature records [count, 14] (device) of the networks."""
        import torch
        with torch.cuda.stream(self.stream):
            feat = torch.zeros(len(nets), GBS_SUR_RECORD, dtype=torch.float64, device="cuda")
        gbs_surrogate_features([n.N for n in nets], [n.M for n in nets], [n.t for n in nets],
                               [n.K1 for n in nets], [n.m_off for n in nets],
                               [n.r for n in nets], feat.data_ptr(), self.stream.cuda_stream)
        return feat

    def _inputs(self, feat, count: int):
        import torch
        with torch.cuda.stream(self.stream):
            X = torch.zeros(count, GBS_SUR_FEATURES, dtype=torch.float32, device="cuda")
            dom = torch.zeros(count, dtype=torch.int32, device="cuda")
        gbs_surrogate_standardize(count, feat.data_ptr(), self.stats.data_ptr(), X.data_ptr(),
                                  dom.data_ptr(), self.stream.cuda_stream)
        return X, dom

    def fit(self, nets: Sequence, P, ldP: int, steps: int = 4000, lr_max: float = 1e-3,
            lr_min: float = 1e-5, seed: int = 0, val_frac: float = 0.1,
            rounds: int = 20) -> dict:
        """Train on the distributions P (device [count, ldP], each network's
        P(m) on its window).

        The ensemble's distributions carry sampling noise, so a network that
        fits them exactly learns the noise.  A fraction val_frac of the
        networks (every k-th) is held back; training runs in `rounds` equal
        parts of one cosine learning-rate schedule, the held-back loss is
        measured after each, and the parameters of the best round are kept
        (early stopping).  The feature statistics come from all networks.
        Returns {"train_loss": per step, "val_loss": per round, "best_round"}."""
        import torch
        count = len(nets)
        if count > self.max_batch:
            raise ValueError("more training networks than max_batch")
        feat = self.records(nets)
        gbs_surrogate_feature_stats(count, feat.data_ptr(), self.stats.data_ptr(),
                                    self.stream.cuda_stream)
        X, _ = self._inputs(feat, count)
        with torch.cuda.stream(self.stream):
            Y = torch.zeros(count, GBS_SUR_OUT, dtype=torch.float32, device="cuda")
        gbs_surrogate_encode(count, feat.data_ptr(), P.data_ptr(), ldP, Y.data_ptr(),
                             self.stream.cuda_stream)
        nval = int(round(val_frac * count)) if count >= 20 else 0
        if nval:
            k = count // nval
            val_idx = np.arange(0, k * nval, k)
            tr_idx = np.setdiff1d(np.arange(count), val_idx)
            with torch.cuda.stream(self.stream):
                vi = torch.from_numpy(val_idx).cuda()
                ti = torch.from_numpy(tr_idx).cuda()
                Xv, Yv = X[vi].contiguous(), Y[vi].contiguous()
                Xt, Yt = X[ti].contiguous(), Y[ti].contiguous()
        else:
            Xt, Yt, Xv, Yv = X, Y, None, None
        ntr = Xt.shape[0]
        self.stream.synchronize()
        gbs_mlp_set_params(self.mlp, init_params(seed, self.width, self.layers))
        lr = cosine_schedule(steps, lr_max, lr_min)
        rounds = max(1, min(rounds, steps))
        edges = np.linspace(0, steps, rounds + 1).astype(int)
        hist, val, best, best_params = [], [], None, None
        for q in range(rounds):
            hist.append(gbs_mlp_train(self.mlp, Xt.data_ptr(), Yt.data_ptr(), ntr,
                                      lr[edges[q]:edges[q + 1]]))
            if Xv is not None:
                vl = _loss(self.mlp, Xv, Yv)
                val.append(vl)
                if best is None or vl < val[best]:
                    best = q
                    best_params = gbs_mlp_get_params(self.mlp)
        if best_params is not None:
            gbs_mlp_set_params(self.mlp, best_params)
        self.trained = True
        return {"train_loss": np.concatenate(hist), "val_loss": np.array(val),
                "best_round": best, "rounds": rounds, "n_train": ntr, "n_val": nval}

    def predict(self, nets: Sequence, ldP: Optional[int] = None):
        """(P [count, ldP] device float64, ldP, in_domain [count] numpy bool)."""
        import torch
        if not self.trained:
            raise RuntimeError("the surrogate is not trained")
        count = len(nets)
        ldP = ldP or max(int(n.K1) for n in nets)
        feat = self.records(nets)
        X, dom = self._inputs(feat, count)
        with torch.cuda.stream(self.stream):
            Y = torch.zeros(count, GBS_SUR_OUT, dtype=torch.float32, device="cuda")
            P = torch.zeros(count, ldP, dtype=torch.float64, device="cuda")
        for a in range(0, count, self.max_batch):
            b = min(count, a + self.max_batch)
            gbs_mlp_forward(self.mlp, X[a:b].data_ptr(), b - a, Y[a:b].data_ptr())
        gbs_surrogate_decode(count, feat.data_ptr(), Y.data_ptr(), P.data_ptr(), ldP,
                             self.stream.cuda_stream)
        self.stream.synchronize()
        return P, ldP, dom.cpu().numpy().astype(bool)

    def predict_or_run(self, nets: Sequence, E: int, n_sub: int, make_T: Callable,
                       precision: str = "bf16x3"):
        """Surrogate predictions where the network lies in the training domain,
        the matrix-P ensemble elsewhere.  Returns (P, ldP, ran_method[count])."""
        P, ldP, dom = self.predict(nets)
        todo = [i for i in range(len(nets)) if not dom[i]]
        if todo:
            Pm, _, ld2 = method_distributions([nets[i] for i in todo], E, n_sub, make_T,
                                              precision, self.stream)
            for j, i in enumerate(todo):
                K1 = int(nets[i].K1)
                P[i, :K1] = Pm[j, :K1]
        self.stream.synchronize()
        return P, ldP, ~dom
