"""GB300-native matrix-P total-count estimator for Gaussian boson sampling.

Python binding of the C ABI in ``include/gbs.h`` and
``include/gbs_surrogate.h`` (libgbs.so, built for
sm_103a by ``paper_2503_12749_gb300.build``).  The functions below carry the
ABI's names and only marshal arguments: every step of the estimator runs in
the library's CUDA kernels.  There is no CPU fallback: if the library cannot
be loaded, the first call raises.

Typical use::

    import paper_2503_12749_gb300 as gbs
    net = gbs.gbs_make_network(T, r, gbs.GBS_BF16X3)
    gbs.gbs_sample(net, seed, 0, E, n_sub, K1)
    P_mP, s_mP, P_pP, s_pP = gbs.gbs_binned_counts(net, m_offset=0)
    gbs.gbs_free_network(net)
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Tuple

import numpy as np

GBS_OK = 0
GBS_EINVAL = -1
GBS_ENOMEM = -2
GBS_ECUDA = -3
GBS_ETIMEOUT = -4
GBS_ENONFINITE = -5
GBS_ENOTSUP = -6

GBS_FP64 = 0
GBS_FP32 = 1
GBS_BF16X3 = 2
GBS_BF16X6 = 3

PRECISIONS = {"fp64": GBS_FP64, "fp32": GBS_FP32, "bf16x3": GBS_BF16X3, "bf16x6": GBS_BF16X6}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgbs.so")
_lock = threading.Lock()
_lib = None


class GbsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[gbs status {code}] {msg}")
        self.code = code


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def lib():
    """The loaded libgbs.so (raises if it is missing or cannot be loaded)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libgbs.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        ip = ctypes.POINTER(ctypes.c_int)
        L.gbs_make_network.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, vp,
                                       ctypes.POINTER(vp)]
        L.gbs_sample.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                 ctypes.c_int, ctypes.c_int]
        L.gbs_binned_counts.argtypes = [vp, ctypes.c_int64, dp, dp, dp, dp]
        L.gbs_binned_counts_device.argtypes = [vp, ctypes.c_int64, vp]
        L.gbs_check_finite.argtypes = [vp, i64p]
        L.gbs_debug_samples.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, dp,
                                        dp]
        L.gbs_get_accumulators.argtypes = [vp, ip, ip, dp, i64p]
        L.gbs_set_accumulators.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, i64p]
        L.gbs_reset.argtypes = [vp]
        L.gbs_network_info.argtypes = [vp, ip, ip, ip, i64p]
        L.gbs_binned_counts_noalloc.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int64, vp, vp]
        L.gbs_set_gemm_config.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.gbs_set_pair_autotune.argtypes = [ctypes.c_int]
        L.gbs_set_wait_limit.argtypes = [vp, ctypes.c_uint64]
        L.gbs_measure_fp64_rate.argtypes = [vp, dp]
        L.gbs_debug_windows.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                        ip]
        L.gbs_make_network_binned.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ip, ctypes.c_int,
                                              vp, ctypes.POINTER(vp)]
        L.gbs_histogram.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ip,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    i64p]
        L.gbs_moments.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        L.gbs_debug_occupations.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                            dp]
        L.gbs_sample_nd.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                    ctypes.c_int, ip]
        L.gbs_binned_counts_nd.argtypes = [vp, i64p, dp, dp, dp, dp]
        L.gbs_sample_2d.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.gbs_binned_counts_2d.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, dp, dp, dp, dp]
        L.gbs_gemm_config.argtypes = [vp, ip, ip, ip]
        L.gbs_set_sampler_fusion.argtypes = [vp, ctypes.c_int]
        L.gbs_sampler_fusion.argtypes = [vp, ip]
        L.gbs_make_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]
        L.gbs_sample_batch.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(ctypes.c_uint64), i64p, ip, ip]
        L.gbs_batch_info.argtypes = [vp, ip, ip, ip, ip, i64p]
        L.gbs_set_batch_config.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.gbs_free_batch.argtypes = [vp]
        L.gbs_free_batch.restype = None
        L.gbs_profile_enable.argtypes = [vp, ctypes.c_int]
        L.gbs_profile_read.argtypes = [vp, dp, i64p]
        L.gbs_free_network.argtypes = [vp]
        L.gbs_free_network.restype = None
        L.gbs_last_error.argtypes = []
        L.gbs_last_error.restype = ctypes.c_char_p
        L.gbs_make_network_device.argtypes = [ctypes.c_int, ctypes.c_int, vp, dp, ctypes.c_int,
                                              vp, ctypes.POINTER(vp)]
        fp = ctypes.POINTER(ctypes.c_float)
        L.gbs_mlp_create.argtypes = [ctypes.c_int] * 5 + [vp, ctypes.POINTER(vp)]
        L.gbs_mlp_param_count.argtypes = [vp, i64p]
        L.gbs_mlp_set_params.argtypes = [vp, fp]
        L.gbs_mlp_get_params.argtypes = [vp, fp]
        L.gbs_mlp_get_adam_state.argtypes = [vp, fp, fp, i64p]
        L.gbs_mlp_forward.argtypes = [vp, vp, ctypes.c_int, vp]
        L.gbs_mlp_gradients.argtypes = [vp, vp, vp, ctypes.c_int, dp, fp]
        L.gbs_mlp_train.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, fp, fp]
        L.gbs_mlp_free.argtypes = [vp]
        L.gbs_mlp_free.restype = None
        L.gbs_surrogate_features.argtypes = [ctypes.c_int, ip, ip, dp, ip, i64p, dp, i64p, vp, vp]
        L.gbs_surrogate_feature_stats.argtypes = [ctypes.c_int, vp, vp, vp]
        L.gbs_surrogate_standardize.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp]
        L.gbs_surrogate_encode.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int64, vp, vp]
        L.gbs_surrogate_decode.argtypes = [ctypes.c_int, vp, vp, vp, vp, ctypes.c_int64]
        for name in ("gbs_make_network", "gbs_sample", "gbs_binned_counts",
                     "gbs_binned_counts_device", "gbs_check_finite", "gbs_debug_samples",
                     "gbs_get_accumulators", "gbs_set_accumulators", "gbs_reset",
                     "gbs_network_info", "gbs_profile_enable", "gbs_profile_read",
                     "gbs_binned_counts_noalloc", "gbs_set_gemm_config", "gbs_gemm_config",
                     "gbs_set_pair_autotune", "gbs_set_wait_limit", "gbs_measure_fp64_rate",
                     "gbs_debug_windows",
                     "gbs_set_sampler_fusion", "gbs_sampler_fusion",
                     "gbs_make_batch", "gbs_sample_batch", "gbs_batch_info", "gbs_set_batch_config",
                     "gbs_make_network_device", "gbs_make_network_binned", "gbs_sample_2d",
                     "gbs_binned_counts_2d", "gbs_sample_nd", "gbs_binned_counts_nd",
                     "gbs_histogram", "gbs_moments",
                     "gbs_debug_occupations", "gbs_mlp_create", "gbs_mlp_param_count",
                     "gbs_mlp_set_params", "gbs_mlp_get_params", "gbs_mlp_get_adam_state",
                     "gbs_mlp_forward", "gbs_mlp_gradients", "gbs_mlp_train",
                     "gbs_surrogate_features", "gbs_surrogate_feature_stats",
                     "gbs_surrogate_standardize", "gbs_surrogate_encode",
                     "gbs_surrogate_decode"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(code: int):
    if code != GBS_OK:
        raise GbsError(code, gbs_last_error())


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gbs_last_error() -> str:
    return lib().gbs_last_error().decode(errors="replace")


class Network:
    """Handle of a network on the device (owns the C-side gbs_net_t)."""

    def __init__(self, handle: int, N: int, M: int, precision: int, stream: int):
        self.handle = ctypes.c_void_p(handle)
        self.N, self.M, self.precision, self.stream = N, M, precision, stream

    def __del__(self):
        try:
            if self.handle and self.handle.value:
                gbs_free_network(self)
        except Exception:
            pass


def gbs_make_network(T: np.ndarray, r: np.ndarray, precision=GBS_FP64,
                     stream: int = 0) -> Network:
    """T: complex (M, N) host array; r: (N,) squeezing; stream: cudaStream_t as int."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    T = np.ascontiguousarray(T, dtype=np.complex128)
    r = np.ascontiguousarray(r, dtype=np.float64)
    M, N = T.shape
    if r.shape != (N,):
        raise ValueError("r must have shape (N,)")
    Tf = T.view(np.float64)
    out = ctypes.c_void_p()
    _check(lib().gbs_make_network(N, M, _dptr(Tf), _dptr(r), int(precision),
                                  ctypes.c_void_p(stream), ctypes.byref(out)))
    return Network(out.value, N, M, int(precision), stream)


def gbs_make_network_device(T_dev_ptr: int, M: int, N: int, r: np.ndarray, precision=GBS_FP64,
                            stream: int = 0) -> Network:
    """T_dev_ptr: device address of an (M, N) complex128 row-major array."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    r = np.ascontiguousarray(r, dtype=np.float64)
    if r.shape != (N,):
        raise ValueError("r must have shape (N,)")
    out = ctypes.c_void_p()
    _check(lib().gbs_make_network_device(N, M, ctypes.c_void_p(T_dev_ptr), _dptr(r),
                                         int(precision), ctypes.c_void_p(stream),
                                         ctypes.byref(out)))
    return Network(out.value, N, M, int(precision), stream)


def gbs_make_network_binned(T: np.ndarray, r: np.ndarray, bins, precision=GBS_FP64,
                            stream: int = 0) -> Network:
    """T: complex (M, N); bins: M ints in 0..d-1 (the bin of each output mode, d <= 4)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    T = np.ascontiguousarray(T, dtype=np.complex128)
    r = np.ascontiguousarray(r, dtype=np.float64)
    b = np.ascontiguousarray(bins, dtype=np.int32)
    M, N = T.shape
    if r.shape != (N,) or b.shape != (M,):
        raise ValueError("r must have shape (N,) and bins (M,)")
    out = ctypes.c_void_p()
    _check(lib().gbs_make_network_binned(N, M, _dptr(T.view(np.float64)), _dptr(r),
                                         b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                         int(precision), ctypes.c_void_p(stream),
                                         ctypes.byref(out)))
    return Network(out.value, N, M, int(precision), stream)


def gbs_histogram(net: Network, seed: int, first_sample: int, E: int, m, lo: float, hi: float,
                  nbins: int) -> np.ndarray:
    """Counts [2][len(m)][nbins + 2] of Re G_0(m) (matrix-P) and Re G_+(m)
    over trajectories first_sample..first_sample+E-1 (bin 0: below lo, last: >= hi)."""
    mm = (ctypes.c_int * len(m))(*[int(x) for x in m])
    out = np.zeros(2 * len(m) * (nbins + 2), dtype=np.int64)
    _check(lib().gbs_histogram(net.handle, seed, first_sample, E, mm, len(m), float(lo),
                               float(hi), nbins,
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return out.reshape(2, len(m), nbins + 2)


def gbs_moments(net: Network, seed: int, first_sample: int, E: int, n_sub: int, mmax: int,
                cmax: int):
    """(mom, sig_mom, marg, sig_marg): normally-ordered moments <:n_j^m:>,
    m = 1..mmax, as [2][M][mmax] and single-mode marginals P_j(c),
    c = 0..cmax, as [2][M][cmax + 1] (index 0 matrix-P, 1 +P), over
    trajectories first_sample..first_sample+E-1 with n_sub sub-ensembles."""
    _, M, _, _ = gbs_network_info(net)
    mom = np.zeros(2 * M * mmax)
    smom = np.zeros(2 * M * mmax)
    marg = np.zeros(2 * M * (cmax + 1))
    smarg = np.zeros(2 * M * (cmax + 1))
    _check(lib().gbs_moments(net.handle, seed, first_sample, E, n_sub, mmax, cmax, _dptr(mom),
                             _dptr(smom), _dptr(marg), _dptr(smarg)))
    return (mom.reshape(2, M, mmax), smom.reshape(2, M, mmax),
            marg.reshape(2, M, cmax + 1), smarg.reshape(2, M, cmax + 1))


def gbs_debug_occupations(net: Network, seed: int, e0: int, count: int) -> np.ndarray:
    """[M][count] complex: n'_i = alpha'_i beta'_i of trajectories e0..e0+count-1."""
    _, M, _, _ = gbs_network_info(net)
    out = np.zeros(2 * M * count)
    _check(lib().gbs_debug_occupations(net.handle, seed, e0, count, _dptr(out)))
    return out.view(np.complex128).reshape(M, count)


def gbs_sample_nd(net: Network, seed: int, first_sample: int, E: int, n_sub: int, K) -> None:
    """Binned sums of a network of d bins on the grid K (d powers of two)."""
    KK = (ctypes.c_int * len(K))(*[int(k) for k in K])
    _check(lib().gbs_sample_nd(net.handle, seed, first_sample, E, n_sub, KK))


def gbs_binned_counts_nd(net: Network, K, m_offset=None):
    """(P_mP, sigma_mP, P_plusP, sigma_plusP), each of shape K, bins m_offset.."""
    K = [int(k) for k in K]
    mo = [0] * len(K) if m_offset is None else [int(v) for v in m_offset]
    MO = (ctypes.c_int64 * len(K))(*mo)
    size = int(np.prod(K))
    outs = [np.zeros(size) for _ in range(4)]
    _check(lib().gbs_binned_counts_nd(net.handle, MO, *[_dptr(o) for o in outs]))
    return tuple(o.reshape(K) for o in outs)


def gbs_sample_2d(net: Network, seed: int, first_sample: int, E: int, n_sub: int, K1: int,
                  K2: int) -> None:
    _check(lib().gbs_sample_2d(net.handle, seed, first_sample, E, n_sub, K1, K2))


def gbs_binned_counts_2d(net: Network, K1: int, K2: int, m1_offset: int = 0, m2_offset: int = 0):
    """(P_mP, sigma_mP, P_plusP, sigma_plusP), each (K1, K2)."""
    outs = [np.zeros(K1 * K2) for _ in range(4)]
    _check(lib().gbs_binned_counts_2d(net.handle, m1_offset, m2_offset, *[_dptr(o) for o in outs]))
    return tuple(o.reshape(K1, K2) for o in outs)


def gbs_sample(net: Network, seed: int, first_sample: int, E: int, n_sub: int, K1: int) -> None:
    _check(lib().gbs_sample(net.handle, seed, first_sample, E, n_sub, K1))


def gbs_binned_counts(net: Network, m_offset: int = 0, K1: Optional[int] = None
                      ) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """(P_mP, sigma_mP, P_plusP, sigma_plusP), each K1 doubles, bins m_offset.."""
    if K1 is None:
        K1 = gbs_get_accumulators(net, with_data=False)[1]
    outs = [np.zeros(K1) for _ in range(4)]
    _check(lib().gbs_binned_counts(net.handle, m_offset, *[_dptr(o) for o in outs]))
    return tuple(outs)


def gbs_binned_counts_device(net: Network, m_offset: int, out_dev_ptr: int) -> None:
    _check(lib().gbs_binned_counts_device(net.handle, m_offset, ctypes.c_void_p(out_dev_ptr)))


def gbs_binned_counts_noalloc(acc_dev_ptr: int, counts_dev_ptr: int, n_sub: int, K1: int,
                              m_offset: int, out_dev_ptr: int, stream: int = 0) -> None:
    """Inversion of caller-owned device sums into a caller-owned device
    buffer; the library allocates nothing (fixed internal work space)."""
    _check(lib().gbs_binned_counts_noalloc(ctypes.c_void_p(acc_dev_ptr),
                                           ctypes.c_void_p(counts_dev_ptr), n_sub, K1, m_offset,
                                           ctypes.c_void_p(out_dev_ptr), ctypes.c_void_p(stream)))


def gbs_check_finite(net: Network) -> int:
    c = ctypes.c_int64()
    code = lib().gbs_check_finite(net.handle, ctypes.byref(c))
    if code not in (GBS_OK, GBS_ENONFINITE):
        _check(code)
    return int(c.value)


def gbs_debug_samples(net: Network, seed: int, e0: int, count: int):
    """Per-trajectory (n[count], n_S[count] complex) from the device kernels."""
    n = np.zeros(count)
    nS = np.zeros(2 * count)
    _check(lib().gbs_debug_samples(net.handle, seed, e0, count, _dptr(n), _dptr(nS)))
    return n, nS.view(np.complex128)


def gbs_debug_windows(net: Network, seed: int, e0: int, count: int) -> np.ndarray:
    """Per-trajectory generating-function windows (w1, w2) as int32 [count, 2]."""
    w = np.zeros(2 * count, dtype=np.int32)
    _check(lib().gbs_debug_windows(net.handle, seed, e0, count,
                                   w.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return w.reshape(count, 2)


def gbs_get_accumulators(net: Network, with_data: bool = True):
    """(n_sub, K1, acc[2][n_sub][K1] complex, counts[n_sub])."""
    ns = ctypes.c_int()
    k1 = ctypes.c_int()
    _check(lib().gbs_get_accumulators(net.handle, ctypes.byref(ns), ctypes.byref(k1), None, None))
    if not with_data or ns.value == 0:
        return ns.value, k1.value, None, None
    acc = np.zeros(4 * ns.value * k1.value)
    cnt = np.zeros(ns.value, dtype=np.int64)
    _check(lib().gbs_get_accumulators(net.handle, ctypes.byref(ns), ctypes.byref(k1), _dptr(acc),
                                      cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return ns.value, k1.value, acc.view(np.complex128).reshape(2, ns.value, k1.value), cnt


def gbs_set_accumulators(net: Network, acc: np.ndarray, counts: np.ndarray) -> None:
    acc = np.ascontiguousarray(acc, dtype=np.complex128)
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    _, n_sub, K1 = acc.shape
    _check(lib().gbs_set_accumulators(net.handle, n_sub, K1, _dptr(acc.view(np.float64)),
                                      counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))


def gbs_reset(net: Network) -> None:
    _check(lib().gbs_reset(net.handle))


def gbs_network_info(net: Network):
    N = ctypes.c_int()
    M = ctypes.c_int()
    p = ctypes.c_int()
    c = ctypes.c_int64()
    _check(lib().gbs_network_info(net.handle, ctypes.byref(N), ctypes.byref(M), ctypes.byref(p),
                                  ctypes.byref(c)))
    return N.value, M.value, p.value, c.value


def gbs_set_gemm_config(net: Network, pair: int, band: int = 0, keep_a: int = 0) -> None:
    """Tile configuration of the tcgen05 GEMM: pair 1 (one CTA per tile) or 2
    (CTA pairs), band = mode-tile groups per band of the tile order (0: plain
    order), keep_a = 1: a band's A tiles with the evict-last L2 policy; pair
    0 = autotune."""
    _check(lib().gbs_set_gemm_config(net.handle, int(pair), int(band), int(keep_a)))


def gbs_gemm_config(net: Network):
    """(pair, band, keep_a) in use; (0, 0, 0) before the first chunk."""
    p = ctypes.c_int()
    b = ctypes.c_int()
    k = ctypes.c_int()
    _check(lib().gbs_gemm_config(net.handle, ctypes.byref(p), ctypes.byref(b), ctypes.byref(k)))
    return p.value, b.value, k.value


def gbs_set_pair_autotune(enable: bool) -> None:
    """Whether the GEMM autotuners also time CTA pairs (process-wide)."""
    _check(lib().gbs_set_pair_autotune(int(bool(enable))))


def gbs_measure_fp64_rate(stream=0) -> float:
    """The device's FP64 FMA rate (TFLOP/s) from a CUDA-event-timed probe."""
    t = ctypes.c_double()
    _check(lib().gbs_measure_fp64_rate(ctypes.c_void_p(stream), ctypes.byref(t)))
    return t.value


def gbs_set_wait_limit(net: Network, limit_ns: int) -> None:
    """Bound (ns) of every pipeline wait in the network's GEMM launches."""
    _check(lib().gbs_set_wait_limit(net.handle, int(limit_ns)))


def gbs_set_sampler_fusion(net: Network, mode) -> None:
    """Sample the next chunk inside the GEMM of this one (BF16X3): 0 / False
    never, 1 / True from 900 output modes (the default), 2 whenever possible."""
    _check(lib().gbs_set_sampler_fusion(net.handle, int(mode)))


def gbs_sampler_fusion(net: Network) -> bool:
    """Whether the next multi-chunk gbs_sample runs the folded sampler."""
    a = ctypes.c_int()
    _check(lib().gbs_sampler_fusion(net.handle, ctypes.byref(a)))
    return bool(a.value)


class Batch:
    """Handle of a batch of networks (the networks stay owned by the caller)."""

    def __init__(self, handle: int, nets):
        self.handle = ctypes.c_void_p(handle)
        self.nets = list(nets)

    def __del__(self):
        try:
            if self.handle and self.handle.value:
                gbs_free_batch(self)
        except Exception:
            pass


def gbs_make_batch(nets) -> Batch:
    arr = (ctypes.c_void_p * len(nets))(*[n.handle.value for n in nets])
    out = ctypes.c_void_p()
    _check(lib().gbs_make_batch(arr, len(nets), ctypes.byref(out)))
    return Batch(out.value, nets)


def gbs_sample_batch(batch: Batch, seeds, first_sample, E, n_sub, K1) -> None:
    n = len(batch.nets)
    u64 = ctypes.c_uint64 * n
    i64 = ctypes.c_int64 * n
    i32 = ctypes.c_int * n
    _check(lib().gbs_sample_batch(batch.handle, u64(*[int(x) for x in seeds]),
                                  u64(*[int(x) for x in first_sample]),
                                  i64(*[int(x) for x in E]), i32(*[int(x) for x in n_sub]),
                                  i32(*[int(x) for x in K1])))


def gbs_set_batch_config(batch: Batch, pair: int, band: int = 0, stages: int = 0) -> None:
    """The batch GEMM's configuration (pair 1 or 2, band >= 0, operand-ring
    stages: 0 = the deepest); pair 0 = autotune."""
    _check(lib().gbs_set_batch_config(batch.handle, int(pair), int(band), int(stages)))


def gbs_batch_info(batch: Batch):
    """((pair, band, ring stages) of the batch GEMM, rounds, GEMM tiles) of
    the last gbs_sample_batch."""
    c = ctypes.c_int()
    b = ctypes.c_int()
    st = ctypes.c_int()
    r = ctypes.c_int()
    t = ctypes.c_int64()
    _check(lib().gbs_batch_info(batch.handle, ctypes.byref(c), ctypes.byref(b), ctypes.byref(st),
                                ctypes.byref(r), ctypes.byref(t)))
    return (c.value, b.value, st.value), r.value, t.value


def gbs_free_batch(batch: Batch) -> None:
    if batch.handle and batch.handle.value:
        lib().gbs_free_batch(batch.handle)
        batch.handle = ctypes.c_void_p()


GBS_NPHASES = 6
PHASES = ("sample", "gemm", "finalize", "gf", "invert", "moments")


def gbs_profile_enable(net: Network, enable: bool = True) -> None:
    _check(lib().gbs_profile_enable(net.handle, 1 if enable else 0))


def gbs_profile_read(net: Network):
    """{phase: (milliseconds, launches)} since the last enable/read."""
    ms = np.zeros(GBS_NPHASES)
    ln = np.zeros(GBS_NPHASES, dtype=np.int64)
    _check(lib().gbs_profile_read(net.handle, _dptr(ms),
                                  ln.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return {PHASES[i]: (float(ms[i]), int(ln[i])) for i in range(GBS_NPHASES)}


def gbs_free_network(net: Network) -> None:
    if net.handle and net.handle.value:
        lib().gbs_free_network(net.handle)
        net.handle = ctypes.c_void_p()


# ----------------------------------------------------------------------------
# Learned surrogate (include/gbs_surrogate.h)
# ----------------------------------------------------------------------------
GBS_SUR_FEATURES = 10
GBS_SUR_RECORD = 14
GBS_SUR_GRID = 256
GBS_SUR_OUT = 512


def _fptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Mlp:
    """Handle of an MLP on the device (owns the C-side gbs_mlp_t)."""

    def __init__(self, handle: int, in_dim: int, width: int, out_dim: int, layers: int):
        self.handle = ctypes.c_void_p(handle)
        self.in_dim, self.width, self.out_dim, self.layers = in_dim, width, out_dim, layers

    def __del__(self):
        try:
            if self.handle and self.handle.value:
                gbs_mlp_free(self)
        except Exception:
            pass


def gbs_mlp_create(in_dim: int, width: int, out_dim: int, layers: int, max_batch: int,
                   stream: int = 0) -> Mlp:
    out = ctypes.c_void_p()
    _check(lib().gbs_mlp_create(in_dim, width, out_dim, layers, max_batch,
                                ctypes.c_void_p(stream), ctypes.byref(out)))
    return Mlp(out.value, in_dim, width, out_dim, layers)


def gbs_mlp_param_count(mlp: Mlp) -> int:
    c = ctypes.c_int64()
    _check(lib().gbs_mlp_param_count(mlp.handle, ctypes.byref(c)))
    return int(c.value)


def gbs_mlp_set_params(mlp: Mlp, params: np.ndarray) -> None:
    params = np.ascontiguousarray(params, dtype=np.float32)
    if params.size != gbs_mlp_param_count(mlp):
        raise ValueError("wrong parameter count")
    _check(lib().gbs_mlp_set_params(mlp.handle, _fptr(params)))


def gbs_mlp_get_params(mlp: Mlp) -> np.ndarray:
    out = np.zeros(gbs_mlp_param_count(mlp), dtype=np.float32)
    _check(lib().gbs_mlp_get_params(mlp.handle, _fptr(out)))
    return out


def gbs_mlp_get_adam_state(mlp: Mlp):
    """(first moments, second moments, Adam steps taken)."""
    n = gbs_mlp_param_count(mlp)
    m1 = np.zeros(n, dtype=np.float32)
    m2 = np.zeros(n, dtype=np.float32)
    st = ctypes.c_int64()
    _check(lib().gbs_mlp_get_adam_state(mlp.handle, _fptr(m1), _fptr(m2), ctypes.byref(st)))
    return m1, m2, int(st.value)


def gbs_mlp_forward(mlp: Mlp, X_dev_ptr: int, batch: int, Y_dev_ptr: int) -> None:
    _check(lib().gbs_mlp_forward(mlp.handle, ctypes.c_void_p(X_dev_ptr), batch,
                                 ctypes.c_void_p(Y_dev_ptr)))


def gbs_mlp_gradients(mlp: Mlp, X_dev_ptr: int, T_dev_ptr: int, batch: int):
    """(loss, packed gradient) of one batch."""
    loss = ctypes.c_double()
    grad = np.zeros(gbs_mlp_param_count(mlp), dtype=np.float32)
    _check(lib().gbs_mlp_gradients(mlp.handle, ctypes.c_void_p(X_dev_ptr),
                                   ctypes.c_void_p(T_dev_ptr), batch, ctypes.byref(loss),
                                   _fptr(grad)))
    return float(loss.value), grad


def gbs_mlp_train(mlp: Mlp, X_dev_ptr: int, T_dev_ptr: int, batch: int, lr) -> np.ndarray:
    """len(lr) full-batch Adam steps; returns the loss before each step."""
    lr = np.ascontiguousarray(lr, dtype=np.float32)
    hist = np.zeros(lr.size, dtype=np.float32)
    _check(lib().gbs_mlp_train(mlp.handle, ctypes.c_void_p(X_dev_ptr), ctypes.c_void_p(T_dev_ptr),
                               batch, int(lr.size), _fptr(lr), _fptr(hist)))
    return hist


def gbs_mlp_free(mlp: Mlp) -> None:
    if mlp.handle and mlp.handle.value:
        lib().gbs_mlp_free(mlp.handle)
        mlp.handle = ctypes.c_void_p()


def gbs_surrogate_features(N, M, t, K1, m_off, r_list, feat_dev_ptr: int, stream: int = 0) -> None:
    """Feature records [count][14] of networks (N[i], M[i], t[i], K1[i],
    m_off[i], squeezing r_list[i]) into device memory."""
    count = len(N)
    i32 = ctypes.c_int * count
    r_all = np.ascontiguousarray(np.concatenate([np.asarray(r, dtype=np.float64) for r in r_list]))
    r_off = np.zeros(count + 1, dtype=np.int64)
    r_off[1:] = np.cumsum([len(r) for r in r_list])
    t = np.ascontiguousarray(t, dtype=np.float64)
    mo = np.ascontiguousarray(m_off, dtype=np.int64)
    _check(lib().gbs_surrogate_features(count, i32(*[int(x) for x in N]),
                                        i32(*[int(x) for x in M]), _dptr(t),
                                        i32(*[int(x) for x in K1]),
                                        mo.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        _dptr(r_all),
                                        r_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        ctypes.c_void_p(stream), ctypes.c_void_p(feat_dev_ptr)))


def gbs_surrogate_feature_stats(count: int, feat_dev_ptr: int, stats_dev_ptr: int,
                                stream: int = 0) -> None:
    _check(lib().gbs_surrogate_feature_stats(count, ctypes.c_void_p(feat_dev_ptr),
                                             ctypes.c_void_p(stream),
                                             ctypes.c_void_p(stats_dev_ptr)))


def gbs_surrogate_standardize(count: int, feat_dev_ptr: int, stats_dev_ptr: int, X_dev_ptr: int,
                              in_domain_dev_ptr: int = 0, stream: int = 0) -> None:
    _check(lib().gbs_surrogate_standardize(count, ctypes.c_void_p(feat_dev_ptr),
                                           ctypes.c_void_p(stats_dev_ptr), ctypes.c_void_p(stream),
                                           ctypes.c_void_p(X_dev_ptr),
                                           ctypes.c_void_p(in_domain_dev_ptr or None)))


def gbs_surrogate_encode(count: int, feat_dev_ptr: int, P_dev_ptr: int, ldP: int, Y_dev_ptr: int,
                         stream: int = 0) -> None:
    _check(lib().gbs_surrogate_encode(count, ctypes.c_void_p(feat_dev_ptr),
                                      ctypes.c_void_p(P_dev_ptr), ldP, ctypes.c_void_p(stream),
                                      ctypes.c_void_p(Y_dev_ptr)))


def gbs_surrogate_decode(count: int, feat_dev_ptr: int, Y_dev_ptr: int, P_dev_ptr: int, ldP: int,
                         stream: int = 0) -> None:
    _check(lib().gbs_surrogate_decode(count, ctypes.c_void_p(feat_dev_ptr),
                                      ctypes.c_void_p(Y_dev_ptr), ctypes.c_void_p(stream),
                                      ctypes.c_void_p(P_dev_ptr), ldP))
