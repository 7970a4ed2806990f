"""CPU FP64 oracle for the matrix-P total-count estimator (arXiv:2503.12749).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline / reference arm may import this package.  It shares no
code with the CUDA library in ``paper_2503_12749_gb300``; both sides take
their inputs from ``workloads``.

``oracle.c`` holds the Monte-Carlo estimator written step by step from the
paper (see its header).  This module compiles it with gcc on first use and
wraps it with ctypes.  ``oracle.exact`` holds the closed-form references.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (plain gcc, OpenMP, no FP
    contraction so x86 and Arm builds round identically)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        u32 = ctypes.POINTER(ctypes.c_uint32)
        i64 = ctypes.POINTER(ctypes.c_int64)
        lib.orc_philox4x32_10.argtypes = [u32, u32, u32]
        lib.orc_philox4x32_10.restype = None
        lib.orc_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, d, d]
        lib.orc_normals.restype = None
        lib.orc_sample_inputs.argtypes = [ctypes.c_int, d, ctypes.c_uint64, ctypes.c_uint64, d, d]
        lib.orc_sample_inputs.restype = ctypes.c_double
        lib.orc_samples.argtypes = [ctypes.c_int, ctypes.c_int, d, d, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_int64, d, d, ctypes.c_int]
        lib.orc_samples.restype = ctypes.c_int
        lib.orc_sample_amplitudes.argtypes = [ctypes.c_int, ctypes.c_int, d, d, ctypes.c_uint64,
                                              ctypes.c_uint64, d, d, d, d]
        lib.orc_sample_amplitudes.restype = None
        lib.orc_projector_direct.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_int, d, d]
        lib.orc_projector_direct.restype = None
        lib.orc_gf_sample.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, d, d]
        lib.orc_gf_sample.restype = None
        lib.orc_accumulate_gf.argtypes = [d, d, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                          ctypes.c_int, d, i64, ctypes.c_int]
        lib.orc_accumulate_gf.restype = ctypes.c_int
        lib.orc_invert.argtypes = [d, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int64, d, d, d,
                                   ctypes.c_int]
        lib.orc_invert.restype = ctypes.c_int
        lib.orc_direct_bins.argtypes = [d, d, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, d, d, ctypes.c_int]
        lib.orc_direct_bins.restype = ctypes.c_int
        lib.orc_run.argtypes = [ctypes.c_int, ctypes.c_int, d, d, ctypes.c_uint64, ctypes.c_uint64,
                                ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int64, d, d,
                                d, ctypes.c_int]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_max_threads.argtypes = []
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _T_interleaved(T: np.ndarray) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.complex128)
    return T.view(np.float64)  # (M, 2N) interleaved re, im


def max_threads() -> int:
    return int(_load().orc_max_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    p = ctypes.POINTER(ctypes.c_uint32)
    lib.orc_philox4x32_10(c.ctypes.data_as(p), k.ctypes.data_as(p), out.ctypes.data_as(p))
    return out


def normals(seed: int, e: int, j: int) -> Tuple[float, float]:
    lib = _load()
    w1 = ctypes.c_double()
    w2 = ctypes.c_double()
    lib.orc_normals(seed, e, j, ctypes.byref(w1), ctypes.byref(w2))
    return w1.value, w2.value


def sample_inputs(r: np.ndarray, seed: int, e: int):
    """(alpha, beta, n) of sample e."""
    lib = _load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    N = r.shape[0]
    a = np.zeros(N)
    b = np.zeros(N)
    n = lib.orc_sample_inputs(N, _dp(r), seed, e, _dp(a), _dp(b))
    return a, b, n


def sample_amplitudes(T: np.ndarray, r: np.ndarray, seed: int, e: int):
    """(alpha, beta, alpha', beta') of sample e; alpha', beta' complex (M,)."""
    lib = _load()
    M, N = T.shape
    Ti = _T_interleaved(T)
    r = np.ascontiguousarray(r, dtype=np.float64)
    a = np.zeros(N)
    b = np.zeros(N)
    ap = np.zeros(2 * M)
    bp = np.zeros(2 * M)
    lib.orc_sample_amplitudes(N, M, _dp(Ti), _dp(r), seed, e, _dp(a), _dp(b), _dp(ap), _dp(bp))
    return a, b, ap.view(np.complex128), bp.view(np.complex128)


def samples(T: np.ndarray, r: np.ndarray, seed: int, e0: int, E: int, threads: int = 0):
    """Per-sample input totals n[E] (float64) and output totals n_S[E] (complex128)."""
    lib = _load()
    M, N = T.shape
    Ti = _T_interleaved(T)
    r = np.ascontiguousarray(r, dtype=np.float64)
    n = np.zeros(E)
    nS = np.zeros(2 * E)
    rc = lib.orc_samples(N, M, _dp(Ti), _dp(r), seed, e0, E, _dp(n), _dp(nS), threads)
    if rc != 0:
        raise RuntimeError(f"orc_samples failed ({rc})")
    return n, nS.view(np.complex128)


def gf_sample(n: float, nS: complex, K1: int):
    """Per-sample generating functions at z_k = exp(2 pi i k / K1): (G_mP, G_+P)."""
    lib = _load()
    gm = np.zeros(2 * K1)
    gp = np.zeros(2 * K1)
    lib.orc_gf_sample(float(n), float(np.real(nS)), float(np.imag(nS)), K1, _dp(gm), _dp(gp))
    return gm.view(np.complex128), gp.view(np.complex128)


def projector_direct(n: float, nS: complex, m0: int, count: int):
    """Per-sample projectors G(m), m = m0..m0+count-1: (matrix-P, +P)."""
    lib = _load()
    gm = np.zeros(2 * count)
    gp = np.zeros(2 * count)
    lib.orc_projector_direct(float(n), float(np.real(nS)), float(np.imag(nS)), m0, count,
                             _dp(gm), _dp(gp))
    return gm.view(np.complex128), gp.view(np.complex128)


def accumulate_gf(n: np.ndarray, nS: np.ndarray, e0: int, n_sub: int, K1: int,
                  threads: int = 0):
    """Sub-ensemble GF sums acc[2][n_sub][K1] (complex) and counts[n_sub]."""
    lib = _load()
    n = np.ascontiguousarray(n, dtype=np.float64)
    nSf = np.ascontiguousarray(nS, dtype=np.complex128).view(np.float64)
    E = n.shape[0]
    acc = np.zeros(4 * n_sub * K1)
    cnt = np.zeros(n_sub, dtype=np.int64)
    rc = lib.orc_accumulate_gf(_dp(n), _dp(nSf), e0, E, n_sub, K1, _dp(acc),
                               cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), threads)
    if rc != 0:
        raise RuntimeError(f"orc_accumulate_gf failed ({rc})")
    return acc.view(np.complex128).reshape(2, n_sub, K1), cnt


def invert(acc: np.ndarray, counts: np.ndarray, m_off: int = 0, threads: int = 0):
    """(P[2][K1], sigma[2][K1], Im_max[2]) from sub-ensemble sums."""
    lib = _load()
    _, n_sub, K1 = acc.shape
    a = np.ascontiguousarray(acc, dtype=np.complex128).view(np.float64)
    cnt = np.ascontiguousarray(counts, dtype=np.int64)
    P = np.zeros(2 * K1)
    s = np.zeros(2 * K1)
    im = np.zeros(2)
    rc = lib.orc_invert(_dp(a), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n_sub, K1,
                        m_off, _dp(P), _dp(s), _dp(im), threads)
    if rc != 0:
        raise RuntimeError(f"orc_invert failed ({rc})")
    return P.reshape(2, K1), s.reshape(2, K1), im


def direct_bins(n: np.ndarray, nS: np.ndarray, e0: int, n_sub: int, m0: int, count: int,
                threads: int = 0):
    """Direct per-bin route: (P[2][count], sigma[2][count])."""
    lib = _load()
    n = np.ascontiguousarray(n, dtype=np.float64)
    nSf = np.ascontiguousarray(nS, dtype=np.complex128).view(np.float64)
    P = np.zeros(2 * count)
    s = np.zeros(2 * count)
    rc = lib.orc_direct_bins(_dp(n), _dp(nSf), e0, n.shape[0], n_sub, m0, count, _dp(P), _dp(s),
                             threads)
    if rc != 0:
        raise RuntimeError(f"orc_direct_bins failed ({rc})")
    return P.reshape(2, count), s.reshape(2, count)


def run(T: np.ndarray, r: np.ndarray, seed: int, e0: int, E: int, n_sub: int, K1: int,
        m_off: int = 0, threads: int = 0):
    """Whole estimator: (P[2][K1], sigma[2][K1], Im_max[2]); row 0 matrix-P, row 1 +P."""
    lib = _load()
    M, N = T.shape
    Ti = _T_interleaved(T)
    r = np.ascontiguousarray(r, dtype=np.float64)
    P = np.zeros(2 * K1)
    s = np.zeros(2 * K1)
    im = np.zeros(2)
    rc = lib.orc_run(N, M, _dp(Ti), _dp(r), seed, e0, E, n_sub, K1, m_off, _dp(P), _dp(s),
                     _dp(im), threads)
    if rc != 0:
        raise RuntimeError(f"orc_run failed ({rc})")
    return P.reshape(2, K1), s.reshape(2, K1), im
