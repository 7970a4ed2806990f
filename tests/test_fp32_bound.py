"""The n_S tolerance of the FP32 path, checked on an emulation of its arithmetic.

The FP32 GEMM forms Re/Im alpha'_i = sum_j fl32(Re/Im T_ij) fl32(alpha_j) by
N fused multiply-adds in FP32 (likewise beta' = T* beta), then the epilogue
takes n'_i = alpha'_i beta'_i and n_S = sum_i n'_i in FP64.  Emulated here on
the CPU: each fused multiply-add is the FP64 value of the exact FP32 product
plus the FP32 accumulator, rounded to FP32 (an FP32 x FP32 product is exact
in FP64).  The bound the GPU tests use,
|d n_S| <= 2 (N + 2) 2^-24 (1 + 2^-10) sum_i A_i B_i with
A_i = sum_j |T_ij| |alpha_j|, must hold for the emulation against the FP64
oracle, sit well above FP64 rounding, and fail (at small N, where the
worst-case bound is not far above the actual errors) when T is rounded to
BF16 instead of FP32 (a plausible mistake in the staging).
"""

import numpy as np

import oracle
import workloads as wl

U32 = 2.0 ** -24


def _round_bf16(x):
    """Round float64 values to BF16 (8-bit significand), round to nearest even."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _emulated_nS(T, alpha, beta, round_T):
    """n_S of one trajectory from the FP32 GEMM's arithmetic (operands of T
    rounded by round_T, samples rounded to FP32)."""
    Tr = round_T(T.real)
    Ti = round_T(T.imag)
    a = np.float32(alpha).astype(np.float64)
    b = np.float32(beta).astype(np.float64)
    M, N = T.shape
    acc = np.zeros((4, M), dtype=np.float32)  # Re T a, Im T a, Re T b, Im T b
    for j in range(N):
        prods = np.stack([Tr[:, j] * a[j], Ti[:, j] * a[j], Tr[:, j] * b[j], Ti[:, j] * b[j]])
        acc = (prods + acc.astype(np.float64)).astype(np.float32)
    ar, ai, br, bi = acc.astype(np.float64)
    return complex(np.sum(ar * br + ai * bi), np.sum(ai * br - ar * bi))


def _check(N, M, seed, E=12):
    net = wl.small_network(N, M=M, r=0.7, t2=0.9, seed=seed, general_loss=True)
    absT = np.abs(net.T)
    _, nSo = oracle.samples(net.T, net.r, net.seed_s, 0, E)
    rel32, relbf = [], []
    for e in range(E):
        alpha, beta, _, _ = oracle.sample_amplitudes(net.T, net.r, net.seed_s, e)
        scale = float(np.sum((absT @ np.abs(alpha)) * (absT @ np.abs(beta))))
        bound = 2.0 * (N + 2) * U32 * (1.0 + 2.0 ** -10) * scale
        fp32 = lambda x: np.float32(x).astype(np.float64)
        rel32.append(abs(_emulated_nS(net.T, alpha, beta, fp32) - nSo[e]) / bound)
        relbf.append(abs(_emulated_nS(net.T, alpha, beta, _round_bf16) - nSo[e]) / bound)
    return np.array(rel32), np.array(relbf)


def test_fp32_bound_holds_for_the_emulated_gemm():
    for N, M, seed in ((16, 16, 1), (9, 7, 2), (257, 40, 3)):
        rel32, _ = _check(N, M, seed)
        assert np.all(rel32 <= 1.0), (N, M, rel32.max())
        # the emulation is not FP64: its errors are far above FP64 rounding
        assert rel32.max() > 2.0 ** -20, (N, M, rel32.max())


def test_fp32_bound_catches_bf16_staging():
    """The bound grows with N (a worst case over rounding signs), so at
    N = 257 BF16 staging stays inside it (0.2 of it for these seeds, the FP32
    errors 3e-5); at small N it exceeds it by 50-300x."""
    for N, M, seed in ((16, 16, 1), (9, 7, 2)):
        _, relbf = _check(N, M, seed)
        assert relbf.max() > 10.0, (N, M, relbf.max())
