"""The error bound the TF32x3 projection parity tests use (CPU): an emulation of the
pipeline -- FP32 operands, tf32 hi/lo parts rounded to nearest (ties away from zero, as the
conversion the kernels use), products hi*hi + hi*lo + lo*hi formed exactly, and an FP32
accumulator rounded to nearest after every 8-element step of each of the three passes, as
one tensor-core MMA adds its 8 products -- stays within it, and the bound is not vacuous."""
import numpy as np
import pytest

import oracle
from tests.systems_small import small
from tests.test_gpu_parity import _tf32x3_x0_bound


def _tf32(x):
    """Round FP32 values to tf32 (10 explicit significand bits), to nearest, ties away."""
    a = np.asarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) >> 13) << 13
    return b.astype(np.uint32).view(np.float32)


def _split(x):
    x = np.asarray(x, dtype=np.float32)
    hi = _tf32(x)
    lo = _tf32((x - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


def _mma_sum(A, B, passes=3):
    """sum_k A[i,k] B[k,j] with TF32x3 parts and an FP32 accumulator rounded after every
    8-wide K step of each pass (the order of the kernels: hi*hi, hi*lo, lo*hi per step);
    passes=1 keeps only hi*hi (a single tf32 pass)."""
    ah, al = _split(A)
    bh, bl = _split(B)
    K = A.shape[1]
    acc = np.zeros((A.shape[0], B.shape[1]), dtype=np.float32)
    for k0 in range(0, K, 8):
        sl = slice(k0, min(K, k0 + 8))
        for x, y in ((ah, bh), (ah, bl), (al, bh))[:passes]:
            acc = (acc.astype(np.float64) + x[:, sl] @ y[sl, :]).astype(np.float32)
    return acc.astype(np.float64)


def _emulate(s, om, u, passes=3):
    psi32 = s.psi.astype(np.float32)
    u32 = u.astype(np.float32)
    b = (psi32 * u32[None, :]).astype(np.float32)
    G = _mma_sum(psi32, b.T, passes)                   # one chunk (N_d < 4096)
    d = s.eps[:, None] - s.eps[None, :] - 1j * om
    C = (-s.dV * G / d)
    Cre = C.real.astype(np.float32)
    Cim = C.imag.astype(np.float32)
    return _mma_sum(psi32.T, Cre, passes).T + 1j * _mma_sum(psi32.T, Cim, passes).T


def test_tf32_rounding_is_to_nearest():
    x = np.array([1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -12, -(1.0 + 2.0 ** -11)], dtype=np.float32)
    assert np.allclose(_tf32(x), [1.0 + 2.0 ** -10, 1.0 + 2.0 ** -10, -(1.0 + 2.0 ** -10)])


@pytest.mark.parametrize("om", [0.0203, 0.69, 8.8])
def test_tf32x3_pipeline_within_bound(om):
    s = small()
    rng = np.random.default_rng(8)
    u = rng.standard_normal(s.N_d)
    x0 = _emulate(s, om, u)
    ref = oracle.galerkin(s, om, u)
    bre, bim = _tf32x3_x0_bound(s, om, u)
    assert np.all(np.abs(x0.real - ref.real) <= bre)
    assert np.all(np.abs(x0.imag - ref.imag) <= bim)
    # not vacuous: the emulated error uses a visible part of the bound (the probabilistic
    # accumulation term sums |terms|, which for the random-sign sums here overstates the
    # error by about sqrt(n); the bound is still ~5e-4 of max|x0|) ...
    ratio = np.max(np.abs(x0 - ref)) / np.max(np.hypot(bre, bim))
    assert ratio > 1e-3, ratio
    # ... and sharp enough that a lost split pass (a single tf32 pass) breaks it
    x1 = _emulate(s, om, u, passes=1)
    assert np.any(np.abs(x1.real - ref.real) > bre) or np.any(np.abs(x1.imag - ref.imag) > bim)
