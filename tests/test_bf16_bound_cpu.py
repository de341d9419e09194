"""The error bound the BF16 projection parity test uses (CPU): an emulation of the BF16
pipeline (operands rounded to bf16 by round-to-nearest-even on the upper 16 bits of the FP32
value, FP32-exact products, FP64 sums, coefficients rounded to bf16 again) stays within it,
and uses a visible fraction of it (the bound is not vacuous)."""
import numpy as np

import oracle
from tests.systems_small import small
from tests.test_gpu_parity import _bf16_x0_bound


def _bf16(x):
    a = np.asarray(x, dtype=np.float32).copy()
    b = a.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = ((b + 0x7FFF + lsb) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_pipeline_within_bound():
    s = small()
    rng = np.random.default_rng(18)
    u = rng.standard_normal(s.N_d)
    for om in (0.0203, 0.69, 8.8):
        psi32 = s.psi.astype(np.float32)
        A = _bf16(psi32)
        B = _bf16(psi32 * u.astype(np.float32))
        G = (A @ B.T).astype(np.float32).astype(np.float64)
        d = s.eps[:, None] - s.eps[None, :] - 1j * om
        Cc = -s.dV * G / d
        x0 = (A.T @ _bf16(Cc.real.astype(np.float32))).T + 1j * (
            A.T @ _bf16(Cc.imag.astype(np.float32))).T
        ref = oracle.galerkin(s, om, u)
        bre, bim = _bf16_x0_bound(s, om, u)
        assert np.all(np.abs(x0.real - ref.real) <= bre + 1e-12)
        assert np.all(np.abs(x0.imag - ref.imag) <= bim + 1e-12)
        # the bound is not vacuous: the observed error uses a visible part of it
        assert np.max(np.abs(x0 - ref)) > 1e-3 * np.max(np.hypot(bre, bim))
