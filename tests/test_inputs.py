"""The synthetic inputs meet what the method assumes of a ground state (CPU): the occupied
orbitals are orthonormal in the dV inner product and are eigenvectors of the discrete H to
the precision the unprojected Sternheimer equations rely on, with a gap above the last
occupied level; the Si-like cells carry the recipe's atom and state counts."""
import numpy as np
import pytest

import oracle
import synth
from tests.systems_small import small, tiny


def _check_ground_state(s, resid_tol):
    G = s.dV * (s.psi @ s.psi.T)
    assert np.allclose(G, np.eye(s.ns), atol=1e-9)
    # residuals with the oracle's matrix-free H (independent of the generator's FFT kinetic
    # term and sparse/dense assembly)
    R = oracle.apply_h(s, s.psi.astype(np.complex128)) - s.eps[:, None] * s.psi
    rel = np.sqrt(s.dV * np.sum(np.abs(R) ** 2, axis=1))
    assert rel.max() < resid_tol, rel.max()
    assert np.all(np.diff(s.eps) >= -1e-12)


@pytest.mark.parametrize("make", [lambda: tiny(), lambda: small(),
                                  lambda: small(bc=(synth.DIRICHLET,) * 3, n=(11, 10, 12),
                                                L=(5.5, 5.0, 6.0), seed=7)])
def test_small_ground_states(make):
    _check_ground_state(make(), 1e-9)


def test_toy_and_si8_ground_states():
    for name in ("toy", "si8"):
        s = synth.named_system(name)
        _check_ground_state(s, 1e-8)
        assert s.gap > 0.01


def test_si8_recipe():
    s = synth.named_system("si8")
    assert s.n == (26, 26, 26) and s.natom == 8 and s.ns == 16
    assert len(s.groups) >= 8  # s and p projector groups on every atom
