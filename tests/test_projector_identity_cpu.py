"""The two identities the fused COCG iteration uses to keep the projector term out of the
stencil kernels (CPU, numpy, on the seeded systems' projectors):

  p^T V_nl p = sum_{g,l} cp_{g,l}^2 / (gamma_{g,l} dV),   cp = gamma dV chi^T p,
  chi_g^T (V_nl p) = sum_h S_{g,h} cp_h,   S_{g,h}(l, m) = sum over common points of chi_{g,l} chi_{h,m},

with V_nl = sum_{g,l} gamma_{g,l} dV chi_{g,l} chi_{g,l}^T, for complex p and the unconjugated
(complex-symmetric) products of COCG.  The overlap blocks are formed here the way the
library forms them, point by point over pairs of groups sharing the point, and compared with
the dense products.
"""
import numpy as np

from tests.systems_small import small


def _dense_projectors(s):
    rows, gam = [], []
    for g in s.groups:
        for l in range(g.chi.shape[0]):
            v = np.zeros(s.N_d)
            v[np.asarray(g.idx)] = g.chi[l]
            rows.append(v)
            gam.append(g.gamma[l])
    return np.array(rows), np.array(gam)


def test_projector_dot_and_overlap_identities():
    s = small()
    dV = s.dV
    X, gam = _dense_projectors(s)  # (nproj, N_d)
    rng = np.random.default_rng(3)
    p = rng.standard_normal(s.N_d) + 1j * rng.standard_normal(s.N_d)
    vnl = X.T @ (gam * dV * (X @ p))
    cp = gam * dV * (X @ p)
    # p^T V_nl p from the coefficients
    lhs = p @ vnl
    rhs = np.sum(cp * cp / (gam * dV))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # chi^T V_nl p = S cp with S built point by point over group pairs
    nproj = [g.chi.shape[0] for g in s.groups]
    off = np.concatenate([[0], np.cumsum(nproj)])
    at = {}
    for gi, g in enumerate(s.groups):
        for k, q in enumerate(np.asarray(g.idx)):
            at.setdefault(int(q), []).append((gi, k))
    S = np.zeros((off[-1], off[-1]))
    for q, ents in at.items():
        for g1, k1 in ents:
            for g2, k2 in ents:
                c1 = s.groups[g1].chi[:, k1]
                c2 = s.groups[g2].chi[:, k2]
                S[off[g1]:off[g1 + 1], off[g2]:off[g2 + 1]] += np.outer(c1, c2)
    assert np.allclose(S, X @ X.T, rtol=1e-12, atol=1e-12 * np.abs(S).max())
    assert np.allclose(X @ vnl, S @ cp, rtol=1e-10, atol=1e-12 * np.abs(X @ vnl).max())
    # and so chi^T r_{k+1} = chi^T rhat - alpha S cp for r_{k+1} = rhat - alpha V_nl p
    rhat = rng.standard_normal(s.N_d) + 1j * rng.standard_normal(s.N_d)
    alpha = 0.37 - 0.21j
    r1 = rhat - alpha * vnl
    assert np.allclose(X @ r1, X @ rhat - alpha * (S @ cp), rtol=1e-10,
                       atol=1e-12 * np.abs(X @ r1).max())
