"""Exact target on tiny grids: dense sum-over-states response (Eq. 2) and f(A) by eigh.

TEST INFRASTRUCTURE ONLY.  This is the second, independent half of the oracle: it never
calls Lanczos, COCG or the mode-product square root.  It diagonalises the full discrete
Hamiltonian, builds chi0 from all occupied/unoccupied pairs (Eq. 2 with occupations 1/0 and
the spin factor 2, written for l2-normalised eigenvectors), forms
A = nu^{1/2} chi0 nu^{1/2} with the square root taken from a dense eigen-decomposition of the
discrete Laplacian, and returns e_j^T f(A) e_j exactly (Eqs. 5-8).

The Hamiltonian matrix is supplied by the caller (``H`` argument), so that the test can build
it independently of the C oracle's matrix-free apply.
"""
from __future__ import annotations

import numpy as np


def fval(x, fkind=0):
    if fkind == 1:
        return x
    if fkind == 2:
        return x * x
    return np.log1p(-x) + x


def dense_laplacian(n, h, bc, weights):
    """Kronecker-sum Laplacian from central weights (w_0..w_R) on a (nx, ny, nz) grid."""
    mats = []
    R = len(weights) - 1
    for a in range(3):
        L = np.zeros((n[a], n[a]))
        for i in range(n[a]):
            L[i, i] += weights[0]
            for m in range(1, R + 1):
                for j in (i + m, i - m):
                    if bc[a] == 0:
                        L[i, j % n[a]] += weights[m]
                    elif 0 <= j < n[a]:
                        L[i, j] += weights[m]
        mats.append(L / (h[a] * h[a]))
    Ix, Iy, Iz = np.eye(n[0]), np.eye(n[1]), np.eye(n[2])
    return (np.kron(Iz, np.kron(Iy, mats[0])) + np.kron(Iz, np.kron(mats[1], Ix))
            + np.kron(mats[2], np.kron(Iy, Ix)))


def nu_half_dense(lap):
    """Symmetric PSD square root of nu = -4 pi lap^+ (zero on the null space)."""
    lam, U = np.linalg.eigh(lap)
    neg = -lam
    thr = 1e-10 * np.abs(lam).max()
    s = np.where(neg > thr, np.sqrt(4.0 * np.pi / np.where(neg > thr, neg, 1.0)), 0.0)
    return (U * s[None, :]) @ U.T


def chi0_dense(H, ns, dV, omega):
    """Matrix of r = chi0 u on grid vectors (the dV-weighted kernel of Eq. 2)."""
    eps, phi = np.linalg.eigh(H)                 # l2-normalised eigenvectors
    occ, uno = phi[:, :ns], phi[:, ns:]
    K = np.zeros_like(H)
    for n in range(ns):
        de = eps[n] - eps[ns:]
        wgt = de / (de * de + omega * omega)     # 4 Re 1/(eps_n - eps_m - i w) / 4
        M = occ[:, n][:, None] * uno              # (psi_n psi_m)(r) for each m
        K += (M * wgt[None, :]) @ M.T
    return (4.0 / dV) * K, eps


def exact_diagonal(H, lap, ns, dV, omega, fkind=0):
    """Exact d_j = [f(A)]_jj for all j, Tr f(A), and spec(A)."""
    K, eps = chi0_dense(H, ns, dV, omega)
    S = nu_half_dense(lap)
    A = S @ K @ S
    A = 0.5 * (A + A.T)
    lam, V = np.linalg.eigh(A)
    d = (V * V) @ fval(lam, fkind)
    return d, float(np.sum(fval(lam, fkind))), lam, A, K, eps
