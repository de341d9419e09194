"""Oracle for the Lanczos-quadrature RPA correlation energy (CPU, FP64).

TEST INFRASTRUCTURE ONLY.  A plain, slow, obviously-correct restatement of the method of
"Highly Parallel Real-Space Random Phase Approximation Using Lanczos Quadrature and
Interpolation" used to check the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the CUDA
library and never imports it.

Pieces:
  * ``oracle.c`` (compiled by :func:`build`): H apply, nu^{1/2} by 1-D mode products, the
    Sternheimer/COCG solves with Galerkin initial guess, Lanczos quadrature per probe,
    tridiagonal f(T)_{11}, Gauss-Legendre frequencies.
  * this module: ctypes marshalling, coarse-grid selection and interpolation (Section 3.2),
    the frequency/probe driver of Algorithm 1, the error metrics of Section 5.2, and the
    block Lanczos quadrature (numpy block recurrence over the C oracle's operator).
  * ``dense.py``: the exact target on tiny grids from the sum-over-states response (Eq. 2).

Parity status of each function (what pins it) is listed in the test-suite
(``tests/test_oracle_pins.py``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()

PERIODIC, DIRICHLET = 0, 1
F_LOG, F_X, F_X2 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liborc.so`` (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    so = os.path.join(_BUILD, "liborc.so")
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-D_GNU_SOURCE", "-o", tmp, src, "-lm"])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.orc_fd_weights.argtypes = [C.c_int, P]
            lib.orc_apply_h_batch.argtypes = [P, C.c_int, P, C.c_double, C.c_double, P]
            lib.orc_nu_half.argtypes = [P, C.c_int, P, P]
            lib.orc_nu_modes.argtypes = [P, C.c_int, P, P]
            lib.orc_chi0.argtypes = [P, C.c_double, P, C.c_double, C.c_int, C.c_int, P, P]
            lib.orc_chi0.restype = C.c_int
            lib.orc_lanczos_batch.argtypes = [P, P, C.c_int, P, P, P, P, P, P, P]
            lib.orc_lanczos_batch.restype = C.c_int
            lib.orc_tridiag_f11.argtypes = [C.c_int, P, P, C.c_int]
            lib.orc_tridiag_f11.restype = C.c_double
            lib.orc_gl_frequencies.argtypes = [C.c_int, P, P]
            lib.orc_jacobi_eig.argtypes = [C.c_int, P, P, P]
            lib.orc_galerkin.argtypes = [P, C.c_double, P, P]
            _LIB = lib
    return _LIB


class _Sys(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double * 3), ("bc", C.c_int * 3),
                ("radius", C.c_int), ("vloc", C.c_void_p), ("nproj", C.c_int),
                ("proj_off", C.c_void_p), ("proj_idx", C.c_void_p), ("proj_val", C.c_void_p),
                ("proj_gamma", C.c_void_p), ("ns", C.c_int), ("psi", C.c_void_p),
                ("eps", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("nl", C.c_int), ("lrtol", C.c_double), ("tol", C.c_double),
                ("maxit", C.c_int), ("reorth", C.c_int), ("fkind", C.c_int),
                ("nthreads", C.c_int)]


def _p(a):
    return C.c_void_p(a.ctypes.data)


class OracleSystem:
    """Holds contiguous FP64 copies of a system's arrays and the C descriptor over them."""

    def __init__(self, s, psi=None, eps=None):
        self.s = s
        self.vloc = np.ascontiguousarray(s.vloc, dtype=np.float64)
        offs, idx, val, gam = [0], [], [], []
        for g in s.groups:
            for l in range(g.chi.shape[0]):
                idx.append(np.asarray(g.idx, dtype=np.int32))
                val.append(np.asarray(g.chi[l], dtype=np.float64))
                gam.append(float(g.gamma[l]))
                offs.append(offs[-1] + len(g.idx))
        self.proj_off = np.asarray(offs, dtype=np.int32)
        self.proj_idx = np.ascontiguousarray(np.concatenate(idx) if idx else np.zeros(1, np.int32))
        self.proj_val = np.ascontiguousarray(np.concatenate(val) if val else np.zeros(1))
        self.proj_gamma = np.asarray(gam if gam else [0.0], dtype=np.float64)
        psi = s.psi if psi is None else psi
        eps = s.eps if eps is None else eps
        self.psi = np.ascontiguousarray(psi, dtype=np.float64)
        self.eps = np.ascontiguousarray(eps, dtype=np.float64)
        c = _Sys()
        c.n[:] = list(s.n)
        c.h[:] = list(s.h)
        c.bc[:] = list(s.bc)
        c.radius = s.fd_radius
        c.vloc = self.vloc.ctypes.data
        c.nproj = len(gam)
        c.proj_off = self.proj_off.ctypes.data
        c.proj_idx = self.proj_idx.ctypes.data
        c.proj_val = self.proj_val.ctypes.data
        c.proj_gamma = self.proj_gamma.ctypes.data
        c.ns = self.psi.shape[0]
        c.psi = self.psi.ctypes.data
        c.eps = self.eps.ctypes.data
        self.c = c
        self.N = s.N_d

    @property
    def ref(self):
        return C.byref(self.c)


def _osys(s):
    return s if isinstance(s, OracleSystem) else OracleSystem(s)


# ---------------------------------------------------------------------------------------
# step functions
# ---------------------------------------------------------------------------------------
def fd_weights(radius: int) -> np.ndarray:
    w = np.zeros(radius + 1)
    _lib().orc_fd_weights(radius, _p(w))
    return w


def apply_h(s, x: np.ndarray, sigma: complex = 0.0) -> np.ndarray:
    """(H - sigma) x for complex x of shape (count, N_d) or (N_d,)."""
    o = _osys(s)
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.complex128)
    y = np.empty_like(x)
    _lib().orc_apply_h_batch(o.ref, x.shape[0], _p(x), float(np.real(sigma)),
                             float(np.imag(sigma)), _p(y))
    return y


def nu_half(s, q: np.ndarray) -> np.ndarray:
    """nu^{1/2} q for real q of shape (count, N_d) or (N_d,)."""
    o = _osys(s)
    q = np.ascontiguousarray(np.atleast_2d(q), dtype=np.float64)
    u = np.empty_like(q)
    _lib().orc_nu_half(o.ref, q.shape[0], _p(q), _p(u))
    return u


def nu_modes(s, axis: int):
    o = _osys(s)
    n = s.n[axis]
    V = np.empty((n, n))
    lam = np.empty(n)
    _lib().orc_nu_modes(o.ref, axis, _p(V), _p(lam))
    return lam, V


def chi0(s, omega: float, u: np.ndarray, tol=1e-12, maxit=5000, nthreads=0, psi=None,
         eps=None):
    """chi0(i omega) u via the N_s Sternheimer solves; returns (r, iterations per state)."""
    o = OracleSystem(s, psi, eps) if (psi is not None or eps is not None) else _osys(s)
    u = np.ascontiguousarray(u, dtype=np.float64)
    r = np.empty_like(u)
    it = np.zeros(o.psi.shape[0], dtype=np.int32)
    st = _lib().orc_chi0(o.ref, float(omega), _p(u), float(tol), int(maxit), int(nthreads),
                         _p(r), _p(it))
    if st != 0:
        raise RuntimeError("oracle COCG did not converge")
    return r, it


def galerkin(s, omega: float, u: np.ndarray) -> np.ndarray:
    """Galerkin initial guesses x0 (ns x N_d complex) of the Sternheimer systems for one u."""
    o = _osys(s)
    u = np.ascontiguousarray(u, dtype=np.float64)
    x0 = np.empty((o.psi.shape[0], s.N_d), dtype=np.complex128)
    _lib().orc_galerkin(o.ref, float(omega), _p(u), _p(x0))
    return x0


def tridiag_f11(alpha, beta, fkind=F_LOG) -> float:
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(np.concatenate([beta, [0.0]]) if len(beta) else np.zeros(1),
                             dtype=np.float64)
    return _lib().orc_tridiag_f11(len(a), _p(a), _p(b), int(fkind))


def jacobi_eig(a: np.ndarray):
    a = np.array(a, dtype=np.float64, copy=True)
    n = a.shape[0]
    lam = np.empty(n)
    V = np.empty((n, n))
    _lib().orc_jacobi_eig(n, _p(a), _p(lam), _p(V))
    return lam, V


def gl_frequencies(nw: int):
    """Mapped Gauss-Legendre nodes/weights on [0, inf) (Eq. 9)."""
    om = np.empty(nw)
    w = np.empty(nw)
    _lib().orc_gl_frequencies(nw, _p(om), _p(w))
    return om, w


def lanczos(s, probes, omegas, nl, tol=1e-10, maxit=5000, lrtol=0.0, reorth=1, fkind=F_LOG,
            nthreads=0):
    """Lanczos quadrature d_j(i omega) for each (probe grid index, omega) pair.

    Returns dict(d, steps, alpha, beta, cocg_iters)."""
    o = _osys(s)
    probes = np.ascontiguousarray(probes, dtype=np.int64)
    omegas = np.ascontiguousarray(np.broadcast_to(omegas, probes.shape), dtype=np.float64)
    cnt = len(probes)
    d = np.zeros(cnt)
    steps = np.zeros(cnt, dtype=np.int32)
    al = np.zeros((cnt, nl))
    be = np.zeros((cnt, nl))
    ci = np.zeros(cnt, dtype=np.int64)
    op = _Opts(nl=int(nl), lrtol=float(lrtol), tol=float(tol), maxit=int(maxit),
               reorth=int(reorth), fkind=int(fkind), nthreads=int(nthreads))
    st = _lib().orc_lanczos_batch(o.ref, C.byref(op), cnt, _p(probes), _p(omegas), _p(d),
                                  _p(steps), _p(al), _p(be), _p(ci))
    if st != 0:
        raise RuntimeError("oracle Lanczos: a Sternheimer solve hit maxit")
    return dict(d=d, steps=steps, alpha=al, beta=be, cocg_iters=ci)


def _fval(x, fkind):
    if fkind == F_X:
        return x
    if fkind == F_X2:
        return x * x
    return np.log1p(-x) + x


def block_lanczos(s, probes, omega, nl, tol=1e-10, maxit=5000, fkind=F_LOG, nthreads=0):
    """Block Lanczos quadrature for one frequency: the b probes share one block Krylov
    recurrence started from Q_1 = [e_j1 ... e_jb] (the block variant of the Lanczos
    quadrature of Section 3.1 that Section 6 names as future work).  After k block steps,
    d_ji = [E_1^T f(T_k) E_1]_ii with the block tridiagonal T_k (diagonal blocks
    A_m = Q_m^T A Q_m, sub-diagonal blocks B_m from the QR factorisation of the next block):
    a block Gauss rule, exact for f of degree <= 2k - 1.  As in the scalar oracle the new
    block is reorthogonalised against every previous block by two classical Gram-Schmidt
    passes; its QR factorisation is Cholesky QR applied twice.  Stops early (fewer steps) when
    a pivot of the factorisation falls below 1e-14 |A_1|.  Returns dict(d, steps)."""
    probes = np.ascontiguousarray(probes, dtype=np.int64)
    b = len(probes)
    N = s.N_d
    Q = np.zeros((N, b))
    Q[probes, np.arange(b)] = 1.0
    blocks = [Q]
    A_blk, B_blk = [], []
    steps = 0
    scale = None
    for k in range(nl):
        U = nu_half(s, Q.T)                                            # b x N
        Rr = np.stack([chi0(s, omega, U[i], tol=tol, maxit=maxit, nthreads=nthreads)[0]
                       for i in range(b)])
        V = nu_half(s, Rr).T                                           # N x b
        Ak = Q.T @ V
        A_blk.append(0.5 * (Ak + Ak.T))
        if scale is None:
            scale = np.max(np.abs(A_blk[0]))
        steps = k + 1
        if k == nl - 1:
            break
        Qall = np.hstack(blocks)
        for _ in range(2):
            V = V - Qall @ (Qall.T @ V)
        # Cholesky QR, twice: V = Q_{k+1} R2 R1
        Rs = []
        ok = True
        for _ in range(2):
            G = V.T @ V
            try:
                L = np.linalg.cholesky(0.5 * (G + G.T))
            except np.linalg.LinAlgError:
                ok = False
                break
            Rm = L.T
            if np.min(np.abs(np.diag(Rm))) <= 1e-14 * scale:
                ok = False
                break
            V = np.linalg.solve(Rm.T, V.T).T                           # V R^-1
            Rs.append(Rm)
        if not ok:
            break
        B_blk.append(Rs[1] @ Rs[0])
        Q = V
        blocks.append(Q)
    T = np.zeros((steps * b, steps * b))
    for k in range(steps):
        T[k * b:(k + 1) * b, k * b:(k + 1) * b] = A_blk[k]
        if k + 1 < steps:
            T[(k + 1) * b:(k + 2) * b, k * b:(k + 1) * b] = B_blk[k]
            T[k * b:(k + 1) * b, (k + 1) * b:(k + 2) * b] = B_blk[k].T
    lam, W = np.linalg.eigh(T)
    d = (W[:b, :] ** 2) @ _fval(lam, fkind)
    return dict(d=d, steps=steps)


# ---------------------------------------------------------------------------------------
# coarse grid C_g and interpolation I_g (Section 3.2)
# ---------------------------------------------------------------------------------------
def coarse_nodes(n: int, g: int, bc: int) -> np.ndarray:
    """Sampled fine indices along one axis: 0, g, 2g, ... (plus n-1 on a Dirichlet axis)."""
    nodes = list(range(0, n, g))
    if bc == DIRICHLET and nodes[-1] != n - 1:
        nodes.append(n - 1)
    return np.asarray(nodes, dtype=np.int64)


def coarse_probes(shape, stride, bc) -> np.ndarray:
    """Flat fine-grid indices of the coarse points, x fastest over coarse nodes."""
    cx, cy, cz = (coarse_nodes(shape[a], stride[a], bc[a]) for a in range(3))
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    return (X + shape[0] * (Y + shape[1] * Z)).ravel()


def _lagrange(xs, t):
    w = np.ones(len(xs))
    for a in range(len(xs)):
        for b in range(len(xs)):
            if a != b:
                w[a] *= (t - xs[b]) / (xs[a] - xs[b])
    return w


def interp_matrix(n: int, g: int, bc: int, kind: str) -> np.ndarray:
    """Fine x coarse matrix W of one axis: fine = W @ coarse (Lagrange, local stencil)."""
    nodes = coarse_nodes(n, g, bc)
    m = len(nodes)
    W = np.zeros((n, m))
    npts = {"linear": 2, "cubic": 4}[kind]
    if m == 1:
        W[:, 0] = 1.0
        return W
    for i in range(n):
        if bc == PERIODIC:
            c = int(np.searchsorted(nodes, i, side="right")) - 1   # nodes[c] <= i
            if npts > m:
                raise ValueError("periodic interpolation needs at least as many coarse nodes as stencil points")
            first = c - (npts // 2 - 1)
            ids = [first + t for t in range(npts)]
            xs = [nodes[k % m] + n * (k // m) for k in ids]
            cols = [k % m for k in ids]
        else:
            c = int(np.searchsorted(nodes, i, side="right")) - 1
            c = min(c, m - 2)
            k = min(npts, m)
            first = min(max(c - (k // 2 - 1), 0), m - k)
            cols = list(range(first, first + k))
            xs = [nodes[q] for q in cols]
        w = _lagrange(np.asarray(xs, dtype=float), float(i))
        for col, wv in zip(cols, w):
            W[i, col] += wv
    return W


def interpolate(dc: np.ndarray, shape, stride, bc, kind: str) -> np.ndarray:
    """Coarse values (flat, x fastest) -> fine values (flat), I_g of Section 3.2.

    kind: 'none' (stride 1 only), 'linear' (trilinear), 'cubic' (tricubic 4-point Lagrange),
    'fourier' (zero-padded spectrum, periodic axes with n divisible by g)."""
    cn = [len(coarse_nodes(shape[a], stride[a], bc[a])) for a in range(3)]
    D = np.asarray(dc, dtype=np.float64).reshape(cn[2], cn[1], cn[0])
    if kind == "none":
        if tuple(stride) != (1, 1, 1):
            raise ValueError("no interpolation needs stride 1")
        return D.ravel().copy()
    if kind == "fourier":
        return _fourier(D, shape, stride, bc).ravel()
    Wx, Wy, Wz = (interp_matrix(shape[a], stride[a], bc[a], kind) for a in range(3))
    F = np.einsum("ia,jb,kc,cba->kji", Wx, Wy, Wz, D)
    return F.ravel()


def _fourier(D, shape, stride, bc):
    if any(b != PERIODIC for b in bc) or any(shape[a] % stride[a] for a in range(3)):
        raise ValueError("Fourier interpolation needs periodic axes with n divisible by g")
    F = D
    for ax_np, ax in ((2, 0), (1, 1), (0, 2)):
        m = F.shape[ax_np]
        n = shape[ax]
        if m == n:
            continue
        S = np.fft.fft(F, axis=ax_np)
        Sm = np.moveaxis(S, ax_np, 0)
        out = np.zeros((n,) + Sm.shape[1:], dtype=complex)
        h = m // 2
        if m % 2 == 1:
            out[: h + 1] = Sm[: h + 1]
            out[n - h:] = Sm[h + 1:]
        else:
            out[:h] = Sm[:h]
            out[n - h + 1:] = Sm[h + 1:]
            out[h] = 0.5 * Sm[h]          # Nyquist split equally between +m/2 and -m/2
            out[n - h] = 0.5 * Sm[h]
        F = np.real(np.moveaxis(np.fft.ifft(out, axis=0), 0, ax_np)) * (n / m)
    return F


def error_metrics(d_ref: np.ndarray, d_hat: np.ndarray):
    """|Delta E|, L1 and error-cancellation ratio of Section 5.2."""
    dd = np.asarray(d_ref) - np.asarray(d_hat)
    s = abs(float(dd.sum()))
    l1 = float(np.abs(dd).sum())
    return dict(abs_err=s, l1=l1, ecr=(s / l1 if l1 > 0 else 0.0))


# ---------------------------------------------------------------------------------------
# Algorithm 1 driver
# ---------------------------------------------------------------------------------------
def energy(s, omegas, weights, stride=(1, 1, 1), nl=20, tol=1e-10, maxit=5000, lrtol=0.0,
           reorth=1, interp="cubic", nthreads=0):
    """E_c = 1/(2 pi) sum_k w_k sum_j d^_j(i omega_k) with d^ = I_g(d on C_g) (Section 3.2).

    Returns dict(ec, d_coarse (nw x P), d_fine (nw x N_d), probes, cocg_iters, steps)."""
    o = _osys(s)
    probes = coarse_probes(s.n, stride, s.bc)
    nw = len(omegas)
    dco = np.zeros((nw, len(probes)))
    dfi = np.zeros((nw, s.N_d))
    iters = np.zeros((nw, len(probes)), dtype=np.int64)
    steps = np.zeros((nw, len(probes)), dtype=np.int32)
    ec = 0.0
    for k in range(nw):
        r = lanczos(o, probes, np.full(len(probes), omegas[k]), nl, tol=tol, maxit=maxit,
                    lrtol=lrtol, reorth=reorth, nthreads=nthreads)
        dco[k] = r["d"]
        iters[k] = r["cocg_iters"]
        steps[k] = r["steps"]
        kind = "none" if tuple(stride) == (1, 1, 1) else interp
        dfi[k] = interpolate(dco[k], s.n, stride, s.bc, kind)
        ec += weights[k] * dfi[k].sum()
    ec /= 2.0 * np.pi
    return dict(ec=ec, d_coarse=dco, d_fine=dfi, probes=probes, cocg_iters=iters, steps=steps)
