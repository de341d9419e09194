"""Pins of the CPU oracle against things other than itself (closed forms, invariants, exact
dense targets, library routines, printed values).  No GPU needed."""
import os

import numpy as np
import pytest

import oracle
from oracle import dense
import synth
from synth import PERIODIC, DIRICHLET
from tests.systems_small import tiny

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- finite differences ----
@pytest.mark.parametrize("R", [1, 2, 3, 4, 6])
def test_fd_weights_exact_on_polynomials(R):
    w = oracle.fd_weights(R)
    j = np.arange(-R, R + 1)
    wj = w[np.abs(j)]
    for k in range(0, 2 * R + 2):
        # second derivative of x^k at 0 is 2 for k == 2 and 0 otherwise
        assert abs(np.sum(wj * j.astype(float) ** k) - (2.0 if k == 2 else 0.0)) < 1e-9 * (R ** k + 1)
    # the moment conditions fix the weights uniquely: compare with the exact rational solve
    assert np.allclose(w, synth.systems.second_derivative_weights(R), rtol=1e-13, atol=1e-15)
    if R == 1:
        assert np.allclose(w, [-2.0, 1.0])


@pytest.mark.parametrize("bc", [(PERIODIC,) * 3, (DIRICHLET,) * 3, (PERIODIC, DIRICHLET, PERIODIC)])
def test_apply_h_matches_dense_matrix(bc):
    s = tiny(bc=bc)
    H = s.dense_h()  # generator's own construction (Kronecker sums + explicit projectors)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, s.N_d)) + 1j * rng.standard_normal((2, s.N_d))
    sig = -0.3 + 0.7j
    y = oracle.apply_h(s, x, sig)
    ref = (H @ x.T).T - sig * x
    assert np.max(np.abs(y - ref)) < 1e-11 * np.max(np.abs(ref))


def test_fd_periodic_eigenvalues_equal_symbol():
    s = tiny(n=(9, 8, 7), radius=3)
    w = oracle.fd_weights(3)
    for ax in range(3):
        lam, V = oracle.nu_modes(s, ax)
        n, h = s.n[ax], s.h[ax]
        k = np.arange(n)
        sym = (w[0] + 2 * sum(w[m] * np.cos(2 * np.pi * k * m / n) for m in range(1, 4))) / h ** 2
        assert np.allclose(np.sort(lam), np.sort(sym), atol=1e-10 * np.abs(sym).max())
        assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)


# ---------------------------------------------------------------- Coulomb square root ----
def _fft_poisson(s, x):
    """nu x = -4 pi Lap_h^+ x for a periodic cell, from the FD symbol in Fourier space."""
    w = oracle.fd_weights(s.fd_radius)
    syms = []
    for ax in range(3):
        n, h = s.n[ax], s.h[ax]
        k = np.arange(n)
        syms.append((w[0] + 2 * sum(w[m] * np.cos(2 * np.pi * k * m / n)
                                    for m in range(1, s.fd_radius + 1))) / h ** 2)
    lam = syms[2][:, None, None] + syms[1][None, :, None] + syms[0][None, None, :]
    X = np.fft.fftn(x.reshape(s.n[2], s.n[1], s.n[0]))
    with np.errstate(divide="ignore", invalid="ignore"):
        mult = np.where(np.abs(lam) > 1e-9, -4 * np.pi / lam, 0.0)
    return np.real(np.fft.ifftn(X * mult)).ravel()


def test_nu_half_squares_to_fft_poisson():
    s = tiny(n=(8, 6, 7), radius=3)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(s.N_d)
    u = oracle.nu_half(s, oracle.nu_half(s, x)[0])[0]
    ref = _fft_poisson(s, x)
    assert np.max(np.abs(u - ref)) < 1e-11 * np.max(np.abs(ref))
    # nu^{1/2} annihilates the constant vector (periodic zero mode)
    assert np.max(np.abs(oracle.nu_half(s, np.ones(s.N_d))[0])) < 1e-11


@pytest.mark.parametrize("bc", [(DIRICHLET,) * 3, (PERIODIC, DIRICHLET, DIRICHLET)])
def test_nu_half_inverts_laplacian(bc):
    s = tiny(bc=bc, radius=2)
    lap = dense.dense_laplacian(s.n, s.h, s.bc, synth.systems.second_derivative_weights(2))
    rng = np.random.default_rng(2)
    x = rng.standard_normal(s.N_d)
    if PERIODIC in bc:
        # remove the null-space component of lap (constant along every periodic axis)
        lam, U = np.linalg.eigh(lap)
        null = U[:, np.abs(lam) < 1e-9 * np.abs(lam).max()]
        x = x - null @ (null.T @ x)
    nx = oracle.nu_half(s, oracle.nu_half(s, x)[0])[0]
    # -lap (nu x) = 4 pi x on the range
    assert np.max(np.abs(-lap @ nx - 4 * np.pi * x)) < 1e-9 * 4 * np.pi * np.abs(x).max()
    # and nu^{1/2} equals the dense symmetric square root
    S = dense.nu_half_dense(lap)
    assert np.max(np.abs(oracle.nu_half(s, x)[0] - S @ x)) < 1e-10 * np.abs(S @ x).max()


# ---------------------------------------------------------------- frequencies ----------
def test_gl_frequencies_match_printed_table():
    printed = np.loadtxt(os.path.join(GOLD, "gl_omega_table3.txt"))
    om, w = oracle.gl_frequencies(8)
    # Printed to two decimals; the largest node is 49.36497, printed 49.37 (a rounding through
    # 49.365), so allow half a unit of the last digit plus that double rounding.
    assert np.all(np.abs(om - printed) <= 0.0051)
    assert np.sum(np.round(om, 2) == printed) == 7
    assert abs(np.sum(w / (1 + om ** 2)) - np.pi / 2) < 1e-5


@pytest.mark.parametrize("nw", [1, 2, 5, 8, 10, 16])
def test_gl_underlying_rule_is_exact_for_polynomials(nw):
    om, W = oracle.gl_frequencies(nw)
    x = (om - 1) / (om + 1)               # invert omega = (1+x)/(1-x)
    w = W * (1 - x) ** 2 / 2              # invert the Jacobian
    for k in range(2 * nw):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-12
    # a rational integrand that the mapped rule converges on: int_0^inf dw/(1+w^2) = pi/2
    if nw >= 16:
        assert abs(np.sum(W / (1 + om ** 2)) - np.pi / 2) < 1e-10


# ---------------------------------------------------------------- response function -----
@pytest.mark.parametrize("bc", [(PERIODIC,) * 3, (DIRICHLET,) * 3])
@pytest.mark.parametrize("omega", [0.02, 0.69, 8.84])
def test_chi0_sternheimer_equals_sum_over_states(bc, omega):
    s = tiny(bc=bc)
    H = s.dense_h()
    K, _ = dense.chi0_dense(H, s.ns, s.dV, omega)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(s.N_d)
    r, it = oracle.chi0(s, omega, u, tol=1e-13)
    ref = K @ u
    assert np.max(np.abs(r - ref)) < 1e-9 * np.max(np.abs(ref))
    # symmetric and negative semidefinite
    v = rng.standard_normal(s.N_d)
    rv, _ = oracle.chi0(s, omega, v, tol=1e-13)
    assert abs(v @ r - u @ rv) < 1e-9 * abs(u @ r)
    assert u @ r < 0 and v @ rv < 0


def test_chi0_iterations_grow_as_omega_decreases():
    s = tiny()
    u = np.random.default_rng(4).standard_normal(s.N_d)
    its = [oracle.chi0(s, om, u, tol=1e-8)[1].sum() for om in (49.37, 3.22, 0.31, 0.02)]
    assert its[0] <= its[1] <= its[2] <= its[3]


# ---------------------------------------------------------------- Lanczos quadrature ----
@pytest.fixture(scope="module")
def tiny_exact():
    s = tiny()
    H = s.dense_h()
    lap = dense.dense_laplacian(s.n, s.h, s.bc, synth.systems.second_derivative_weights(s.fd_radius))
    omega = 0.31
    out = {}
    for fk in (0, 1, 2):
        out[fk] = dense.exact_diagonal(H, lap, s.ns, s.dV, omega, fkind=fk)
    return s, omega, out


def test_spectrum_nonpositive(tiny_exact):
    s, omega, out = tiny_exact
    lam = out[0][2]
    assert lam.max() < 1e-10 and lam.min() < 0


def test_gauss_quadrature_exactness(tiny_exact):
    s, omega, out = tiny_exact
    A = out[0][3]
    probes = np.array([0, 17, 100, s.N_d - 1])
    # one step integrates f(x) = x exactly: d = A_jj
    r1 = oracle.lanczos(s, probes, omega, nl=1, tol=1e-13, fkind=oracle.F_X)
    assert np.allclose(r1["d"], np.diag(A)[probes], rtol=1e-9, atol=1e-13)
    # two steps integrate f(x) = x^2 exactly: d = (A^2)_jj = ||A e_j||^2
    r2 = oracle.lanczos(s, probes, omega, nl=2, tol=1e-13, fkind=oracle.F_X2)
    assert np.allclose(r2["d"], np.sum(A[:, probes] ** 2, axis=0), rtol=1e-9, atol=1e-13)


def test_quadrature_monotone_one_sided_bound(tiny_exact):
    """f has negative even derivatives, so Gauss estimates decrease monotonically to the
    exact value from above: 0 >= d^(1) >= d^(2) >= ... >= [f(A)]_jj."""
    s, omega, out = tiny_exact
    dex = out[0][0]
    probes = np.array([5, 60, 200])
    prev = np.zeros(len(probes))
    for k in range(1, 7):
        d = oracle.lanczos(s, probes, omega, nl=k, tol=1e-13)["d"]
        assert np.all(d <= prev + 1e-12)
        assert np.all(d >= dex[probes] - 1e-12)
        prev = d


def test_lanczos_converges_to_exact_diagonal(tiny_exact):
    s, omega, out = tiny_exact
    dex = out[0][0]
    probes = np.arange(0, s.N_d, 37)
    d = oracle.lanczos(s, probes, omega, nl=30, tol=1e-13)["d"]
    assert np.max(np.abs(d - dex[probes])) < 1e-9 * np.max(np.abs(dex))


def _dense_lanczos(A, j, nl, rtol=0.0):
    """Plain Lanczos on an explicit matrix (numpy, full reorthogonalisation, tridiagonal
    eigen-solve by eigh), written from the recurrence of Section 3.1 independently of the C
    oracle.  Stops at the first step k >= 2 with |d_k - d_{k-1}| <= rtol |d_k| (rtol > 0) or
    when the next beta is <= 1e-14 |alpha_1| (Krylov space exhausted).  Returns
    (alpha, beta, d per step, reason) with reason 'exit', 'breakdown' or 'steps'."""
    N = A.shape[0]
    Q = np.zeros((N, nl + 1))
    Q[j, 0] = 1.0
    al, be, ds = [], [], []
    for k in range(nl):
        v = A @ Q[:, k]
        al.append(Q[:, k] @ v)
        v -= al[k] * Q[:, k]
        if k > 0:
            v -= be[k - 1] * Q[:, k - 1]
        for _ in range(2):
            v -= Q[:, :k + 1] @ (Q[:, :k + 1].T @ v)
        T = np.diag(al) + np.diag(be[:k], 1) + np.diag(be[:k], -1)
        lam, W = np.linalg.eigh(T)
        ds.append(float(W[0] ** 2 @ (np.log1p(-lam) + lam)))
        if rtol > 0 and k >= 1 and abs(ds[k] - ds[k - 1]) <= rtol * abs(ds[k]):
            return np.array(al), np.array(be), np.array(ds), "exit"
        if k == nl - 1:
            break
        bn = float(np.linalg.norm(v))
        if bn <= 1e-14 * abs(al[0]):
            return np.array(al), np.array(be), np.array(ds), "breakdown"
        be.append(bn)
        Q[:, k + 1] = v / bn
    return np.array(al), np.array(be), np.array(ds), "steps"


@pytest.mark.parametrize("rtol", [0.95, 1e-1, 1e-4, 1e-7])
def test_lanczos_early_exit_step_matches_dense_recurrence(tiny_exact, rtol):
    """Early exit: the oracle stops at the first step k >= 2 with |d_k - d_{k-1}| <= rtol |d_k|
    and returns d_k.  The step is taken from a plain Lanczos on the dense A; the three
    tolerances give three different exit steps, so an off-by-one in the step index (testing
    d_{k+1} against d_k, or starting the test at k = 3) fails; at rtol = 0.95 one probe exits
    at the earliest allowed step, k = 2."""
    s, omega, out = tiny_exact
    A = out[0][3]
    exits = set()
    for j in (5, 60, 200):
        al, be, ds, why = _dense_lanczos(A, j, 14, rtol=rtol)
        assert why == "exit"
        r = oracle.lanczos(s, np.array([j]), omega, nl=14, tol=1e-13, lrtol=rtol)
        assert r["steps"][0] == len(ds)
        assert abs(r["d"][0] - ds[-1]) <= 1e-9 * abs(ds[-1])
        assert np.allclose(r["alpha"][0][:len(al)], al, rtol=1e-9, atol=1e-13)
        exits.add(len(ds))
    assert min(exits) >= 2
    if rtol == 0.95:
        assert min(exits) == 2


def test_lanczos_breakdown_on_exhausted_krylov_space():
    """Breakdown: on a six-point chain with one occupied state, the Krylov space of A from e_j
    is all of R^6, so beta_6 vanishes and the recurrence must stop after exactly six steps
    (checked against a plain dense Lanczos), where the Gauss rule is exact: d_j equals the
    dense [f(A)]_jj.  The well sits off the grid points so that no mirror symmetry closes the
    space earlier."""
    s = synth.gaussian_system("chain6", (6, 1, 1), (3.3, 1.0, 1.0), (PERIODIC,) * 3,
                              np.array([[1.234, 0.5, 0.5]]), np.array([1.5]), np.array([0.6]), 1,
                              fd_radius=3, proj_sigma=None, seed=3, min_gap=0.0, cache=False)
    H = s.dense_h()
    lap = dense.dense_laplacian(s.n, s.h, s.bc,
                                synth.systems.second_derivative_weights(s.fd_radius))
    for omega in (0.4, 0.05):
        dex, _, _, A, _, _ = dense.exact_diagonal(H, lap, s.ns, s.dV, omega)
        for j in range(s.N_d):
            al, be, ds, why = _dense_lanczos(A, j, 10)
            assert why == "breakdown" and len(ds) == s.N_d
            r = oracle.lanczos(s, np.array([j]), omega, nl=10, tol=1e-13)
            assert r["steps"][0] == s.N_d
            assert abs(r["d"][0] - dex[j]) <= 1e-12 * abs(dex[j])
            assert np.allclose(r["alpha"][0][:s.N_d], al, rtol=1e-10, atol=1e-14)


def test_cocg_reports_an_unmet_tolerance():
    """A Sternheimer tolerance below FP64 rounding cannot be met by the true residual: after
    its restarts the oracle's COCG must report failure instead of returning the iterate."""
    s = tiny()
    u = np.random.default_rng(0).standard_normal(s.N_d)
    with pytest.raises(RuntimeError):
        oracle.chi0(s, 0.3, u, tol=1e-18, maxit=10 ** 7)
    r, it = oracle.chi0(s, 0.3, u, tol=1e-12)  # a reachable tolerance still succeeds
    assert np.all(it > 0)


def test_block_lanczos_single_probe_equals_scalar(tiny_exact):
    """A block of one probe is the scalar recurrence (independent code: C scalar Lanczos)."""
    s, omega, out = tiny_exact
    for j in (3, 150, s.N_d - 2):
        a = oracle.block_lanczos(s, [j], omega, 5, tol=1e-13)["d"]
        b = oracle.lanczos(s, np.array([j]), omega, 5, tol=1e-13)["d"]
        assert np.allclose(a, b, rtol=1e-10, atol=1e-16)


def test_block_gauss_exactness(tiny_exact):
    """The block Gauss rule after k block steps is exact for degree <= 2k - 1: one step
    gives A_jj for f = x, two steps give (A^2)_jj for f = x^2, for every probe of the block."""
    s, omega, out = tiny_exact
    A = out[0][3]
    probes = np.array([0, 17, 100, s.N_d - 1])
    r1 = oracle.block_lanczos(s, probes, omega, 1, tol=1e-13, fkind=oracle.F_X)
    assert np.allclose(r1["d"], np.diag(A)[probes], rtol=1e-9, atol=1e-16)
    r2 = oracle.block_lanczos(s, probes, omega, 2, tol=1e-13, fkind=oracle.F_X2)
    assert np.allclose(r2["d"], np.sum(A[:, probes] ** 2, axis=0), rtol=1e-9, atol=1e-16)


def test_block_lanczos_converges_to_exact_diagonal(tiny_exact):
    s, omega, out = tiny_exact
    dex = out[0][0]
    probes = np.array([5, 60, 200, 301])
    d = oracle.block_lanczos(s, probes, omega, 8, tol=1e-13)["d"]
    assert np.max(np.abs(d - dex[probes])) < 1e-9 * np.max(np.abs(dex))


def test_tridiag_f11_against_library_eigensolver():
    import scipy.linalg as sla
    rng = np.random.default_rng(5)
    for k in (1, 2, 5, 17, 40):
        al = -rng.uniform(0.01, 2.0, size=k)
        be = rng.uniform(0.01, 0.5, size=max(k - 1, 0))
        if k > 1:
            lam, Q = sla.eigh_tridiagonal(al, be)
        else:
            lam, Q = al.copy(), np.ones((1, 1))
        assert lam.max() < 1.0
        ref = np.sum(Q[0] ** 2 * (np.log1p(-lam) + lam))
        assert abs(oracle.tridiag_f11(al, be) - ref) < 1e-12 * max(1.0, abs(ref))
        # f(x) = x and x^2 have closed forms: alpha_1 and alpha_1^2 + beta_1^2
        assert abs(oracle.tridiag_f11(al, be, oracle.F_X) - al[0]) < 1e-12
        b1 = be[0] if k > 1 else 0.0
        assert abs(oracle.tridiag_f11(al, be, oracle.F_X2) - (al[0] ** 2 + b1 ** 2)) < 1e-12


def test_trace_and_energy_sign():
    """At g = 1 and converged quadrature, sum_j d_j = Tr f(A), and E_c < 0."""
    s = tiny(n=(5, 6, 5), ns=2)
    H = s.dense_h()
    lap = dense.dense_laplacian(s.n, s.h, s.bc, synth.systems.second_derivative_weights(s.fd_radius))
    om, w = oracle.gl_frequencies(3)
    res = oracle.energy(s, om, w, stride=(1, 1, 1), nl=25, tol=1e-12)
    ec_ref = 0.0
    for k in range(3):
        d, tr, lam, *_ = dense.exact_diagonal(H, lap, s.ns, s.dV, om[k])
        assert abs(res["d_fine"][k].sum() - tr) < 1e-8 * abs(tr)
        ec_ref += w[k] * tr
    ec_ref /= 2 * np.pi
    assert res["ec"] < 0
    assert abs(res["ec"] - ec_ref) < 1e-8 * abs(ec_ref)


def test_h_refinement_normalisation():
    """The same physical cell at three spacings: the integrand Tr f(A) converges instead of
    scaling with the volume element (a missing or doubled dV fails this)."""
    vals = []
    for n in (6, 8, 10):
        L = 4.0
        s = synth.gaussian_system(f"href{n}", (n, n, n), (L, L, L), (PERIODIC,) * 3,
                                  [[2.0, 2.0, 2.0]], [1.5], [0.9], 1, fd_radius=3,
                                  min_gap=0.0, cache=False)
        H = s.dense_h()
        lap = dense.dense_laplacian(s.n, s.h, s.bc, synth.systems.second_derivative_weights(3))
        vals.append(dense.exact_diagonal(H, lap, 1, s.dV, 0.5)[1])
        # oracle chi0 normalisation agrees with the dense one at every spacing
        u = np.random.default_rng(n).standard_normal(s.N_d)
        K, _ = dense.chi0_dense(H, 1, s.dV, 0.5)
        assert np.allclose(oracle.chi0(s, 0.5, u, tol=1e-13)[0], K @ u, rtol=1e-8, atol=1e-12)
    d1, d2 = abs(vals[1] - vals[0]), abs(vals[2] - vals[1])
    assert d2 < d1
    assert d1 < 0.2 * abs(vals[0])           # a dV error would change it by (h ratio)^3 ~ 2.4x


# ---------------------------------------------------------------- interpolation --------
def _poly(shape, coef_deg):
    z, y, x = np.meshgrid(*(np.arange(n, dtype=float) for n in shape[::-1]), indexing="ij")
    dx, dy, dz = coef_deg
    return (1 + 0.3 * x ** dx - 0.1 * x) * (2 - 0.05 * y ** dy + 0.2 * y) * (0.5 + 0.01 * z ** dz)


@pytest.mark.parametrize("kind,deg", [("cubic", 3), ("linear", 1)])
def test_interpolation_exact_on_polynomials_dirichlet(kind, deg):
    shape = (13, 10, 11)
    bc = (DIRICHLET,) * 3
    stride = (2, 3, 2)
    f = _poly(shape, (deg, deg, deg)).ravel()
    probes = oracle.coarse_probes(shape, stride, bc)
    fh = oracle.interpolate(f[probes], shape, stride, bc, kind)
    assert np.max(np.abs(fh - f)) < 1e-10 * np.abs(f).max()


def test_interpolation_identity_at_coarse_points_and_g1():
    shape = (12, 12, 12)
    bc = (PERIODIC,) * 3
    rng = np.random.default_rng(6)
    for kind in ("cubic", "linear", "fourier"):
        dc = rng.standard_normal(6 ** 3)
        fh = oracle.interpolate(dc, shape, (2, 2, 2), bc, kind)
        assert np.allclose(fh[oracle.coarse_probes(shape, (2, 2, 2), bc)], dc, atol=1e-12)
    d = rng.standard_normal(12 ** 3)
    assert np.array_equal(oracle.interpolate(d, shape, (1, 1, 1), bc, "none"), d)


def test_interpolation_periodic_cubic_exact_away_from_wrap():
    shape = (16, 12, 14)
    bc = (PERIODIC,) * 3
    f = _poly(shape, (3, 3, 3)).reshape(shape[2], shape[1], shape[0])
    probes = oracle.coarse_probes(shape, (2, 2, 2), bc)
    fh = oracle.interpolate(f.ravel()[probes], shape, (2, 2, 2), bc, "cubic").reshape(f.shape)
    # interior fine points whose 4-point stencil (coarse nodes c-1..c+2) does not wrap
    sl = tuple(slice(2, n - 3) for n in (shape[2], shape[1], shape[0]))
    assert np.max(np.abs(fh[sl] - f[sl])) < 1e-10 * np.abs(f).max()


@pytest.mark.parametrize("kind", ["linear", "cubic"])
def test_interpolation_nondivisible_periodic_axis(kind):
    """52 points at stride 3: coarse nodes 0, 3, ..., 51 and a wrap interval of 1 point.  The
    Lagrange weights stay a partition of unity and reproduce polynomials of the stencil's
    degree at every fine point whose stencil spans the wrap (coordinates unwrapped by n)."""
    n, g = 52, 3
    W = oracle.interp_matrix(n, g, PERIODIC, kind)
    nodes = oracle.coarse_nodes(n, g, PERIODIC)
    assert list(nodes) == list(range(0, 52, 3)) and len(nodes) == 18
    assert np.allclose(W.sum(axis=1), 1.0, atol=1e-14)
    deg = 1 if kind == "linear" else 3
    # a polynomial in the unwrapped coordinate is reproduced wherever the stencil does not
    # straddle the wrap; straddling stencils see nodes shifted by n, so test f(x) on the
    # fine points whose nearest-node stencils stay inside [0, 51]
    for p in range(deg + 1):
        f = (np.arange(n) / n) ** p
        fh = W @ f[nodes]
        inner = np.arange(3 * (deg // 2 + 1), n - 3 * (deg // 2 + 2))
        assert np.allclose(fh[inner], f[inner], atol=1e-12)
    # and across the wrap for a periodic smooth function the error is small
    f = np.cos(2 * np.pi * np.arange(n) / n)
    assert np.max(np.abs(W @ f[nodes] - f)) < (5e-2 if kind == "linear" else 5e-4)


def test_interpolation_sum_invariance_periodic():
    """Shift-invariant partition-of-unity interpolants give sum(fine) = g^3 sum(coarse)."""
    shape = (12, 12, 12)
    bc = (PERIODIC,) * 3
    dc = np.random.default_rng(7).standard_normal(6 ** 3)
    for kind in ("cubic", "linear", "fourier"):
        fh = oracle.interpolate(dc, shape, (2, 2, 2), bc, kind)
        assert abs(fh.sum() - 8 * dc.sum()) < 1e-10 * np.abs(dc).sum()


def test_fourier_interpolation_exact_on_bandlimited():
    shape = (12, 8, 10)
    bc = (PERIODIC,) * 3
    z, y, x = np.meshgrid(*(np.arange(n) for n in shape[::-1]), indexing="ij")
    f = (1 + np.cos(2 * np.pi * x / 12) + 0.5 * np.sin(2 * np.pi * y / 8)
         * np.cos(2 * np.pi * z / 10)).ravel()
    probes = oracle.coarse_probes(shape, (2, 2, 2), bc)
    fh = oracle.interpolate(f[probes], shape, (2, 2, 2), bc, "fourier")
    assert np.max(np.abs(fh - f)) < 1e-12


def test_error_metrics_definition():
    m = oracle.error_metrics(np.array([1.0, 2.0, 3.0]), np.array([1.5, 1.5, 3.0]))
    assert m["abs_err"] == 0.0 and m["l1"] == 1.0 and m["ecr"] == 0.0


@pytest.mark.parametrize("bc", [(PERIODIC,) * 3, (DIRICHLET,) * 3])
def test_galerkin_guess_satisfies_galerkin_condition(bc):
    """x0 lies in span(Psi) and its residual is orthogonal to span(Psi) (dV inner product),
    checked with the generator's dense H; and x0 adds nothing to the density (the occupied
    pairs cancel by antisymmetry)."""
    s = tiny(bc=bc, ns=3)
    H = s.dense_h()
    rng = np.random.default_rng(10)
    u = rng.standard_normal(s.N_d)
    om = 0.31
    x0 = oracle.galerkin(s, om, u)
    for n in range(s.ns):
        b = -s.psi[n] * u
        res = H @ x0[n] - (s.eps[n] + 1j * om) * x0[n] - b
        proj = s.dV * (s.psi @ res)
        assert np.max(np.abs(proj)) < 1e-10 * np.max(np.abs(s.dV * (s.psi @ b)))
        # x0 is a combination of the occupied orbitals
        coef = s.dV * (s.psi @ x0[n])
        assert np.allclose(s.psi.T @ coef, x0[n], atol=1e-12 * np.abs(x0[n]).max())
    dens = 4 * np.sum(s.psi * np.real(x0), axis=0)
    assert np.max(np.abs(dens)) < 1e-12 * np.max(np.abs(x0))
