"""Parity on the full-size workload grids (GPU).

* Uneven batch: Si-like cells of 8, 16 and 32 atoms (26^3, 26x26x52, 26x52x52, periodic)
  and a 12-atom Gaussian cluster (40^3, zero-Dirichlet walls) in one rpa_batch_energy call,
  with per-probe Lanczos early exit at 1e-6 relative change, autotuned tiling and CUDA-graph
  replay: the batch equals the separate runs, and a sampled Lanczos density of every system
  equals the oracle's.
* Interpolation sweep on the 64-atom grid (52^3): strides 1, 2 and 3 (3 does not divide 52,
  so the wrap interval is shorter and the Lagrange weights non-uniform), each operator
  against the oracle on the full fine grid.

Tolerances: FP64 form with Sternheimer tol 1e-10 on both sides; d_j within 1e-9 absolute
(the per-point bound stated for the FP64 form).  Interpolation is a fixed linear map:
1e-12 relative.
"""
import numpy as np
import pytest

import oracle
import paper_2609_16408_gb300 as R
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    R.load()


C4 = ("si8", "si16", "si32", "cluster12")
_SYS = {}


def system(name):
    if name not in _SYS:
        _SYS[name] = synth.named_system(name)
    return _SYS[name]


def c4_context(s, **kw):
    om, w = oracle.gl_frequencies(2)
    # two coarse points per axis keeps the full E_c of each system to a few dozen probes
    stride = tuple(max(1, n // 2) for n in s.n)
    opts = dict(precision="fp64", lanczos_max=6, lanczos_rtol=1e-6, stern_tol=1e-10,
                stern_maxit=8000, stride=stride, interp="linear")
    opts.update(kw)
    return R.Context.from_system(s, om, w, **opts), om, w


def test_uneven_batch_matches_separate_runs():
    ctxs, refs = [], []
    for name in C4:
        s = system(name)
        c, om, _ = c4_context(s)
        P = R.rpa_num_probes(c.ctx)
        _, _, ec, st = R.rpa_energy_density(c.ctx, len(om), P, s.N_d, want_fine=False)
        assert ec < 0 and st["probe_points"] == P * len(om)
        ctxs.append(c)
        refs.append(ec)
    ec, stats = R.rpa_batch_energy([c.ctx for c in ctxs])
    assert np.allclose(ec, refs, rtol=1e-9, atol=0)
    # early exit retired some probes before the step cap
    assert any(st["lanczos_steps_max"] <= 6 for st in stats)


@pytest.mark.parametrize("name", C4)
def test_sampled_density_vs_oracle(name):
    s = system(name)
    nl = 2
    c, om, _ = c4_context(s, lanczos_max=nl, lanczos_rtol=0.0)
    rng = np.random.default_rng(C4.index(name) + 40)
    probe = np.array([int(rng.integers(s.N_d))], dtype=np.int64)
    freq = np.array([1], dtype=np.int32)
    out = R.rpa_probe_density(c.ctx, probe, freq, nl=nl)
    ref = oracle.lanczos(s, probe, om[freq], nl, tol=1e-10, maxit=8000)
    assert np.max(np.abs(out["d"] - ref["d"])) <= 1e-9


def test_si64_bench_path_vs_oracle():
    """The headline workload through the path the benchmark times: the 64-atom Si-like cell
    (52^3 grid, 128 states), mixed form at Sternheimer tol 1e-4 with FP64 refinement (the
    double-float refinement residual), two probe-points in one wave (256 systems: launches
    over more than 32 systems use the bulk tiling, the tail the tail tiling, chunks replay
    from CUDA graphs, small launches split z), autotuned tiling; and the FP64 form at tol
    1e-10.  Probe-points at the smallest frequency node and at a middle one, two Lanczos
    steps each, against the oracle at tol 1e-10.

    Tolerances: FP64 form 1e-9 per point (the per-point bound of the FP64 form).  Mixed form
    5e-4 relative per point: if every density erred by the same relative amount in the same
    direction, E_c would err by that amount times |E_c|, and with |E_c| ~ 0.2 Ha/atom (the
    paper's silicon values) 5e-4 keeps that worst case at the 0.1 mHa/atom the mixed form is
    held to."""
    s = system("si64")
    om, w = oracle.gl_frequencies(10)
    probes_c = oracle.coarse_probes(s.n, (2, 2, 2), s.bc)
    rng = np.random.default_rng(64)
    probes = np.asarray(probes_c[rng.choice(len(probes_c), 2, replace=False)], dtype=np.int64)
    freqs = np.array([9, 4], dtype=np.int32)  # the smallest node and a middle one
    ref = oracle.lanczos(s, probes, om[freqs], 2, tol=1e-10, maxit=20000)
    c = R.Context.from_system(s, om, w, precision="fp64", lanczos_max=2, stern_tol=1e-10,
                              stern_maxit=20000, stride=(2, 2, 2))
    out = R.rpa_probe_density(c.ctx, probes, freqs, nl=2, want_tridiag=True)
    assert np.max(np.abs(out["d"] - ref["d"])) <= 1e-9
    assert np.allclose(out["alpha"], ref["alpha"], rtol=1e-8, atol=1e-12)
    c.close()
    c = R.Context.from_system(s, om, w, precision="mixed", lanczos_max=2, stern_tol=1e-4,
                              stern_maxit=20000, stride=(2, 2, 2), refine=4)
    out = R.rpa_probe_density(c.ctx, probes, freqs, nl=2)
    st = out["stats"]
    assert st["solves"] == 2 * 2 * s.ns and st["nonconv_solves"] == 0
    assert np.all(np.abs(out["d"] - ref["d"]) <= 5e-4 * np.abs(ref["d"]))
    c.close()


@pytest.mark.parametrize("tile", [-113, -126, -6])
def test_band_tiling_si8_mixed(tile):
    """Full-row tilings of the mixed form on the full Si8 grid (26^3, 16 states): two bands
    of 13 rows (halo rows from the neighbouring band and across the periodic wrap), one band
    of the whole plane (halo rows wrap onto the band itself), and the two-point kernel on
    packed full rows (19 rows of 13 pairs per tile, a ragged last tile of 7 rows whose halo
    wraps onto the first tile); chi0 u against the oracle."""
    s = system("si8")
    om, w = oracle.gl_frequencies(2)
    c = R.Context.from_system(s, om, w, precision="mixed", stern_tol=1e-10, refine=4,
                              stern_maxit=20000, tile=tile)
    rng = np.random.default_rng(31)
    u = rng.standard_normal((1, s.N_d))
    r, _ = R.rpa_chi0(c.ctx, np.array([0.4]), u, s.ns)
    ref, _ = oracle.chi0(s, 0.4, u[0], tol=1e-12, maxit=20000)
    assert np.max(np.abs(r[0] - ref)) <= 1e-7 * np.max(np.abs(ref))
    c.close()


def test_lih4_density_vs_oracle():
    """Second workload of the paper's scaling runs: a LiH-like rock-salt cell (16^3, 8
    states), two Lanczos steps, no interpolation (stride 1); FP64 form at tol 1e-10 within
    1e-9 per point, and the mixed form within its own solve tolerance."""
    s = system("lih4")
    om, w = oracle.gl_frequencies(8)
    probes = np.array([0, 1234, 4095], dtype=np.int64)
    freqs = np.array([7, 3, 0], dtype=np.int32)
    ref = oracle.lanczos(s, probes, om[freqs], 2, tol=1e-10, maxit=20000)
    c = R.Context.from_system(s, om, w, precision="fp64", lanczos_max=2, stern_tol=1e-10,
                              stride=(1, 1, 1), interp="none")
    out = R.rpa_probe_density(c.ctx, probes, freqs, nl=2, want_tridiag=True)
    assert np.max(np.abs(out["d"] - ref["d"])) <= 1e-9
    assert np.allclose(out["alpha"], ref["alpha"], rtol=1e-8, atol=1e-12)
    c.close()
    c = R.Context.from_system(s, om, w, precision="mixed", lanczos_max=2, stern_tol=1e-8,
                              stride=(1, 1, 1), interp="none")
    out = R.rpa_probe_density(c.ctx, probes, freqs, nl=2)
    assert np.all(np.abs(out["d"] - ref["d"]) <= 1e-6 * np.abs(ref["d"]) + 1e-12)
    c.close()


@pytest.mark.parametrize("g", [1, 2, 3])
@pytest.mark.parametrize("kind", ["linear", "cubic", "fourier"])
def test_interpolation_si64_grid(g, kind):
    if g == 1 and kind != "cubic":
        pytest.skip("stride 1 is the identity for every operator")
    if g == 3 and kind == "fourier":
        pytest.skip("Fourier interpolation needs a stride that divides the periodic axis")
    n, bc = (52, 52, 52), (synth.PERIODIC,) * 3
    c = R.Context(n, (20.52 / 52,) * 3, bc, 6)
    om, w = oracle.gl_frequencies(2)
    R.rpa_set_frequencies(c.ctx, om, w)
    R.rpa_set_options(c.ctx, stride=(g, g, g), interp=kind)
    P = R.rpa_num_probes(c.ctx)
    assert np.array_equal(R.rpa_probe_indices(c.ctx), oracle.coarse_probes(n, (g,) * 3, bc))
    dc = -np.abs(np.random.default_rng(g).standard_normal((2, P)))
    dfi, ec = R.rpa_interpolate(c.ctx, dc, int(np.prod(n)))
    ref = np.stack([oracle.interpolate(dc[k], n, (g,) * 3, bc, kind) for k in range(2)])
    assert np.max(np.abs(dfi - ref)) <= 1e-12 * np.max(np.abs(ref))
    ec_ref = sum(w[k] * ref[k].sum() for k in range(2)) / (2 * np.pi)
    assert abs(ec - ec_ref) <= 1e-12 * abs(ec_ref)
