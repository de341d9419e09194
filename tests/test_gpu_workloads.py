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
