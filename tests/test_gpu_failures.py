"""Failure paths on the GPU, none of which faults, traps or hangs it (every wait in the
library is bounded; failures come back as statuses):

* an unreachable Sternheimer tolerance within stern_maxit -> RPA_ENOCONV, results written;
* refinement rounds used up with the residual still above the tolerance -> RPA_ENOCONV;
* NaN in the occupied orbitals -> RPA_EBREAKDOWN (the COCG scalars and the Lanczos scalars
  are checked for finiteness), no hang;
* a bounded tensor-core wait made to expire (options.debug_expire_waits waits on a barrier
  that nothing arrives on) -> RPA_ETIMEOUT, with the tensor memory freed and the context
  usable afterwards.
"""
import numpy as np
import pytest

import oracle
import paper_2609_16408_gb300 as R
from tests.systems_small import small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    R.load()


_S = {}


def _sys():
    if "s" not in _S:
        _S["s"] = small()
    return _S["s"]


def _ctx(s, **opts):
    om, w = oracle.gl_frequencies(4)
    return R.Context.from_system(s, om, w, **opts), om, w


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_iteration_cap_reports_enoconv_and_writes_results(prec):
    s = _sys()
    c, om, _ = _ctx(s, precision=prec, stern_tol=1e-12, stern_maxit=3, lanczos_max=2)
    probes = np.array([5, 300], dtype=np.int64)
    freqs = np.array([0, 3], dtype=np.int32)
    out = R.rpa_probe_density(c.ctx, probes, freqs, nl=2, allow_nonconv=True)
    assert out["status"] == R.RPA_ENOCONV
    d = np.asarray(out["d"])
    assert np.all(np.isfinite(d))
    with pytest.raises(R.RpaError) as ei:
        R.rpa_probe_density(c.ctx, probes, freqs, nl=2)
    assert ei.value.status == R.RPA_ENOCONV
    # the same context still solves to tolerance with a usable cap
    R.rpa_set_options(c.ctx, precision=prec, stern_tol=1e-8, stern_maxit=20000, lanczos_max=2)
    ok = R.rpa_probe_density(c.ctx, probes, freqs, nl=2)
    assert ok["status"] == R.RPA_OK
    c.close()


def test_refinement_rounds_used_up_report_enoconv():
    """One refinement round cannot take a 1e-3 FP32 inner tolerance to 1e-12: the final
    FP64 check reports it instead of passing the last correction silently."""
    s = _sys()
    c, om, _ = _ctx(s, precision="mixed", stern_tol=1e-12, refine=1, inner_tol=1e-3,
                    stern_maxit=20000)
    u = np.random.default_rng(1).standard_normal((1, s.N_d))
    with pytest.raises(R.RpaError) as ei:
        R.rpa_chi0(c.ctx, np.array([0.3]), u, s.ns)
    assert ei.value.status == R.RPA_ENOCONV
    c.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nan_in_orbitals_reports_breakdown(prec):
    s = _sys()
    c, om, _ = _ctx(s, precision=prec, stern_tol=1e-8, lanczos_max=3)
    psi = np.array(s.psi, copy=True)
    psi[1, 17] = np.nan
    R.rpa_set_occupied(c.ctx, psi, s.eps)
    with pytest.raises(R.RpaError) as ei:
        R.rpa_probe_density(c.ctx, np.array([5, 44], dtype=np.int64),
                            np.array([1, 2], dtype=np.int32), nl=3)
    assert ei.value.status == R.RPA_EBREAKDOWN
    # clean orbitals: the context works again
    R.rpa_set_occupied(c.ctx, s.psi, s.eps)
    out = R.rpa_probe_density(c.ctx, np.array([5], dtype=np.int64), np.array([1], dtype=np.int32),
                              nl=3)
    assert np.all(np.isfinite(out["d"]))
    c.close()


@pytest.mark.parametrize("proj", ["mixed", "mixed_bf16"])
def test_expired_tensor_core_wait_reports_timeout_and_recovers(proj):
    s = _sys()
    c, om, _ = _ctx(s, precision=proj, debug_expire_waits=1, stern_tol=1e-8, lanczos_max=2)
    u = np.random.default_rng(3).standard_normal((2, s.N_d))
    oms = np.array([0.05, 2.0])
    with pytest.raises(R.RpaError) as ei:
        R.rpa_galerkin(c.ctx, oms, u, s.ns)
    assert ei.value.status == R.RPA_ETIMEOUT
    with pytest.raises(R.RpaError) as ei:
        R.rpa_probe_density(c.ctx, np.array([7], dtype=np.int64), np.array([1], dtype=np.int32),
                            nl=2)
    assert ei.value.status == R.RPA_ETIMEOUT
    # the waits are normal again: same context, same kernels, correct results
    R.rpa_set_options(c.ctx, precision=proj, debug_expire_waits=0, stern_tol=1e-8,
                      lanczos_max=2)
    x0 = R.rpa_galerkin(c.ctx, oms, u, s.ns)
    for i in range(2):
        ref = oracle.galerkin(s, oms[i], u[i])
        assert np.max(np.abs(x0[i] - ref)) <= 0.05 * np.max(np.abs(ref))
    out = R.rpa_probe_density(c.ctx, np.array([7], dtype=np.int64), np.array([1], dtype=np.int32),
                              nl=2)
    assert out["status"] == R.RPA_OK and np.all(np.isfinite(out["d"]))
    c.close()
