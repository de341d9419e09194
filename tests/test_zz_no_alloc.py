"""rpa_galerkin_noalloc: the Galerkin projection for callers that cannot allocate device
memory (it works in a fixed scratch array inside the library).  Checked against the
allocating entry point rpa_galerkin on two calls in a row, with the FP64 tolerance the
parity tests use.  This file is named to be collected last."""
import numpy as np
import pytest

import paper_2609_16408_gb300 as R
from tests.systems_small import small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    R.load()
    return torch


def test_noalloc_matches_allocating_entry_point_twice(torch_cuda):
    torch = torch_cuda
    s = small()
    c = R.Context.from_system(s, np.array([0.5]), np.array([1.0]), precision="fp64")
    rng = np.random.default_rng(21)
    dev = torch.device("cuda")
    psi = torch.from_numpy(np.ascontiguousarray(s.psi)).to(dev)
    eps = torch.from_numpy(np.ascontiguousarray(s.eps)).to(dev)
    for call in range(2):
        u = rng.standard_normal((3, s.N_d))
        om = np.array([0.0203, 0.69, 8.8]) * (1.0 + 0.1 * call)
        ref = R.rpa_galerkin(c.ctx, om, u, s.ns)
        x0 = torch.zeros((3, s.ns, s.N_d), dtype=torch.complex128, device=dev)
        R.rpa_galerkin_noalloc(psi, eps, s.dV, torch.from_numpy(om).to(dev),
                               torch.from_numpy(u).to(dev), x0)
        torch.cuda.synchronize()
        got = x0.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    c.close()


def test_noalloc_matches_oracle_on_a_stream(torch_cuda):
    """Against the oracle's projection (Section 4) on a system of 40 states -- two state tiles
    of 32, the second ragged -- with the work queued on a non-default stream."""
    import oracle
    torch = torch_cuda
    s = small(ns=40, min_gap=0.0)
    dev = torch.device("cuda")
    psi = torch.from_numpy(np.ascontiguousarray(s.psi)).to(dev)
    eps = torch.from_numpy(np.ascontiguousarray(s.eps)).to(dev)
    rng = np.random.default_rng(22)
    u = rng.standard_normal((2, s.N_d))
    om = np.array([0.05, 1.7])
    x0 = torch.zeros((2, s.ns, s.N_d), dtype=torch.complex128, device=dev)
    ut, omt = torch.from_numpy(u).to(dev), torch.from_numpy(om).to(dev)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    R.rpa_galerkin_noalloc(psi, eps, s.dV, omt, ut, x0, stream=st)
    st.synchronize()
    got = x0.cpu().numpy()
    for i in range(2):
        ref = oracle.galerkin(s, om[i], u[i])
        assert np.max(np.abs(got[i] - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_noalloc_rejects_sizes_beyond_scratch(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda")
    # 1024 states need 1024^2 x 8 bytes of partial sums alone: beyond the 8 MiB scratch;
    # the call is rejected before it reads any buffer
    psi = torch.zeros((1024, 8), dtype=torch.float64, device=dev)
    eps = torch.zeros(1024, dtype=torch.float64, device=dev)
    u = torch.zeros((1, 8), dtype=torch.float64, device=dev)
    om = torch.ones(1, dtype=torch.float64, device=dev)
    x0 = torch.zeros((1, 1024, 8), dtype=torch.complex128, device=dev)
    with pytest.raises(R.RpaError, match="scratch"):
        R.rpa_galerkin_noalloc(psi, eps, 0.1, om, u, x0)
