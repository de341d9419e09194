"""Argument checks of the allocation-free Galerkin entry point's binding (CPU): wrong dtypes,
shapes, layouts or devices raise ValueError before anything reaches the C library, whose
kernels would otherwise read or write past the caller's buffers."""
import numpy as np
import pytest

import paper_2609_16408_gb300 as R

torch = pytest.importorskip("torch")


def _args(ns=4, nd=30, count=2):
    return dict(psi=torch.zeros((ns, nd), dtype=torch.float64),
                eps=torch.zeros(ns, dtype=torch.float64),
                omega=torch.ones(count, dtype=torch.float64),
                u=torch.zeros((count, nd), dtype=torch.float64),
                x0=torch.zeros((count, ns, nd), dtype=torch.complex128))


def _call(a):
    R.rpa_galerkin_noalloc(a["psi"], a["eps"], 0.1, a["omega"], a["u"], a["x0"])


@pytest.mark.parametrize("bad", [
    ("psi", lambda a: a["psi"].float(), "float64"),
    ("x0", lambda a: a["x0"].to(torch.complex64), "complex128"),
    ("eps", lambda a: a["eps"][:3].clone(), "shape"),
    ("omega", lambda a: torch.ones(3, dtype=torch.float64), "shape"),
    ("u", lambda a: torch.zeros((2, 29), dtype=torch.float64), "shape"),
    ("x0", lambda a: torch.zeros((2, 5, 30), dtype=torch.complex128), "shape"),
    ("psi", lambda a: torch.zeros((30, 4), dtype=torch.float64).t(), "contiguous"),
    ("u", lambda a: a["u"].numpy(), "torch tensor"),
])
def test_bad_arguments_raise_before_the_call(bad):
    name, make, msg = bad
    a = _args()
    a[name] = make(a)
    with pytest.raises(ValueError, match=msg):
        _call(a)


def test_host_tensors_are_refused():
    with pytest.raises(ValueError, match="CUDA tensor"):
        _call(_args())
