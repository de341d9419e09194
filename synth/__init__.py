"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package builds the *inputs* of the RPA correlation-energy method: a finite-difference
grid, a local potential, nonlocal projector groups, and the occupied Kohn-Sham pairs
(psi_n, eps_n) of the resulting Hamiltonian (Eq. 3).  The paper takes these from a DFT
ground state; here they come from seeded Gaussian model potentials and this package's own
eigensolver.  Nothing in here evaluates the response function, the Coulomb square root,
Lanczos quadrature or interpolation, and nothing here is imported by ``oracle/`` or by the
CUDA library: both receive the arrays this package produces.
"""
from .systems import (  # noqa: F401
    PERIODIC, DIRICHLET, System, ProjectorGroup, toy_system, si_like_system,
    cluster_system, gaussian_system, named_system, probe_sample, lih_like_system,
)
