"""Tiny seeded systems for CPU pins and parity tests (dense ground state, < 1 s each)."""
import numpy as np

import synth
from synth import PERIODIC, DIRICHLET


def tiny(bc=(PERIODIC,) * 3, n=(6, 7, 8), L=(4.2, 4.5, 4.8), radius=3, ns=3, proj=True, seed=11):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.25, 0.75, size=(3, 3)) * np.asarray(L)
    depth = rng.uniform(1.0, 2.0, size=3)
    sigma = rng.uniform(0.7, 1.0, size=3)
    return synth.gaussian_system(
        f"tiny_{''.join(map(str, bc))}_{'x'.join(map(str, n))}_r{radius}_p{int(proj)}", n, L, bc,
        centres, depth, sigma, ns, fd_radius=radius, proj_sigma=(0.6 if proj else None),
        seed=seed, min_gap=0.0, cache=False)


def small(bc=(PERIODIC,) * 3, n=(10, 11, 12), L=(5.0, 5.5, 6.0), radius=6, ns=4, proj=True,
          seed=5, min_gap=0.02):
    """A few thousand points, several kernel tiles with ragged tails in every direction."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, size=(3, 3)) * np.asarray(L)
    depth = rng.uniform(1.2, 1.8, size=3)
    sigma = rng.uniform(0.8, 1.1, size=3)
    return synth.gaussian_system(
        f"small_{''.join(map(str, bc))}_{'x'.join(map(str, n))}_r{radius}_p{int(proj)}", n, L, bc,
        centres, depth, sigma, ns, fd_radius=radius, proj_sigma=(0.7 if proj else None),
        seed=seed, min_gap=min_gap, cache=False)
