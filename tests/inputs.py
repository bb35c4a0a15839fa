"""Seeded synthetic inputs shared by the oracle and the CUDA path in tests.

This module holds no step of the method: it only draws positions,
velocities and mesh vectors from numpy's seeded generator, with the
shapes and value ranges of the manufactured-solution workloads.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def particles(n_particles: int, seed: int, v_mean=0.2, v_sigma=1.0, clustered_cells: int = 0, n: int = 8):
    """Positions uniform in [0,1)^3 (or packed into ``clustered_cells`` cells of
    an n^3 mesh, to make crowded cells), Gaussian velocities. Returns
    (x[N,3], v[N,3]) in pid order."""
    g = rng(seed)
    if clustered_cells:
        h = 1.0 / n
        corners = g.integers(0, n, size=(clustered_cells, 3)) * h
        which = g.integers(0, clustered_cells, size=n_particles)
        x = corners[which] + g.random((n_particles, 3)) * h
        x = np.minimum(x, np.nextafter(1.0, 0.0))
    else:
        x = g.random((n_particles, 3))
    v = v_mean + v_sigma * g.standard_normal((n_particles, 3))
    return x, v


def mesh_vector(n: int, seed: int, zero_mean: bool = True) -> np.ndarray:
    g = rng(seed)
    b = g.standard_normal(n ** 3)
    if zero_mean:
        b -= b.mean()
    return b
