"""Seeded synthetic inputs shared by the tests, the oracle legs and the bench.

This module holds no arithmetic of the method: it only draws seeded random
numbers and cavity configurations.  Both the CUDA path and the oracle receive
the arrays it returns as plain inputs.
"""

from __future__ import annotations


import numpy as np


def random_populations(grid, q: int, seed: int, spread: float = 0.2, mean: float | None = None):
    """Positive, non-equilibrium populations shaped [q][z][y][x] (float32).

    Each value is ``mean * (1 + spread * U(-1, 1))`` with ``mean = 1/q`` by
    default, so the cell density is near 1 and the velocity small.
    """
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    m = (1.0 / q) if mean is None else mean
    a = m * (1.0 + spread * rng.uniform(-1.0, 1.0, size=(q, nz, ny, nx)))
    return a.astype(np.float32)


def random_thermal_populations(grid, seed: int, amplitude: float = 0.05):
    """D3Q7 populations [7][z][y][x] (float32), uniform in +-amplitude."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    return rng.uniform(-amplitude, amplitude, size=(7, nz, ny, nx)).astype(np.float32)


def random_fields(grid, seed: int, drho: float = 0.01, du: float = 0.01, dtheta: float = 0.2):
    """Macroscopic fields (rho[z,y,x], u[3,z,y,x], theta[z,y,x]) as float32."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    rho = 1.0 + drho * rng.uniform(-1, 1, size=(nz, ny, nx))
    u = du * rng.uniform(-1, 1, size=(3, nz, ny, nx))
    th = dtheta * rng.uniform(-1, 1, size=(nz, ny, nx))
    return rho.astype(np.float32), u.astype(np.float32), th.astype(np.float32)


def ensemble_draws(n: int = 64, seed: int = 1234, edges=(32, 48, 64, 96),
                   log10_ra=(3.0, 6.0), types=(1, 2, 3)):
    """Cavity ensemble: edge uniform over `edges`, log10 Ra uniform, type uniform.

    Returns a list of dicts {"n": edge, "Ra": Ra, "wall": type}.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        edge = int(rng.choice(edges))
        ra = float(10.0 ** rng.uniform(*log10_ra))
        wall = int(rng.choice(types))
        out.append({"n": edge, "Ra": ra, "wall": wall})
    return out


def random_weights(count: int, seed: int, scale: float = 0.3):
    """`count` float32 values uniform in +-scale (network parameters)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=count).astype(np.float32)


def random_targets(shape, seed: int, scale: float = 1.0):
    """float32 normal values of the given shape (training targets)."""
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal(size=shape)).astype(np.float32)


def sample_cells(grid, count: int, seed: int):
    """`count` distinct flat cell indices (x fastest), always including the
    eight corners, for sampled comparisons on large grids."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    cells = nx * ny * nz
    corners = [((z * ny + y) * nx + x) for z in (0, nz - 1) for y in (0, ny - 1) for x in (0, nx - 1)]
    rest = rng.choice(cells, size=min(count, cells), replace=False)
    return np.unique(np.concatenate([np.array(corners, dtype=np.int64), rest.astype(np.int64)]))


__all__ = ["random_populations", "random_thermal_populations", "random_fields",
           "ensemble_draws", "random_weights", "random_targets", "sample_cells"]
