"""Test infrastructure: closed-form free-space potentials (Delta phi = f,
phi ~ -(int f)/(4 pi |x|), the sign convention of Sec. 1) for the test
charges.  Used only by the tests and the benchmark's error report.
"""
from __future__ import annotations

import numpy as np


def bump_potential_radial(rho: np.ndarray, a: float, A: float) -> np.ndarray:
    """Potential of f = A (1 - rho^2)^4 (rho = r/a < 1).  Derived by integrating
    the radial Poisson equation term by term; total charge
    4 pi a^3 A * 128/3465 gives the exterior monopole."""
    rho = np.asarray(rho, dtype=np.float64)
    inner = a * a * A * (rho ** 2 / 6 - rho ** 4 / 5 + rho ** 6 / 7 - rho ** 8 / 18 + rho ** 10 / 110 - 0.1)
    outer = -(128.0 / 3465.0) * a * a * A / np.maximum(rho, 1e-300)
    return np.where(rho < 1.0, inner, outer)


def bumps_potential(N: int, bumps, nodes: int | None = None) -> np.ndarray:
    """Superposed exact potential of a bump sum at the nodes g h, g in [0,nodes)^3."""
    nodes = N if nodes is None else nodes
    x = np.arange(nodes, dtype=np.float64) / N
    phi = np.zeros((nodes,) * 3)
    for c, a, A in zip(bumps.centres, bumps.radii, bumps.amplitudes):
        r = np.sqrt((x[:, None, None] - c[0]) ** 2 + (x[None, :, None] - c[1]) ** 2
                    + (x[None, None, :] - c[2]) ** 2)
        phi += bump_potential_radial(r / a, a, A)
    return phi


def smooth_charge(r: np.ndarray) -> np.ndarray:
    """Sec. 7.1 smooth charge (r - r^2)^4 on r < 1 (r scaled by R_o)."""
    return np.where(r < 1.0, (r - r * r) ** 4, 0.0)


def smooth_potential(r: np.ndarray, Ro: float) -> np.ndarray:
    """Sec. 7.1 exact potential of the smooth charge (scaled radius r = |x - x_o|/R_o)."""
    inner = Ro * Ro * (r ** 6 / 42 - r ** 7 / 14 + r ** 8 / 12 - 2 * r ** 9 / 45 + r ** 10 / 110 - 1.0 / 1260)
    outer = -Ro * Ro / (2310.0 * np.maximum(r, 1e-300))
    return np.where(r < 1.0, inner, outer)
