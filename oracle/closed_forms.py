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


def smooth_potential_grid(N: int, nodes: int | None = None, Ro: float = 0.25, centre=(0.5, 0.5, 0.5)) -> np.ndarray:
    """Sec. 7.1 exact potential at the nodes g h, g in [0, nodes)^3."""
    nodes = N if nodes is None else nodes
    x = np.arange(nodes, dtype=np.float64) / N
    r = np.sqrt((x[:, None, None] - centre[0]) ** 2 + (x[None, :, None] - centre[1]) ** 2
                + (x[None, None, :] - centre[2]) ** 2) / Ro
    return smooth_potential(r, Ro)


# Sec. 7.2: oscillatory charge (1/R_o^3) (r - r^2)^2 sin^2(gamma r / 2) on r < 1,
# gamma = 4 mu pi with mu = 7, three copies of radius R_o = 0.05.
OSC_GAMMA = 28.0 * np.pi
OSC_RADIUS = 0.05
OSC_CENTRES = ((3 / 16, 7 / 16, 13 / 16), (7 / 16, 13 / 16, 3 / 16), (13 / 16, 3 / 16, 7 / 16))


def oscillatory_potential(r: np.ndarray, Ro: float, gamma: float = OSC_GAMMA) -> np.ndarray:
    """Sec. 7.2 exact potential of one oscillatory charge, r = |x - x_o| / R_o.

    Inside, a polynomial in r plus 1/r terms and cos(gamma r), sin(gamma r)
    terms whose 1/r parts cancel as r -> 0 (the value at r = 0 is the limit);
    outside, the monopole whose strength makes value and slope continuous at
    r = 1 for gamma a multiple of 2 pi."""
    r = np.asarray(r, dtype=np.float64)
    g = gamma
    rs = np.where(r > 0.0, r, 1.0)  # the centre takes the r -> 0 limit below
    c, s = np.cos(g * rs), np.sin(g * rs)
    poly = rs ** 6 / 84 - rs ** 5 / 30 + rs ** 4 / 40 + 60 / g ** 6 - 9 / g ** 4 - 1.0 / 120 + 120 / (g ** 6 * rs)
    ccoef = (-120 / (g ** 6 * rs) - 9 / g ** 4 + 300 / g ** 6 + 36 * rs / g ** 4 + rs ** 2 / (2 * g ** 2)
             - 30 * rs ** 2 / g ** 4 - rs ** 3 / g ** 2 + rs ** 4 / (2 * g ** 2))
    scoef = (12 / (g ** 5 * rs) - 360 / (g ** 7 * rs) - 96 / g ** 5 + 120 * rs / g ** 5 - 3 * rs / g ** 3
             + 8 * rs ** 2 / g ** 3 - 5 * rs ** 3 / g ** 3)
    inner = poly + ccoef * c + scoef * s
    inner = np.where(r > 0.0, inner, -1.0 / 120 - 6 / g ** 4)
    outer = (-1.0 / 210 - 12 / g ** 4 + 360 / g ** 6) / rs
    return np.where(r < 1.0, inner, outer) / Ro


def oscillatory_potential_grid(N: int, nodes: int | None = None, Ro: float = OSC_RADIUS,
                               centres=OSC_CENTRES, gamma: float = OSC_GAMMA) -> np.ndarray:
    """Superposed Sec. 7.2 potential of the three charges at the nodes g h, g in [0, nodes)^3."""
    nodes = N if nodes is None else nodes
    x = np.arange(nodes, dtype=np.float64) / N
    phi = np.zeros((nodes,) * 3)
    for c in centres:
        r = np.sqrt((x[:, None, None] - c[0]) ** 2 + (x[None, :, None] - c[1]) ** 2
                    + (x[None, None, :] - c[2]) ** 2) / Ro
        phi += oscillatory_potential(r, Ro, gamma)
    return phi
