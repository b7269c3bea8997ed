"""Seeded synthetic charge densities for the free-space Poisson problem.

This module only draws random parameters and samples a charge density on the
grid; it holds none of the solver's arithmetic.  Both the CUDA path (through
the tests and the benchmark) and the CPU oracle read their inputs from here.

Charge family: sums of radial bumps f(x) = A (1 - (r/a)^2)^4 for r < a, zero
outside, r = |x - c|.  This is the same smooth, compactly supported kind of
charge the paper uses in its numerical tests (Sec. 7.1), with the centre,
radius and amplitude drawn per bump.

Grid convention (shared by every component): the unit cube is sampled at the
nodes x = g h, h = 1/N, g in [0, N)^3.  An array ``f`` of shape (N, N, N) holds
``f[g0, g1, g2]`` at position (g0 h, g1 h, g2 h); axis 2 is contiguous in
memory.  Bump centres are given in the same axis order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Bumps:
    centres: np.ndarray  # (k, 3), axis order (0, 1, 2)
    radii: np.ndarray  # (k,)
    amplitudes: np.ndarray  # (k,)

    @property
    def count(self) -> int:
        return int(self.radii.shape[0])


def draw_bumps(k: int, seed: int, centre_lo: float = 0.25, centre_hi: float = 0.75,
               a_lo: float = 0.08, a_hi: float = 0.2) -> Bumps:
    """Draw k bumps from numpy's default_rng(seed) in the order: centres (k x 3),
    radii (k), amplitudes (k)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(centre_lo, centre_hi, size=(k, 3))
    radii = rng.uniform(a_lo, a_hi, size=k)
    amps = rng.uniform(-1.0, 1.0, size=k)
    return Bumps(centres, radii, amps)


def single_bump(centre=(0.5, 0.5, 0.5), radius: float = 0.35, amplitude: float = 1.0) -> Bumps:
    return Bumps(np.asarray([centre], dtype=np.float64), np.asarray([radius], dtype=np.float64),
                 np.asarray([amplitude], dtype=np.float64))


def sample_bumps(N: int, bumps: Bumps, nodes: int | None = None, dtype=np.float64) -> np.ndarray:
    """Sample the bump sum at the nodes g h, g in [0, nodes)^3 (nodes defaults to N).

    Values are computed in FP64 and cast to ``dtype`` at the end."""
    nodes = N if nodes is None else nodes
    h = 1.0 / N
    x = np.arange(nodes, dtype=np.float64) * h
    f = np.zeros((nodes, nodes, nodes), dtype=np.float64)
    for c, a, A in zip(bumps.centres, bumps.radii, bumps.amplitudes):
        # restrict to the bounding box of the support for speed
        lo = [max(0, int(math.floor((c[d] - a) / h))) for d in range(3)]
        hi = [min(nodes, int(math.ceil((c[d] + a) / h)) + 1) for d in range(3)]
        if any(hi[d] <= lo[d] for d in range(3)):
            continue
        d0 = (x[lo[0]:hi[0]] - c[0])[:, None, None]
        d1 = (x[lo[1]:hi[1]] - c[1])[None, :, None]
        d2 = (x[lo[2]:hi[2]] - c[2])[None, None, :]
        rho2 = (d0 * d0 + d1 * d1 + d2 * d2) / (a * a)
        val = np.where(rho2 < 1.0, A * (1.0 - rho2) ** 4, 0.0)
        f[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] += val
    return f.astype(dtype, copy=False)


def _radial_samples(N: int, nodes: int | None, centre, Ro: float):
    """r = |x - centre| / Ro at the nodes g h, g in [0, nodes)^3."""
    nodes = N if nodes is None else nodes
    x = np.arange(nodes, dtype=np.float64) / N
    return np.sqrt((x[:, None, None] - centre[0]) ** 2 + (x[None, :, None] - centre[1]) ** 2
                   + (x[None, None, :] - centre[2]) ** 2) / Ro


def paper_smooth_charge(N: int, nodes: int | None = None, dtype=np.float64) -> np.ndarray:
    """The smooth test charge of Sec. 7.1: (r - r^2)^4 for r < 1, r = |x - 1/2| / R_o,
    R_o = 1/4 (no random draw)."""
    r = _radial_samples(N, nodes, (0.5, 0.5, 0.5), 0.25)
    return np.where(r < 1.0, (r - r * r) ** 4, 0.0).astype(dtype, copy=False)


PAPER_OSC_CENTRES = ((3 / 16, 7 / 16, 13 / 16), (7 / 16, 13 / 16, 3 / 16), (13 / 16, 3 / 16, 7 / 16))


def paper_oscillatory_charge(N: int, nodes: int | None = None, dtype=np.float64) -> np.ndarray:
    """The oscillatory test charge of Sec. 7.2: three copies of
    (1/R_o^3) (r - r^2)^2 sin^2(gamma r / 2), r < 1, with R_o = 0.05,
    gamma = 4 mu pi, mu = 7, at the three centres the paper gives."""
    Ro, gamma = 0.05, 28.0 * math.pi
    f = 0.0
    for c in PAPER_OSC_CENTRES:
        r = _radial_samples(N, nodes, c, Ro)
        f = f + np.where(r < 1.0, (r - r * r) ** 2 * np.sin(0.5 * gamma * r) ** 2, 0.0) / Ro ** 3
    return np.asarray(f).astype(dtype, copy=False)


# ---------------------------------------------------------------------------
# Named workloads.  Each is (solver sizes, charge recipe).  The solver sizes
# follow the problem statement: N nodes per axis, patch side n, support s
# (the local field box is the patch grown by s), coarsening C = 4, P Legendre
# orders, Q the Mehrstellen order (4 -> 19-point, 6 -> 27-point).
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    n: int
    s: int
    Q: int
    P: int = 4
    C: int = 4
    bumps: Bumps = field(default=None, repr=False)
    charge_dtype: str = "f64"
    charge_kind: str = "bumps"  # or "paper_smooth" (Sec. 7.1 charge, no random draw)

    def charge(self, nodes: int | None = None) -> np.ndarray:
        dt = np.float32 if self.charge_dtype == "f32" else np.float64
        if self.charge_kind == "paper_smooth":
            return paper_smooth_charge(self.N, nodes=nodes, dtype=dt)
        return sample_bumps(self.N, self.bumps, nodes=nodes, dtype=dt)


def workload(name: str) -> Workload:
    """The named synthetic workloads.

    single_bump_32: 32^3, 64 patches of 8^3, support 8, Q=4; one bump a=0.35 at the centre.
    bumps8_128:     128^3, 512 patches of 16^3, support 16, Q=4; 8 bumps from seed 1.
    bumps32_256_q6: 256^3, 4096 patches of 16^3, support 16, Q=6; 32 bumps from seed 3, FP32 charge.
    bumps16_128_q6: 128^3, 512 patches of the same geometry, 16 bumps from seed 3, FP32 charge.
    paper_smooth_128_n32: 128^3, 64 patches of 32^3 (the paper's n), support 24, Q=6, the
                    Sec. 7.1 smooth charge in FP32 (profiling case of the 128-point kernels).
    paper_smooth_256_n32_q10: 256^3, 512 patches of 32^3, support 32, the q = 10 operator
                    (b = 4: alpha = 2, beta = 3.25), the Sec. 7.1 smooth charge in FP32.
    """
    if name == "single_bump_32":
        return Workload(name, 32, 8, 8, 4, bumps=single_bump())
    if name == "bumps8_128":
        return Workload(name, 128, 16, 16, 4, bumps=draw_bumps(8, 1))
    if name == "bumps32_256_q6":
        return Workload(name, 256, 16, 16, 6, bumps=draw_bumps(32, 3), charge_dtype="f32")
    if name == "bumps16_128_q6":
        # profiling case: the per-patch kernels of bumps32_256_q6 on 512 patches
        return Workload(name, 128, 16, 16, 6, bumps=draw_bumps(16, 3), charge_dtype="f32")
    if name == "paper_smooth_128_n32":
        return Workload(name, 128, 32, 24, 6, charge_dtype="f32", charge_kind="paper_smooth")
    if name == "paper_smooth_256_n32_q10":
        return Workload(name, 256, 32, 32, 10, charge_dtype="f32", charge_kind="paper_smooth")
    if name == "bumps8_64_q6":
        # reduced-size case with the 27-point operator: same patch geometry as bumps32_256_q6
        return Workload(name, 64, 16, 16, 6, bumps=draw_bumps(8, 7))
    raise KeyError(name)


def batch_problems(count: int = 48, seed: int = 4):
    """Uneven batch: side lengths from {32,48,64,96,128,160}; patch 8 for side 32, else 16;
    support = patch side; Q=4; 1..16 bumps per problem from seed 4000+k."""
    rng = np.random.default_rng(seed)
    sides = rng.choice(np.array([32, 48, 64, 96, 128, 160]), size=count)
    nb = rng.integers(1, 17, size=count)
    out = []
    for k in range(count):
        N = int(sides[k])
        n = 8 if N == 32 else 16
        out.append(Workload(f"batch{k}", N, n, n, 4, bumps=draw_bumps(int(nb[k]), 4000 + k)))
    return out


def serving_requests(count: int = 2000, seed: int = 5, lo: int = 64, hi: int = 384):
    """Request mix: side log-uniform in [lo, hi] rounded to a multiple of 16, patch 16,
    support 16, Q in {4, 6}, tier 50/50 FP64/split, 1..32 bumps (seed 50000+k)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        side = int(16 * round(math.exp(rng.uniform(math.log(lo), math.log(hi))) / 16))
        side = max(lo, min(hi, side))
        Q = int(rng.choice([4, 6]))
        tier = "fp64" if rng.uniform() < 0.5 else "split"
        nb = int(rng.integers(1, 33))
        out.append((Workload(f"req{k}", side, 16, 16, Q, bumps=draw_bumps(nb, 50000 + k)), tier))
    return out
