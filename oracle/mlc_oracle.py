"""FP64 CPU oracle for the two-level Method of Local Corrections.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA library; the only common module is
the seeded input generator ``paper_1702_08111_gb300.inputs``.

The oracle follows the fully discrete two-level algorithm of Sec. 4 step by
step, in the paper's notation, with the plainest computation for each step:

* the discrete Green's function (DGF) is built as in App. A.1 (Dirichlet
  problem on [-zeta nD, zeta nD]^3 with the exact kernel as boundary values,
  residual-correction form, DST-I), using scipy's DST-I;
* every convolution is a direct sum (a dense matrix product with the
  Green's-function lag matrix, or the plain loops of ``direct_sum.c``);
* Legendre moments use composite Boole's rule (Sec. 4, Step 1);
* the Dirichlet solves use dense DST-I matrices;
* the boundary values are formed literally as in eqs. (philocmlcII) and
  (mlcfulldiscr): phi^{loc,g} is accumulated at g and at every point of its
  interpolation stencil, then phi^B = phi^loc + I^H(phi^H - phi^loc).

Readings of points where the paper is silent or garbled:

R1  Grid: unit cube, h = 1/N, nodes [0, N]^3; patches are the closed cubes
    n i + [0, n]^3, i in [0, N/n)^3 (Sec. 4).  The charge is given on
    [0, N]^3 internally; the library's arrays hold [0, N)^3 and treat node N
    as zero charge.
R2  Support s: the local field box G(Omega_alpha, C b) is the patch grown by s,
    so the alpha growth is g_alpha = s - C b; g_beta = ceil((beta-1) n / 2)
    with beta = 3 for Q = 4 and 3.25 for Q = 6 (Sec. 7 settings).  MLC-0 is
    g_beta = g_alpha.
R3  Legendre basis: orthonormal Q^p(x) = R^{-3/2} prod_d sqrt((2p_d+1)/2)
    P_{p_d}((x_d - c_d)/R), index set |p|_1 <= P-1 in lexicographic order
    with p_2 fastest (eq. led3d, normalisation made orthonormal).  The
    coefficients are the Boole-rule inner products of the unweighted f with
    Q^p over the closed patch; the discrete Legendre charge is
    P^h(f^{i,h}) = chi * sum_p c_p Q^p(gh).
R4  Interpolant I^H (Sec. 4, Step 3): tensor-product Lagrange interpolation
    in the face plane.  Along an axis where g is a coarse node the stencil is
    that node alone; otherwise it is the 2b+2 coarse nodes k0-b .. k0+b+1,
    k0 = floor(g/4).  Order q_I = 2b+2.
R5  Region membership is by closed boxes; the ring is
    Omega_beta \\ Omega_alpha at the fine level and C(Omega_beta) \\
    C(Omega_alpha) at the coarse level.  Sums over patches run in ascending
    patch linear index.
R6  phi^H is evaluated on the coarse nodes [-b, N/4 + b]^3, the nodes the
    interpolation reads.
R7  Delta^H is the same Mehrstellen operator at spacing H = C h applied to the
    fine field sampled at coarse nodes; G^H = H^{-1} G^{h=1}.
R16 Multilevel MLC (Sec. 5), levels > 2: with every level covering the whole
    grid, chi-tilde vanishes, and the level-l charge of patch i is the coarse
    charge F^{h_l} (the sum of the finer patches' contributions, eq. FDLD)
    restricted to the patch, as the fine charge is in Sec. 4.  The downward
    pass, the level-0 solve and the upward pass are then, level by level, the
    two-level steps with the global coarse solve phi^H = G^H * F^H replaced by
    the MLC solve of F^H on the coarse grid: its domain is the smallest box of
    whole patches from min(F^H lo, phi^H lo) that holds the support of F^H and
    the nodes phi^H is needed on (the proper nesting of eq.
    propernesting2fdiscr), with the same n, P, Q, b, g_beta and mode, and
    the support s, or coarse_s where given (a larger inner radius alpha at
    the coarser levels, as Sec. 7.2 suggests).  The
    upward pass interpolates the uncorrected coarse solution (eq.
    mlcmultilevel); the Mehrstellen correction (eq.
    mcapplicationfullmultipole) adds C2 h_l^2 times the level's own charge
    term chi-tilde f, zero on the coarse levels, so only the finest level is
    corrected.
R18 The q = 10 operator of Sec. 8 (Q = 10): the six-orbit, 57-point solution
    of the q = 10 conditions of eq. mehrstellenTau (STENCIL_ORBITS, derived in
    derive_q10.py), C2 = 2/35.  Its DGF takes the free-space kernel as the
    residual-correction reference field on the whole box (_dgf_full_wide).
    The final Dirichlet step has a second boundary layer, one node outside
    the closed faces.  Its boundary values come from eqs. philocmlcII and
    mlcfulldiscr with the R4 interpolation factor on all three axes
    (outer_nodes, stencils3_for), and the step is a sparse LU solve with two
    layers (dirichlet_solve_wide).  phi^H is kept one coarse node further out.
    Defaults b = 4, beta = 3.25: on the Sec. 7.1 charge at 256^3, n = 32, the
    q = 10 solve beats L27 only from g_alpha = 16 on, and b = 5 (q_I = q + 2)
    leaves no room for that inside a period-128 field box.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass
from fractions import Fraction
from functools import lru_cache

import numpy as np
import scipy.fft

_HERE = os.path.dirname(os.path.abspath(__file__))
_CACHE = os.path.join(_HERE, "_cache")
_BUILD = os.path.join(_HERE, "_build")

# App. A.1: a_j = b_{|j|} / h^2, |j| = number of nonzero components of j.
STENCIL_B = {
    4: (-4.0, 1.0 / 3.0, 1.0 / 6.0, 0.0),  # L19, q = 4
    6: (-64.0 / 15.0, 7.0 / 15.0, 1.0 / 10.0, 1.0 / 30.0),  # L27, q = 6
}
C2 = 1.0 / 12.0  # Sec. 2, eq. (msCorr4), for L19 and L27

# R18 (Sec. 8): a q = 10 Mehrstellen operator in the 5 x 5 x 5 block (s = 2).
# a_j depends on the orbit of j under the cube's symmetries, named by the
# sorted absolute components.  These are the six orbits with the smallest
# offsets for which the six conditions of Sec. 2 (eq. mehrstellenTau with
# q = 10) have a solution: sum a_j = 0; sum a_j j_0^2 = 2 (consistency); and
# sum a_j p(j) = 0 for every harmonic homogeneous polynomial p of degree 4, 6,
# 8 and 10 (so the truncation error vanishes on harmonic functions up to
# h^10).  Exact rationals; derived by oracle/derive_q10.py (sympy).
STENCIL_ORBITS = {
    10: {(0, 0, 0): Fraction(-1079, 210), (1, 0, 0): Fraction(24, 35), (1, 1, 0): Fraction(17, 210),
         (1, 1, 1): Fraction(11, 420), (2, 0, 0): Fraction(-1, 60), (2, 1, 0): Fraction(-1, 420)},
}
# C2 of eq. (mehrstellenTau) for each operator: the h^2 term of the truncation
# error is C2 h^2 Delta^2 phi, C2 = sum a_j j_0^4 / 4!  (1/12 for L19 and L27,
# 2/35 for the q = 10 operator); the 4th-order correction adds C2 h^2 f.
C2_OF = {4: 1.0 / 12.0, 6: 1.0 / 12.0, 10: 2.0 / 35.0}
QS = (4, 6, 10)


def stencil_reach(Q: int) -> int:
    """Largest |offset component| of the operator (s of eq. discreteLaplacian)."""
    return 2 if Q in STENCIL_ORBITS else 1


# ---------------------------------------------------------------------------
# Parameters (R2)
# ---------------------------------------------------------------------------

@dataclass
class Params:
    N: int
    n: int
    s: int
    P: int = 4
    Q: int = 4
    C: int = 4
    beta: float | None = None
    b: int | None = None
    mode: str = "mlc"  # "mlc" (alpha < beta) or "mlc0" (alpha = beta)
    nD: int = 128
    zeta: int = 2
    levels: int = 2          # Sec. 5: number of levels (2: the two-level algorithm of Sec. 4)
    coarse_s: int | None = None  # support s of the coarser levels (R16; None: s)
    h_level: float | None = None   # mesh spacing of this level (default 1/N, the finest level)
    correction: bool = True  # add C2 h^2 f at the end (eq. mcapplicationfulldiscr); R16

    def __post_init__(self):
        if self.Q not in QS:
            raise ValueError("Q must be 4, 6 or 10")
        if self.C != 4:
            raise ValueError("coarsening ratio is 4 (Sec. 2)")
        if self.N % self.n or self.n % 4 or self.s % 4:
            raise ValueError("need n | N, 4 | n, 4 | s")
        if self.b is None:  # q_I = 2b + 2 = q + 2 (Sec. 7); b = 4 for q = 10 (R18)
            self.b = {4: 2, 6: 3, 10: 4}[self.Q]
        if self.beta is None:  # Sec. 7 settings; q = 10 as L27 (R18)
            self.beta = {4: 3.0, 6: 3.25, 10: 3.25}[self.Q]
        if self.levels < 2:
            raise ValueError("levels >= 2")
        if self.Q == 10 and self.levels != 2:
            raise ValueError("the q = 10 operator runs two levels (R18)")
        self.h = 1.0 / self.N if self.h_level is None else float(self.h_level)
        self.H = self.C * self.h
        self.R = self.n * self.h / 2.0
        self.np_ = self.N // self.n
        self.g_alpha = self.s - self.C * self.b
        if self.g_alpha < 0:
            raise ValueError("support smaller than C*b")
        if self.mode == "mlc0":
            self.g_beta = self.g_alpha
        else:
            self.g_beta = math.ceil((Fraction(self.beta) - 1) * self.n / 2)
        if self.g_beta < self.g_alpha:
            raise ValueError("g_beta < g_alpha")

    # relative boxes (per axis, inclusive), relative to the patch origin n*i
    @property
    def alpha_box(self):
        return (-self.g_alpha, self.n + self.g_alpha)

    @property
    def beta_box(self):
        return (-self.g_beta, self.n + self.g_beta)

    @property
    def field_box(self):
        return (-self.s, self.n + self.s)

    # coarse boxes relative to the patch's coarse origin n*i/4 (Sec. 2, C(D))
    @property
    def c_alpha(self):
        return (math.floor(-self.g_alpha / 4), math.ceil((self.n + self.g_alpha) / 4))

    @property
    def c_beta(self):
        return (math.floor(-self.g_beta / 4), math.ceil((self.n + self.g_beta) / 4))

    @property
    def fh_extent(self):
        lo, hi = self.c_beta
        return (lo, (self.np_ - 1) * self.n // 4 + hi)

    @property
    def phih_extent(self):
        # R6; R18: the second boundary layer (one node off the face planes)
        # reaches one coarse node further
        e = self.b + (1 if stencil_reach(self.Q) > 1 else 0)
        return (-e, self.N // 4 + e)

    @property
    def c2(self):
        return C2_OF[self.Q]

    @property
    def npatch(self):
        return self.np_ ** 3


def patch_origin(prm: Params, i: int) -> np.ndarray:
    i0, rem = divmod(i, prm.np_ * prm.np_)
    i1, i2 = divmod(rem, prm.np_)
    return np.array([i0, i1, i2], dtype=np.int64) * prm.n


# ---------------------------------------------------------------------------
# Mehrstellen operators (Sec. 2, App. A.1)
# ---------------------------------------------------------------------------

def stencil(Q: int):
    """List of (offset, a_offset) (h = 1) over [-s,s]^3 with nonzero coefficient."""
    out = []
    if Q in STENCIL_ORBITS:
        orb = STENCIL_ORBITS[Q]
        for s0 in range(-2, 3):
            for s1 in range(-2, 3):
                for s2 in range(-2, 3):
                    key = tuple(sorted((abs(s0), abs(s1), abs(s2)), reverse=True))
                    if key in orb:
                        out.append(((s0, s1, s2), float(orb[key])))
        return out
    b = STENCIL_B[Q]
    for s0 in (-1, 0, 1):
        for s1 in (-1, 0, 1):
            for s2 in (-1, 0, 1):
                nz = (s0 != 0) + (s1 != 0) + (s2 != 0)
                if b[nz] != 0.0:
                    out.append(((s0, s1, s2), b[nz]))
    return out


def apply_laplacian(phi: np.ndarray, Q: int, h: float) -> np.ndarray:
    """Eq. (discreteLaplacian) on the interior G(D,-s) of the array's box."""
    r = stencil_reach(Q)
    n0, n1, n2 = phi.shape
    out = np.zeros((n0 - 2 * r, n1 - 2 * r, n2 - 2 * r))
    for (s0, s1, s2), c in stencil(Q):
        out += c * phi[r + s0:n0 - r + s0, r + s1:n1 - r + s1, r + s2:n2 - r + s2]
    return out / (h * h)


def symbol(Q: int, c0, c1, c2):
    """Eigenvalue (h = 1) of the stencil on the product of 1D modes whose
    shift-pair eigenvalues are 2 c_d: sum_j a_j prod_d cos(j_d theta_d) with
    cos(2 theta) = 2 c^2 - 1."""
    if Q in STENCIL_ORBITS:
        cs = (c0, c1, c2)
        lam = 0.0
        for off, a in stencil(Q):
            t = a
            for d in range(3):
                k = abs(off[d])
                t = t * (1.0 if k == 0 else (cs[d] if k == 1 else 2.0 * cs[d] * cs[d] - 1.0))
            lam = lam + t
        return lam
    b0, b1, b2, b3 = STENCIL_B[Q]
    return (b0 + 2 * b1 * (c0 + c1 + c2) + 4 * b2 * (c0 * c1 + c0 * c2 + c1 * c2)
            + 8 * b3 * c0 * c1 * c2)


# ---------------------------------------------------------------------------
# Discrete Green's function (Sec. 2 eq. dgf; App. A.1)
# ---------------------------------------------------------------------------

def dgf_full(Q: int, nD: int, zeta: int) -> np.ndarray:
    """Solve L G = delta_0 on G(D_zeta,-1), G = -1/(4 pi |g|) on the boundary of
    D_zeta = [-zeta nD, zeta nD]^3; returns G on all of D_zeta."""
    M = zeta * nD
    if stencil_reach(Q) > 1:
        return _dgf_full_wide(Q, M)
    x = np.arange(-M, M + 1, dtype=np.float64)
    G = np.zeros((2 * M + 1,) * 3)
    # boundary values: exact free-space Green's function
    for axis in range(3):
        for end in (0, 2 * M):
            sl = [slice(None)] * 3
            sl[axis] = end
            grids = np.meshgrid(*[x if d != axis else x[end:end + 1] for d in range(3)], indexing="ij")
            r = np.sqrt(grids[0] ** 2 + grids[1] ** 2 + grids[2] ** 2)
            G[tuple(sl)] = (-1.0 / (4.0 * math.pi * r)).reshape(G[tuple(sl)].shape)
    # residual-correction form: L u = delta - L(G_boundary), u = 0 on the boundary
    rhs = -apply_laplacian(G, Q, 1.0)
    rhs[M - 1, M - 1, M - 1] += 1.0
    K = 2 * M - 1
    c = np.cos(np.pi * np.arange(1, K + 1) / (2 * M))
    lam = symbol(Q, c[:, None, None], c[None, :, None], c[None, None, :])
    uh = scipy.fft.dstn(rhs, type=1, workers=os.cpu_count())
    del rhs
    uh /= lam
    u = scipy.fft.idstn(uh, type=1, workers=os.cpu_count())
    G[1:-1, 1:-1, 1:-1] += u
    return G


def _dgf_full_wide(Q: int, M: int) -> np.ndarray:
    """R18: the DGF of a two-layer operator (s = 2) on D_zeta = [-M, M]^3.

    Residual-correction form with the free-space kernel w = -1/(4 pi |g|)
    (w(0) = 0) as the reference field on the whole box: L u = delta - L w on
    the nodes |g|_inf <= M - 1, u = 0 on |g|_inf = M, and G = w + u.  DST-I
    continues u oddly across the boundary, so where the stencil reaches the
    second layer |g|_inf = M + 1 it reads w minus the mirrored u; u = G - w
    is O(|g|^-5) there (1e-12 of G at M = 256), far below the O((zeta nD)^-4)
    effect of the boundary values themselves (App. A.1)."""
    x = np.arange(-M - 1, M + 2, dtype=np.float64)
    W = np.empty((2 * M + 3,) * 3)
    for i, xi in enumerate(x):
        r = np.sqrt(xi * xi + x[:, None] ** 2 + x[None, :] ** 2)
        with np.errstate(divide="ignore"):
            W[i] = -1.0 / (4.0 * math.pi * r)
    W[M + 1, M + 1, M + 1] = 0.0
    rhs = -apply_laplacian(W, Q, 1.0)  # nodes [-M+1, M-1]^3
    rhs[M - 1, M - 1, M - 1] += 1.0
    K = 2 * M - 1
    c = np.cos(np.pi * np.arange(1, K + 1) / (2 * M))
    lam = symbol(Q, c[:, None, None], c[None, :, None], c[None, None, :])
    uh = scipy.fft.dstn(rhs, type=1, workers=os.cpu_count())
    del rhs
    uh /= lam
    u = scipy.fft.idstn(uh, type=1, workers=os.cpu_count())
    del uh
    G = W[1:-1, 1:-1, 1:-1].copy()
    del W
    G[1:-1, 1:-1, 1:-1] += u
    return G


def dgf_octant(Q: int, nD: int = 128, zeta: int = 2) -> np.ndarray:
    """G^{h=1} on the octant [0, nD]^3 (cached on disk)."""
    return _dgf_octant_cached(Q, nD, zeta).copy()


@lru_cache(maxsize=8)
def _dgf_octant_cached(Q: int, nD: int, zeta: int) -> np.ndarray:
    path = os.path.join(_CACHE, f"dgf_Q{Q}_nD{nD}_z{zeta}.npy")
    if os.path.exists(path):
        return np.load(path)
    M = zeta * nD
    G = dgf_full(Q, nD, zeta)
    oct_ = np.ascontiguousarray(G[M:M + nD + 1, M:M + nD + 1, M:M + nD + 1])
    del G
    os.makedirs(_CACHE, exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp.npy"
    np.save(tmp, oct_)
    os.replace(tmp, path)
    return oct_


# ---------------------------------------------------------------------------
# Direct sums
# ---------------------------------------------------------------------------

def _direct_lib():
    so = os.path.join(_BUILD, "liboracle_direct.so")
    src = os.path.join(_HERE, "direct_sum.c")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        build_c()
    lib = ctypes.CDLL(so)
    lib.oracle_direct_sum.restype = ctypes.c_int
    return lib


def build_c():
    """Compile the oracle's C helper (plain loops + OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    so = os.path.join(_BUILD, "liboracle_direct.so")
    tmp = so + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp,
                           os.path.join(_HERE, "direct_sum.c")])
    os.replace(tmp, so)
    return so


def direct_sum(T: np.ndarray, src: np.ndarray, src_lo, out_lo, out_shape, scale: float) -> np.ndarray:
    """out[o] = scale * sum_k T[|o-k|] src[k] by plain loops (direct_sum.c)."""
    lib = _direct_lib()
    T = np.ascontiguousarray(T, dtype=np.float64)
    src = np.ascontiguousarray(src, dtype=np.float64)
    out = np.zeros(tuple(out_shape), dtype=np.float64)
    L = T.shape[0] - 1
    ia = ctypes.c_int * 3
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.oracle_direct_sum(T.ctypes.data_as(dp), ctypes.c_int(L), src.ctypes.data_as(dp),
                               ia(*src_lo), ia(*src.shape), out.ctypes.data_as(dp),
                               ia(*out_lo), ia(*out_shape), ctypes.c_double(scale))
    if rc != 0:
        raise ValueError("lag beyond the DGF table")
    return out


def green_matrix(G1: np.ndarray, pts: np.ndarray, src: np.ndarray, chunk: int = 512) -> np.ndarray:
    """Lag matrix M[a, j] = G1[|pts[a] - src[j]|] (per-axis absolute lags)."""
    out = np.empty((pts.shape[0], src.shape[0]))
    for a0 in range(0, pts.shape[0], chunk):
        p = pts[a0:a0 + chunk]
        d = np.abs(p[:, None, :] - src[None, :, :])
        out[a0:a0 + chunk] = G1[d[..., 0], d[..., 1], d[..., 2]]
    return out


# ---------------------------------------------------------------------------
# Patch quantities: chi, Boole weights, Legendre basis (Sec. 3 eq. led3d, Sec. 4)
# ---------------------------------------------------------------------------

def box_points(lo, hi, step: int = 1) -> np.ndarray:
    r = np.arange(lo, hi + 1, step, dtype=np.int64)
    g = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1)
    return g.reshape(-1, 3)


def chi_1d(n: int) -> np.ndarray:
    w = np.ones(n + 1)
    w[0] = w[-1] = 0.5
    return w


def chi_patch(n: int) -> np.ndarray:
    """Discrete characteristic function of the closed patch (Sec. 4): 1/8 at
    corners, 1/4 on edges, 1/2 on faces, 1 inside -- flattened over [0,n]^3."""
    w = chi_1d(n)
    return (w[:, None, None] * w[None, :, None] * w[None, None, :]).reshape(-1)


def boole_weights_1d(n: int, h: float) -> np.ndarray:
    """Composite Boole's rule on [0, n h] with n/4 panels."""
    if n % 4:
        raise ValueError("Boole's rule needs 4 | n")
    w = np.zeros(n + 1)
    panel = (2.0 * h / 45.0) * np.array([7.0, 32.0, 12.0, 32.0, 7.0])
    for p in range(n // 4):
        w[4 * p:4 * p + 5] += panel
    return w


def legendre_index(P: int):
    return [(p0, p1, p2) for p0 in range(P) for p1 in range(P) for p2 in range(P) if p0 + p1 + p2 < P]


def legendre_1d(k: int, t: np.ndarray) -> np.ndarray:
    """Orthonormal Legendre polynomial sqrt((2k+1)/2) P_k(t) on [-1, 1]."""
    coef = np.zeros(k + 1)
    coef[k] = 1.0
    return math.sqrt((2 * k + 1) / 2.0) * np.polynomial.legendre.legval(t, coef)


def legendre_patch(prm: Params) -> np.ndarray:
    """Q^p at the closed-patch nodes m in [0,n]^3: array (npoly, (n+1)^3)."""
    n = prm.n
    t = 2.0 * np.arange(n + 1) / n - 1.0  # (x - c)/R at the nodes
    vals = [legendre_1d(k, t) for k in range(prm.P)]
    out = []
    for p0, p1, p2 in legendre_index(prm.P):
        v = vals[p0][:, None, None] * vals[p1][None, :, None] * vals[p2][None, None, :]
        out.append(v.reshape(-1) * prm.R ** -1.5)
    return np.array(out)


def moment_matrix(prm: Params) -> np.ndarray:
    """Row p: Boole weight times Q^p at the patch nodes, so c = M @ f_patch."""
    w = boole_weights_1d(prm.n, prm.h)
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).reshape(-1)
    return legendre_patch(prm) * W[None, :]


# ---------------------------------------------------------------------------
# Face lattice and interpolation stencils (R4)
# ---------------------------------------------------------------------------

def lagrange_weights(t: float, nodes: np.ndarray) -> np.ndarray:
    w = np.ones(len(nodes))
    for j in range(len(nodes)):
        for l in range(len(nodes)):
            if l != j:
                w[j] *= (t - nodes[l]) / (nodes[j] - nodes[l])
    return w


def axis_stencil(g: int, b: int):
    """(coarse nodes, weights) of the 1D factor of I^H at fine coordinate g."""
    if g % 4 == 0:
        return np.array([g // 4]), np.array([1.0])
    k0 = g // 4
    nodes = np.arange(k0 - b, k0 + b + 2)
    return nodes, lagrange_weights(g / 4.0, nodes.astype(np.float64))


def face_stencil(g, b: int):
    """Stencil of I^H at a face-lattice node g, padded to (2b+2)^2 entries.

    Returns (coarse points (S,3), weights (S,)).  Padding entries repeat the
    first point with weight 0."""
    per_axis = [axis_stencil(int(g[d]), b) for d in range(3)]
    nontriv = [d for d in range(3) if len(per_axis[d][0]) > 1]
    if len(nontriv) > 2:
        raise ValueError("node is not on a face plane")
    S = (2 * b + 2) ** 2
    pts = np.zeros((S, 3), dtype=np.int64)
    wts = np.zeros(S)
    k = 0
    for a0, w0 in zip(*per_axis[0]):
        for a1, w1 in zip(*per_axis[1]):
            for a2, w2 in zip(*per_axis[2]):
                pts[k] = (a0, a1, a2)
                wts[k] = w0 * w1 * w2
                k += 1
    pts[k:] = pts[0]
    return pts, wts


def face_nodes_in_box(prm: Params, lo: int, hi: int) -> np.ndarray:
    """Face-lattice nodes (some coordinate a multiple of n) in the relative box [lo,hi]^3."""
    pts = box_points(lo, hi)
    on_face = np.any(pts % prm.n == 0, axis=1)
    return pts[on_face]


def stencils_for(prm: Params, nodes: np.ndarray):
    """Vectorised I^H stencils (R4) for many face-lattice nodes.

    The first axis on which the node sits on a face plane is taken as the face
    normal (weight 1 there); the two in-plane axes carry 2b+2 entries each, a
    trivial in-plane axis (node on a coarse line) having weights (1, 0, ...)
    at one repeated node.  Returns coarse points (A, S, 3) and weights (A, S),
    S = (2b+2)^2; the nonzero terms are the same as in face_stencil."""
    b = prm.b
    K = 2 * b + 2
    g = np.asarray(nodes, dtype=np.int64)
    A = g.shape[0]
    onface = (g % prm.n) == 0
    if not np.all(np.any(onface, axis=1)):
        raise ValueError("node is not on a face plane")
    dstar = np.argmax(onface, axis=1)
    kn = np.zeros((A, 3, K), dtype=np.int64)
    wt = np.zeros((A, 3, K))
    j = np.arange(K)
    for d in range(3):
        gd = g[:, d]
        triv = (gd % 4) == 0
        k0 = gd // 4
        nd = k0[:, None] - b + j[None, :]
        r = (gd - 4 * k0).astype(np.float64) / 4.0  # t - k0 in [0, 1)
        w = np.ones((A, K))
        for jj in range(K):
            for ll in range(K):
                if ll != jj:
                    w[:, jj] *= (r + b - ll) / float(jj - ll)
        kn[:, d, :] = np.where(triv[:, None], k0[:, None], nd)
        wt[:, d, :] = np.where(triv[:, None], (j[None, :] == 0).astype(np.float64), w)
    a1 = np.where(dstar == 0, 1, 0)
    a2 = np.where(dstar == 2, 1, 2)
    rows = np.arange(A)
    P = np.zeros((A, K, K, 3), dtype=np.int64)
    P[:, :, :, :] = (g // 4)[:, None, None, :]
    P[rows, :, :, a1] = kn[rows, a1, :][:, :, None]
    P[rows, :, :, a2] = kn[rows, a2, :][:, None, :]
    W = wt[rows, a1, :][:, :, None] * wt[rows, a2, :][:, None, :]
    return P.reshape(A, K * K, 3), W.reshape(A, K * K)


def offplane_mask(pts: np.ndarray, n: int) -> np.ndarray:
    """R18: nodes one step off a face plane along some axis (a coordinate that
    is 1 or n-1 modulo n)."""
    m = np.asarray(pts) % n
    return np.any((m == 1) | (m == n - 1), axis=1)


def outer_nodes(prm: Params) -> np.ndarray:
    """R18: the second boundary layer of the s = 2 operator, globally: the
    nodes on the planes n j -+ 1 (j in [0, N/n]) of some axis whose other two
    coordinates lie in [0, N] (patch i reads the plane n i_d - 1 and
    n i_d + n + 1 over its closed face), sorted."""
    N, n = prm.N, prm.n
    r = np.arange(0, N + 1, dtype=np.int64)
    u, v = np.meshgrid(r, r, indexing="ij")
    out = []
    for d in range(3):
        e1, e2 = [e for e in range(3) if e != d]
        for c in sorted({n * j + sg for j in range(prm.np_ + 1) for sg in (-1, 1)}):
            g = np.empty((u.size, 3), dtype=np.int64)
            g[:, d] = c
            g[:, e1] = u.ravel()
            g[:, e2] = v.ravel()
            out.append(g)
    return np.unique(np.concatenate(out), axis=0)


def stencils3_for(prm: Params, nodes: np.ndarray):
    """R18: I^H stencils at nodes off the face planes: R4's tensor-product
    Lagrange factor on every axis (the coarse node alone where the coordinate
    is a multiple of 4, else the 2b+2 coarse nodes k0-b .. k0+b+1, k0 =
    floor(g/4)); trivial axes carry weights (1, 0, ...) at a repeated node.
    Returns coarse points (A, K^3, 3) and weights (A, K^3), K = 2b+2."""
    b = prm.b
    K = 2 * b + 2
    g = np.asarray(nodes, dtype=np.int64)
    A = g.shape[0]
    kn = np.zeros((A, 3, K), dtype=np.int64)
    wt = np.zeros((A, 3, K))
    j = np.arange(K)
    for d in range(3):
        gd = g[:, d]
        triv = (gd % 4) == 0
        k0 = gd // 4
        r = (gd - 4 * k0).astype(np.float64) / 4.0
        w = np.ones((A, K))
        for jj in range(K):
            for ll in range(K):
                if ll != jj:
                    w[:, jj] *= (r + b - ll) / float(jj - ll)
        kn[:, d, :] = np.where(triv[:, None], k0[:, None], k0[:, None] - b + j[None, :])
        wt[:, d, :] = np.where(triv[:, None], (j[None, :] == 0).astype(np.float64), w)
    P = np.empty((A, K, K, K, 3), dtype=np.int64)
    P[..., 0] = kn[:, 0, :][:, :, None, None]
    P[..., 1] = kn[:, 1, :][:, None, :, None]
    P[..., 2] = kn[:, 2, :][:, None, None, :]
    W = wt[:, 0, :][:, :, None, None] * wt[:, 1, :][:, None, :, None] * wt[:, 2, :][:, None, None, :]
    return P.reshape(A, K ** 3, 3), W.reshape(A, K ** 3)


class PointSet:
    """A set of relative integer points with a dense lookup map over a box."""

    def __init__(self, pts: np.ndarray):
        pts = np.unique(pts, axis=0)
        self.pts = pts
        self.lo = pts.min(axis=0)
        self.hi = pts.max(axis=0)
        shape = tuple(self.hi - self.lo + 1)
        self.map = -np.ones(shape, dtype=np.int64)
        q = pts - self.lo
        self.map[q[:, 0], q[:, 1], q[:, 2]] = np.arange(len(pts))

    def index(self, q: np.ndarray) -> np.ndarray:
        r = q - self.lo
        if np.any(r < 0) or np.any(r >= np.array(self.map.shape)):
            raise IndexError("point outside the computed set")
        idx = self.map[r[..., 0], r[..., 1], r[..., 2]]
        if np.any(idx < 0):
            raise IndexError("point not in the computed set")
        return idx


# ---------------------------------------------------------------------------
# The two-level solve (Sec. 4)
# ---------------------------------------------------------------------------

def pad_charge(f: np.ndarray) -> np.ndarray:
    """[0,N)^3 charge -> [0,N]^3 with zero charge on the nodes N (R1)."""
    N = f.shape[0]
    fc = np.zeros((N + 1,) * 3)
    fc[:N, :N, :N] = f
    return fc


def required_dgf_extent(prm: Params) -> int:
    n, s, gb, b = prm.n, prm.s, prm.g_beta, prm.b
    local = n + s
    basis = n + gb + 4 * b + 4 + 4 if gb > prm.g_alpha else 0
    flo, fhi = prm.fh_extent
    olo, ohi = prm.phih_extent
    coarse = max(fhi - olo, ohi - flo)
    return max(local, basis, coarse)


def mlc_solve(prm: Params, f_closed: np.ndarray, G1: np.ndarray | None = None, stages: dict | None = None):
    """Two-level MLC (Sec. 4) for the charge f on [0,N]^3 (shape (N+1)^3).

    Returns phi^{MLC,h} on [0,N]^3.  If ``stages`` is a dict it is filled with
    the intermediate results (moments, F^H, phi^H, phi^B)."""
    N, n, h, H = prm.N, prm.n, prm.h, prm.H
    if f_closed.shape != (N + 1,) * 3:
        raise ValueError("charge must be given on [0,N]^3")
    if G1 is None:
        G1 = dgf_octant(prm.Q, prm.nD, prm.zeta)
    if required_dgf_extent(prm) > G1.shape[0] - 1:
        raise ValueError("DGF table too small for these parameters")
    NP = prm.npatch
    src = box_points(0, n)  # closed-patch nodes m
    chi = chi_patch(n)
    origins = np.array([patch_origin(prm, i) for i in range(NP)])
    # charges of all patches as columns: f[n i + m]
    Fcols = np.empty((src.shape[0], NP))
    for i in range(NP):
        g = origins[i][None, :] + src
        Fcols[:, i] = f_closed[g[:, 0], g[:, 1], g[:, 2]]

    lap = stencil(prm.Q)
    wide = stencil_reach(prm.Q) > 1  # R18: a second boundary layer one node off the faces
    ga_lo, ga_hi = prm.alpha_box
    gb_lo, gb_hi = prm.beta_box

    # ---- Step 1: local convolutions phi^{i,h} = G^h * f^{i,h} (eq. initiallocalproblemsmlcII)
    fb_lo, fb_hi = prm.field_box
    face_alpha = face_nodes_in_box(prm, ga_lo, ga_hi)
    coarse_field = box_points(fb_lo, fb_hi, 4)
    pts_list = [coarse_field, face_alpha]
    if wide:
        bx = box_points(ga_lo, ga_hi)
        outer_alpha = bx[offplane_mask(bx, n)]
        pts_list.append(outer_alpha)
    phi_set = PointSet(np.concatenate(pts_list))
    Kphi = green_matrix(G1, phi_set.pts, src) * (h * h) * chi[None, :]
    PHI = Kphi @ Fcols  # (points, patches)
    del Kphi

    # Legendre coefficients by composite Boole's rule (Sec. 4, Step 1)
    Cmom = moment_matrix(prm) @ Fcols  # (npoly, patches)

    ca_lo, ca_hi = prm.c_alpha
    cb_lo, cb_hi = prm.c_beta
    ck_alpha = box_points(ca_lo, ca_hi)
    ring = prm.g_beta > prm.g_alpha
    if ring:
        ck_beta = box_points(cb_lo, cb_hi)
        in_alpha = np.all((ck_beta >= ca_lo) & (ck_beta <= ca_hi), axis=1)
        ck_ring = ck_beta[~in_alpha]
        face_beta = face_nodes_in_box(prm, gb_lo, gb_hi)
        inA = np.all((face_beta >= ga_lo) & (face_beta <= ga_hi), axis=1)
        face_ring = face_beta[~inA]
        st_ring_P, st_ring_W = stencils_for(prm, face_ring)
        # points at which the basis fields G^h * P^h are needed
        lap_pts = (4 * (ck_ring[:, None, :] + np.array([o for o, _ in lap])[None, :, :])).reshape(-1, 3)
        b_list = [lap_pts, face_ring, 4 * st_ring_P.reshape(-1, 3)]
        if wide:
            bxb = box_points(gb_lo, gb_hi)
            ob = bxb[offplane_mask(bxb, n)]
            outer_ring = ob[~np.all((ob >= ga_lo) & (ob <= ga_hi), axis=1)]
            # every coarse point a 3D stencil of a beta-box node can reach
            k_lo, k_hi = gb_lo // 4 - prm.b - 1, -(-gb_hi // 4) + prm.b + 1
            b_list += [outer_ring, 4 * box_points(k_lo, k_hi)]
        B_set = PointSet(np.concatenate(b_list))
        Lcharge = (legendre_patch(prm) * chi[None, :]).T  # (src, npoly)
        BV = (green_matrix(G1, B_set.pts, src) * (h * h)) @ Lcharge  # (points, npoly)

    # local coarse charges F^{i,H} (eq. FDLD) and their sum F^H (Step 2)
    flo, fhi = prm.fh_extent
    nf = fhi - flo + 1
    FH = np.zeros((nf, nf, nf))
    offs = np.array([o for o, _ in lap])
    coefs = np.array([c for _, c in lap]) / (H * H)
    idxA = phi_set.index(4 * (ck_alpha[:, None, :] + offs[None, :, :]))  # (|Calpha|, nst)
    LapA = np.einsum("s,asp->ap", coefs, PHI[idxA])  # (|Calpha|, patches)
    if ring:
        idxR = B_set.index(4 * (ck_ring[:, None, :] + offs[None, :, :]))
        T = np.einsum("s,asq->aq", coefs, BV[idxR])  # Delta^H (G^h * Q^p) on the ring, (|ring|, npoly)
        LapR = T @ Cmom  # (|ring|, patches)
    for i in range(NP):
        co = origins[i] // 4
        k = ck_alpha + co - flo
        FH[k[:, 0], k[:, 1], k[:, 2]] += LapA[:, i]
        if ring:
            k = ck_ring + co - flo
            FH[k[:, 0], k[:, 1], k[:, 2]] += LapR[:, i]

    # ---- Step 2: global coarse solve phi^H = G^H * F^H, G^H = H^{-1} G^{h=1}
    olo, ohi = prm.phih_extent
    no = ohi - olo + 1
    if prm.levels > 2:
        # Sec. 5 (R16): the coarse solve is itself an MLC solve of F^H
        phiH = coarse_level_solve(prm, FH, G1)
    else:
        phiH = direct_sum(G1, FH, (flo,) * 3, (olo,) * 3, (no,) * 3, H * H)

    # ---- Step 3: boundary values by local corrections (eqs. philocmlcII, mlcfulldiscr)
    gpts = box_points(0, N)
    gface = gpts[np.any(gpts % n == 0, axis=1)]
    del gpts
    gmap = -np.ones((N + 1,) * 3, dtype=np.int64)
    gmap[gface[:, 0], gface[:, 1], gface[:, 2]] = np.arange(len(gface))
    S = (2 * prm.b + 2) ** 2
    # phi^{loc,g} at g itself and at the S points 4k of its stencil
    loc_self = np.zeros(len(gface))
    loc_st = np.zeros((len(gface), S))
    stA_P, _ = stencils_for(prm, face_alpha)
    idx_selfA = phi_set.index(face_alpha)
    idx_stA = phi_set.index(4 * stA_P)  # (|faceA|, S)
    if ring:
        BV_self = BV[B_set.index(face_ring)]  # (|faceR|, npoly)
        BV_st = BV[B_set.index(4 * st_ring_P)].reshape(-1, BV.shape[1])  # (|faceR| S, npoly)
    chunk = 32
    for c0 in range(0, NP, chunk):
        c1 = min(NP, c0 + chunk)
        if ring:
            R_self = BV_self @ Cmom[:, c0:c1]  # (|faceR|, chunk)
            R_st = (BV_st @ Cmom[:, c0:c1]).reshape(len(face_ring), S, c1 - c0)
        for i in range(c0, c1):
            org = origins[i]
            g = face_alpha + org
            ok = np.all((g >= 0) & (g <= N), axis=1)
            gi = gmap[g[ok, 0], g[ok, 1], g[ok, 2]]
            loc_self[gi] += PHI[idx_selfA[ok], i]
            loc_st[gi] += PHI[idx_stA[ok], i]
            if ring:
                g = face_ring + org
                ok = np.all((g >= 0) & (g <= N), axis=1)
                gi = gmap[g[ok, 0], g[ok, 1], g[ok, 2]]
                loc_self[gi] += R_self[ok, i - c0]
                loc_st[gi] += R_st[ok, :, i - c0]
    phiB = np.empty(len(gface))
    for a0 in range(0, len(gface), 1 << 18):
        a1 = min(len(gface), a0 + (1 << 18))
        stG_P, stG_W = stencils_for(prm, gface[a0:a1])
        q = stG_P - olo
        phiH_at = phiH[q[..., 0], q[..., 1], q[..., 2]]
        phiB[a0:a1] = loc_self[a0:a1] + np.sum(stG_W * (phiH_at - loc_st[a0:a1]), axis=1)
    del loc_st

    if wide:
        # ---- R18: the same eqs. (philocmlcII, mlcfulldiscr) on the second
        # ---- boundary layer, with the interpolation stencil on all three axes
        gout = outer_nodes(prm)
        omap = -np.ones((N + 3,) * 3, dtype=np.int64)  # nodes [-1, N+1]^3
        omap[gout[:, 0] + 1, gout[:, 1] + 1, gout[:, 2] + 1] = np.arange(len(gout))
        K3 = (2 * prm.b + 2) ** 3
        oself = np.zeros(len(gout))
        ost = np.zeros((len(gout), K3))
        st3A_P, _ = stencils3_for(prm, outer_alpha)
        i_selfA = phi_set.index(outer_alpha)
        i_stA = phi_set.index(4 * st3A_P)  # (|outerA|, K3)
        del st3A_P
        if ring:
            st3R_P, _ = stencils3_for(prm, outer_ring)
            BVo_self = BV[B_set.index(outer_ring)]
            i_stR = B_set.index(4 * st3R_P)
            del st3R_P

        def in_outer(g):
            ok = np.all((g >= -1) & (g <= N + 1), axis=1)
            gi = -np.ones(len(g), dtype=np.int64)
            gi[ok] = omap[g[ok, 0] + 1, g[ok, 1] + 1, g[ok, 2] + 1]
            return gi >= 0, gi

        for i in range(NP):
            org = origins[i]
            ok, gi = in_outer(outer_alpha + org)
            oself[gi[ok]] += PHI[i_selfA[ok], i]
            ost[gi[ok]] += PHI[i_stA[ok], i]
            if ring:
                ok, gi = in_outer(outer_ring + org)
                oself[gi[ok]] += BVo_self[ok] @ Cmom[:, i]
                ost[gi[ok]] += BV[i_stR[ok]] @ Cmom[:, i]
        phiB_out = np.empty(len(gout))
        for a0 in range(0, len(gout), 4096):
            a1 = min(len(gout), a0 + 4096)
            P3, W3 = stencils3_for(prm, gout[a0:a1])
            q = P3 - olo
            phiB_out[a0:a1] = oself[a0:a1] + np.sum(W3 * (phiH[q[..., 0], q[..., 1], q[..., 2]] - ost[a0:a1]),
                                                     axis=1)
        del ost

    # ---- Dirichlet problems on each patch (eq. last_step_fulldiscr) and the
    # ---- Mehrstellen correction (eq. mcapplicationfulldiscr)
    fp = np.empty((NP,) + (n + 1,) * 3)
    for i in range(NP):
        o = origins[i]
        fp[i] = f_closed[o[0]:o[0] + n + 1, o[1]:o[1] + n + 1, o[2]:o[2] + n + 1]
    if wide:
        # R18: the two boundary layers of [-1, n+1]^3: the closed faces (phi^B)
        # and the layer one node outside them (phi^B on the outer nodes)
        U2 = np.zeros((NP,) + (n + 3,) * 3)
        rel = box_points(-1, n + 1)
        inside = np.all((rel >= 0) & (rel <= n), axis=1)
        face = inside & np.any((rel == 0) | (rel == n), axis=1)
        ext = (np.sum((rel == -1) | (rel == n + 1), axis=1) == 1) & \
            (np.sum((rel >= 0) & (rel <= n), axis=1) == 2)
        for i in range(NP):
            g = rel[face] + origins[i]
            U2[i][tuple((rel[face] + 1).T)] = phiB[gmap[g[:, 0], g[:, 1], g[:, 2]]]
            g = rel[ext] + origins[i]
            U2[i][tuple((rel[ext] + 1).T)] = phiB_out[omap[g[:, 0] + 1, g[:, 1] + 1, g[:, 2] + 1]]
        U = dirichlet_solve_wide(prm, U2, fp)
    else:
        U = np.zeros((NP,) + (n + 1,) * 3)
        bnd = np.zeros((n + 1,) * 3, dtype=bool)
        bnd[0, :, :] = bnd[-1, :, :] = bnd[:, 0, :] = bnd[:, -1, :] = bnd[:, :, 0] = bnd[:, :, -1] = True
        bl = np.argwhere(bnd)
        gb = origins[:, None, :] + bl[None, :, :]  # (NP, |bnd|, 3)
        U[:, bnd] = phiB[gmap[gb[..., 0], gb[..., 1], gb[..., 2]]]
        U = dirichlet_solve(prm, U, fp)
    if prm.correction:
        U += prm.c2 * h * h * fp
    phi = np.zeros((N + 1,) * 3)
    for i in range(NP):
        o = origins[i]
        phi[o[0]:o[0] + n + 1, o[1]:o[1] + n + 1, o[2]:o[2] + n + 1] = U[i]

    if stages is not None:
        # local fields at the coarse points of each field box, (patches, points)
        stages["coarse_samples"] = PHI[phi_set.index(coarse_field)].T.copy()
        stages["moments"] = Cmom.T.copy()
        stages["FH"] = FH
        stages["FH_lo"] = flo
        stages["phiH"] = phiH
        stages["phiH_lo"] = olo
        stages["face_nodes"] = gface
        stages["phiB"] = phiB
        if wide:
            stages["outer_nodes"] = gout
            stages["phiB_outer"] = phiB_out
    return phi


def coarse_level_params(prm: Params):
    """Sec. 5 (R16): origin c0 (in coarse nodes of this level) and parameters
    of the next coarser level's MLC problem."""
    flo, fhi = prm.fh_extent
    olo, ohi = prm.phih_extent
    c0 = min(flo, olo)
    top = max(fhi, ohi)
    Nc = prm.n * (-(-(top - c0 + 1) // prm.n))  # whole patches; node c0 + Nc carries no charge
    cs = prm.s if prm.coarse_s is None else prm.coarse_s
    child = Params(N=Nc, n=prm.n, s=cs, P=prm.P, Q=prm.Q, C=prm.C, beta=prm.beta, b=prm.b,
                   mode=prm.mode, nD=prm.nD, zeta=prm.zeta, levels=prm.levels - 1,
                   h_level=prm.H, correction=False, coarse_s=prm.coarse_s)
    assert child.g_beta == prm.g_beta or prm.mode == "mlc0"
    return c0, child


def coarse_level_solve(prm: Params, FH: np.ndarray, G1: np.ndarray) -> np.ndarray:
    """phi^H on [olo, ohi]^3 by the MLC solve of F^H on the coarser level (R16)."""
    flo, _ = prm.fh_extent
    olo, ohi = prm.phih_extent
    c0, child = coarse_level_params(prm)
    fc = np.zeros((child.N + 1,) * 3)
    a, nf = flo - c0, FH.shape[0]
    fc[a:a + nf, a:a + nf, a:a + nf] = FH
    phic = mlc_solve(child, fc, G1=G1)
    a, no = olo - c0, ohi - olo + 1
    return phic[a:a + no, a:a + no, a:a + no].copy()


# ---------------------------------------------------------------------------
# Patch indexing of Sec. 4 by membership tests (regions are closed boxes, R5)
# ---------------------------------------------------------------------------

def _members_1d(lo: int, hi: int, count: int, c: int, step: int) -> list:
    """Patch indices i (one axis) with c in [step i + lo, step i + hi]."""
    return [i for i in range(count) if step * i + lo <= c <= step * i + hi]


def face_patch_index(prm: Params, nodes: np.ndarray):
    """For each face-lattice node g (rows of ``nodes``), the patches i with g in
    Omega_beta(i) = G(Omega_i, g_beta) in ascending linear index, as entries
    2 i + 0 if g is in Omega_alpha(i) as well and 2 i + 1 otherwise (the sums
    of eq. philocmlcII).  Boxes are products of intervals, so membership is
    tested axis by axis.  Returns (offsets, entries), node k owning
    entries[offsets[k]:offsets[k+1]]."""
    n, npp = prm.n, prm.np_
    alo, ahi = prm.alpha_box
    blo, bhi = prm.beta_box
    offs = [0]
    ent = []
    for g in np.asarray(nodes, dtype=np.int64):
        per_b = [_members_1d(blo, bhi, npp, int(g[d]), n) for d in range(3)]
        per_a = [_members_1d(alo, ahi, npp, int(g[d]), n) for d in range(3)]
        for i0 in per_b[0]:
            for i1 in per_b[1]:
                for i2 in per_b[2]:
                    inA = i0 in per_a[0] and i1 in per_a[1] and i2 in per_a[2]
                    ent.append(2 * ((i0 * npp + i1) * npp + i2) + (0 if inA else 1))
        offs.append(len(ent))
    return np.array(offs, dtype=np.int64), np.array(ent, dtype=np.int64)


def coarse_patch_index(prm: Params):
    """For each coarse node k of the F^H extent ([k0][k1][k2] order), the
    patches i with k in C(Omega_beta(i)) in ascending linear index, as entries
    2 i + 0 if k is in C(Omega_alpha(i)) as well and 2 i + 1 otherwise (the
    two cases of eq. FDLD).  Returns (offsets, entries)."""
    q, npp = prm.n // 4, prm.np_
    calo, cahi = prm.c_alpha
    cblo, cbhi = prm.c_beta
    flo, fhi = prm.fh_extent
    offs = [0]
    ent = []
    for k in box_points(flo, fhi):
        per_b = [_members_1d(cblo, cbhi, npp, int(k[d]), q) for d in range(3)]
        per_a = [_members_1d(calo, cahi, npp, int(k[d]), q) for d in range(3)]
        for i0 in per_b[0]:
            for i1 in per_b[1]:
                for i2 in per_b[2]:
                    inA = i0 in per_a[0] and i1 in per_a[1] and i2 in per_a[2]
                    ent.append(2 * ((i0 * npp + i1) * npp + i2) + (0 if inA else 1))
        offs.append(len(ent))
    return np.array(offs, dtype=np.int64), np.array(ent, dtype=np.int64)


def dirichlet_solve(prm: Params, U: np.ndarray, fp: np.ndarray) -> np.ndarray:
    """Solve Delta^h u = f on the patch interiors with u = U on the patch
    boundaries (eq. last_step_fulldiscr) by dense DST-I matrices.

    U, fp: (patches, n+1, n+1, n+1); returns U with the interior filled."""
    n, h = prm.n, prm.h
    lap = stencil(prm.Q)
    rhs = fp[:, 1:-1, 1:-1, 1:-1].copy()
    for (s0, s1, s2), c in lap:
        rhs -= (c / (h * h)) * U[:, 1 + s0:n + s0, 1 + s1:n + s1, 1 + s2:n + s2]
    k = np.arange(1, n)
    Sm = np.sin(np.pi * np.outer(k, k) / n)  # DST-I matrix, Sm @ Sm = (n/2) I
    cth = np.cos(np.pi * k / n)
    lam = symbol(prm.Q, cth[:, None, None], cth[None, :, None], cth[None, None, :]) / (h * h)

    def dst3(x):
        x = np.einsum("ai,pijk->pajk", Sm, x)
        x = np.einsum("bj,pajk->pabk", Sm, x)
        return np.einsum("ck,pabk->pabc", Sm, x)

    out = U.copy()
    out[:, 1:-1, 1:-1, 1:-1] = dst3(dst3(rhs) / lam[None]) * (2.0 / n) ** 3
    return out


def dirichlet_solve_wide(prm: Params, U: np.ndarray, fp: np.ndarray) -> np.ndarray:
    """R18: Delta^h u = f on the patch interior [1, n-1]^3 of an s = 2
    operator, u = U on the two boundary layers (the closed faces and the layer
    one node outside them), by a sparse LU factorisation of the operator on
    the interior nodes (eq. last_step_fulldiscr with the second layer).

    U: (patches, n+3, n+3, n+3) over the relative nodes [-1, n+1]^3 (entries
    off the two layers are never read); fp: (patches, n+1, n+1, n+1) over
    [0, n]^3.  Returns u on [0, n]^3 with the faces taken from U."""
    import scipy.sparse
    import scipy.sparse.linalg
    n, h = prm.n, prm.h
    m = n - 1
    lap = stencil(prm.Q)
    for off, _ in lap:  # only offsets the two layers hold: at most one component of size 2
        assert sum(abs(c) == 2 for c in off) <= 1
    idx = np.arange(m ** 3).reshape(m, m, m)
    rows, cols, vals = [], [], []
    for (s0, s1, s2), c in lap:
        a0, a1 = max(0, -s0), min(m, m - s0)
        b0, b1 = max(0, -s1), min(m, m - s1)
        c0, c1 = max(0, -s2), min(m, m - s2)
        rows.append(idx[a0:a1, b0:b1, c0:c1].ravel())
        cols.append(idx[a0 + s0:a1 + s0, b0 + s1:b1 + s1, c0 + s2:c1 + s2].ravel())
        vals.append(np.full(rows[-1].size, c / (h * h)))
    A = scipy.sparse.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(m ** 3, m ** 3))
    Ub = U.copy()
    Ub[:, 2:m + 2, 2:m + 2, 2:m + 2] = 0.0  # boundary-layer values only
    rhs = fp[:, 1:-1, 1:-1, 1:-1].copy()
    for (s0, s1, s2), c in lap:
        rhs -= (c / (h * h)) * Ub[:, 2 + s0:m + 2 + s0, 2 + s1:m + 2 + s1, 2 + s2:m + 2 + s2]
    lu = scipy.sparse.linalg.splu(A)
    u = lu.solve(rhs.reshape(rhs.shape[0], -1).T).T
    out = U[:, 1:n + 2, 1:n + 2, 1:n + 2].copy()
    out[:, 1:n, 1:n, 1:n] = u.reshape(-1, m, m, m)
    return out


def plain_solution(prm: Params, f_closed: np.ndarray, G1: np.ndarray | None = None) -> np.ndarray:
    """The plain definition G^h * f^h + C2 h^2 f^h on [0,N]^3 (eq. msCorr4),
    by a global direct sum."""
    N, h = prm.N, prm.h
    if G1 is None:
        G1 = dgf_octant(prm.Q, prm.nD, prm.zeta)
    conv = direct_sum(G1, f_closed, (0, 0, 0), (0, 0, 0), (N + 1,) * 3, h * h)
    return conv + prm.c2 * h * h * f_closed


def solve_open(prm: Params, f: np.ndarray, **kw) -> np.ndarray:
    """Oracle in the library's array convention: f on [0,N)^3 -> phi on [0,N)^3."""
    N = prm.N
    phi = mlc_solve(prm, pad_charge(np.asarray(f, dtype=np.float64)), **kw)
    return phi[:N, :N, :N]
