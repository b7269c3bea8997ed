"""Pins of the oracle's q = 10 operator (Sec. 8; reading R18) against facts
fixed by mathematics and by the paper's own statements about Mehrstellen
operators (Sec. 2): the coefficients annihilate harmonic polynomials up to
degree 11 (exact rational arithmetic) and not degree 12, the h^2 term of the
truncation error is C2 h^2 Delta^2, the symbol is negative away from zero, the
DGF solves its defining equation and the truncation error of the exact kernel
decays like |g|^-(q+3) (Fig. 1 prints -7 and -9 for q = 4 and 6), the
two-layer Dirichlet solve recovers a discrete solution, the 3D interpolation
is exact on polynomials of per-axis degree 2b+1, and the whole solve keeps the
ring identity and the barrier behaviour of Sec. 4.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import mlc_oracle as O
from paper_1702_08111_gb300 import inputs as I

ND = 32


@pytest.fixture(scope="module")
def G10():
    return O.dgf_octant(10, ND, 2)


def _gauss_pow(z, k):
    """(a + i b)^k for Gaussian rationals z = (a, b), exactly."""
    re, im = Fraction(1), Fraction(0)
    for _ in range(k):
        re, im = re * z[0] - im * z[1], re * z[1] + im * z[0]
    return re, im


# isotropic integer vectors u (u.u = 0) as (real, imaginary) parts per axis;
# (u.x)^k is a harmonic homogeneous polynomial of degree k, and these span them
ISOTROPIC = [((1, 0), (0, 1), (0, 0)), ((0, 0), (1, 0), (0, 1)), ((0, 1), (0, 0), (1, 0)),
             ((3, 0), (4, 0), (0, 5)), ((0, 5), (3, 0), (4, 0)), ((4, 0), (0, 5), (3, 0)),
             ((1, 1), (1, -1), (0, 0)), ((1, 2), (2, -1), (0, 0)), ((2, 1), (0, 0), (1, -2))]


def _moment(u, k):
    """sum_j a_j (u . j)^k for the q = 10 operator, exactly (Gaussian rationals)."""
    re, im = Fraction(0), Fraction(0)
    orb = O.STENCIL_ORBITS[10]
    for s0 in range(-2, 3):
        for s1 in range(-2, 3):
            for s2 in range(-2, 3):
                key = tuple(sorted((abs(s0), abs(s1), abs(s2)), reverse=True))
                if key not in orb:
                    continue
                z = (sum(u[d][0] * s for d, s in enumerate((s0, s1, s2))),
                     sum(u[d][1] * s for d, s in enumerate((s0, s1, s2))))
                pr, pi = _gauss_pow(z, k)
                re += orb[key] * pr
                im += orb[key] * pi
    return re, im


def test_q10_annihilates_harmonic_polynomials_to_degree_11():
    for u in ISOTROPIC:
        uu = sum((a * a - b * b) for a, b in u), sum(2 * a * b for a, b in u)
        assert uu == (0, 0)
        for k in range(0, 12):
            assert _moment(u, k) == (0, 0), (u, k)
    # and not to degree 12: q is exactly 10
    assert any(_moment(u, 12) != (0, 0) for u in ISOTROPIC)


def test_q10_consistency_and_c2():
    orb = O.STENCIL_ORBITS[10]
    pts = [(s, orb[tuple(sorted(map(abs, s), reverse=True))])
           for s in np.ndindex(5, 5, 5) for s in [tuple(int(c) - 2 for c in s)]
           if tuple(sorted(map(abs, s), reverse=True)) in orb]
    assert len(pts) == 57
    assert sum(c for _, c in pts) == 0
    assert sum(c * s[0] ** 2 for s, c in pts) == 2
    m4 = sum(c * s[0] ** 4 for s, c in pts)
    m22 = sum(c * s[0] ** 2 * s[1] ** 2 for s, c in pts)
    # D4 = (m4 sum d^4 + 6 m22 sum d_i^2 d_j^2) / 4! must be C2 Delta^2
    assert Fraction(m4, 24) * 2 == Fraction(6 * m22, 24)
    assert O.C2_OF[10] == float(Fraction(m4, 24)) == 2.0 / 35.0
    # tau = C2 h^2 Delta^2 phi + O(h^4) on phi = x^4 (as for L19, L27 in App. A.1)
    for h in (0.05, 0.025):
        x = np.arange(7) * h + 0.3
        X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
        tau = O.apply_laplacian(X ** 4, 10, h) - 12 * X[2:-2, 2:-2, 2:-2] ** 2
        assert np.allclose(tau, O.C2_OF[10] * h * h * 24, rtol=1e-6, atol=1e-9)


def test_q10_derivation_reproduces_coefficients():
    pytest.importorskip("sympy")
    from oracle import derive_q10
    got = derive_q10.derive()
    assert {k: Fraction(int(v.p), int(v.q)) for k, v in got.items()} == O.STENCIL_ORBITS[10]


def test_q10_symbol():
    th = np.linspace(-np.pi, np.pi, 33)
    T0, T1, T2 = np.meshgrid(th, th, th, indexing="ij")
    lam = O.symbol(10, np.cos(T0), np.cos(T1), np.cos(T2))
    # the same eigenvalue written as sum_j a_j cos(j . theta)
    direct = np.zeros_like(T0)
    for (s0, s1, s2), c in O.stencil(10):
        direct += c * np.cos(s0 * T0 + s1 * T1 + s2 * T2)
    assert np.abs(lam - direct).max() < 1e-12
    r2 = T0 ** 2 + T1 ** 2 + T2 ** 2
    off = r2 > 0
    assert lam[off].max() < 0  # invertible away from theta = 0: the DGF exists
    # -theta^2 + C2 theta^4 + O(theta^6) along an axis
    for t in (1e-2, 2e-2):
        assert abs(O.symbol(10, math.cos(t), 1.0, 1.0) - (-t * t + O.C2_OF[10] * t ** 4)) < 1e-2 * t ** 6


def test_q10_dgf_residual_symmetry_far_field(G10):
    L = G10.shape[0] - 1
    F = np.concatenate([G10[:0:-1], G10], 0)
    F = np.concatenate([F[:, :0:-1], F], 1)
    F = np.concatenate([F[:, :, :0:-1], F], 2)
    R = O.apply_laplacian(F, 10, 1.0)
    c = R.shape[0] // 2
    R[c, c, c] -= 1.0
    assert np.abs(R).max() < 1e-12
    assert np.abs(G10 - G10.transpose(1, 0, 2)).max() < 1e-15
    assert np.abs(G10 - G10.transpose(0, 2, 1)).max() < 1e-15
    # G^h - G decays like |g|^-5 (the first multipole the cube allows, l = 4)
    d = [G10[k, 0, 0] + 1.0 / (4 * math.pi * k) for k in (4, 8, 16)]
    assert 24 < d[0] / d[1] < 40 and 24 < d[1] / d[2] < 40
    assert abs(d[2]) < 1e-7


@pytest.mark.parametrize("Q,slope", [(4, -7.0), (6, -9.0), (10, -13.0)])
def test_truncation_error_of_the_kernel_decays_like_q_plus_3(Q, slope):
    # Fig. 1: log|Delta^{h=1} G| against log|g|_inf has slope -7 (L19) and -9
    # (L27); eq. q1 gives -(q+3) in general, -13 for q = 10
    # distances where the FP64 evaluation still resolves |g|^-13
    r = 2
    ks = np.array([5.0, 7.0, 10.0, 14.0])
    vals = []
    for k in ks:
        x = np.arange(-r, r + 1, dtype=np.float64)
        X, Y, Z = np.meshgrid(k + x, 0.37 * k + x, 0.61 * k + x, indexing="ij")
        G = -1.0 / (4 * math.pi * np.sqrt(X * X + Y * Y + Z * Z))
        rr = O.stencil_reach(Q)
        sl = slice(r - rr, r + rr + 1)
        vals.append(abs(O.apply_laplacian(G[sl, sl, sl], Q, 1.0)[0, 0, 0]))
    fit = np.polyfit(np.log(ks), np.log(vals), 1)[0]
    assert abs(fit - slope) < 0.3, fit


def test_wide_dirichlet_recovers_discrete_solution():
    prm = O.Params(N=32, n=8, s=20, Q=10)
    n = prm.n
    rng = np.random.default_rng(5)
    psi = rng.standard_normal((2,) + (n + 3,) * 3)  # nodes [-1, n+1]^3
    f = np.zeros((2,) + (n + 1,) * 3)
    for p in range(2):
        f[p, 1:-1, 1:-1, 1:-1] = O.apply_laplacian(psi[p], 10, prm.h)
    U = psi.copy()
    U[:, 2:-2, 2:-2, 2:-2] = np.nan  # the interior is not read
    # nor are the edges and corners of the outer layer (no offset reaches them)
    for a in (0, -1):
        for b in (0, -1):
            U[:, a, b, :] = U[:, a, :, b] = U[:, :, a, b] = np.nan
    out = O.dirichlet_solve_wide(prm, U, f)
    assert np.abs(out - psi[:, 1:-1, 1:-1, 1:-1]).max() < 1e-11 * np.abs(psi).max()


@pytest.mark.parametrize("b", [2, 5])
def test_3d_interpolant_exact_and_reduces_to_face_stencil(b):
    prm = O.Params(N=32, n=8, s=4 * b, Q=10, b=b)
    rng = np.random.default_rng(b)
    c = rng.standard_normal((2 * b + 2,) * 3)
    deg = 2 * b + 1

    def poly(p):  # per-axis degree <= 2b+1 polynomial in coarse units
        t = np.asarray(p, dtype=np.float64) / 7.0
        v = 0.0
        for i in range(0, deg + 1, 3):
            for j in range(0, deg + 1, 4):
                for k in range(0, deg + 1, 5):
                    v = v + c[i % c.shape[0], j % c.shape[1], k % c.shape[2]] * t[..., 0] ** i * \
                        t[..., 1] ** j * t[..., 2] ** k
        return v
    nodes = np.array([[1, 5, 9], [-1, 3, 4], [7, 8, 13], [9, 2, 6], [15, 17, 8]])
    P, W = O.stencils3_for(prm, nodes)
    got = np.sum(W * poly(P), axis=1)
    assert np.allclose(got, poly(nodes / 4.0), rtol=1e-9, atol=1e-9)
    # on a face plane (a coordinate a multiple of n) it is the face stencil of R4
    fn = np.array([[8, 5, 9], [3, 16, 7]])
    P3, W3 = O.stencils3_for(prm, fn)
    P2, W2 = O.stencils_for(prm, fn)
    for a in range(len(fn)):
        d3 = {tuple(p): 0.0 for p in P3[a]}
        for p, w in zip(P3[a], W3[a]):
            d3[tuple(p)] += w
        d2 = {tuple(p): 0.0 for p in P2[a]}
        for p, w in zip(P2[a], W2[a]):
            d2[tuple(p)] += w
        keys = set(d3) | set(d2)
        assert max(abs(d3.get(k, 0.0) - d2.get(k, 0.0)) for k in keys) < 1e-14


def test_outer_nodes_cover_every_patch_second_layer():
    prm = O.Params(N=32, n=8, s=20, Q=10)
    g = O.outer_nodes(prm)
    have = {tuple(x) for x in g}
    n = prm.n
    for i in range(prm.npatch):
        o = O.patch_origin(prm, i)
        for d in range(3):
            for c in (-1, n + 1):
                for u in range(n + 1):
                    for v in range(0, n + 1, 3):
                        p = [0, 0, 0]
                        e1, e2 = [e for e in range(3) if e != d]
                        p[d], p[e1], p[e2] = c, u, v
                        assert tuple(o + np.array(p)) in have
    assert len(g) == len(have)
    assert np.all(O.offplane_mask(g, n))


def test_q10_ring_field_is_exact_for_quadratic_charges(G10):
    # as for L19 / L27: for f of degree <= 2, MLC(alpha < beta) == MLC-0(beta),
    # here with the second boundary layer and its 3D interpolation in play
    N = 32
    x = np.arange(N + 1) / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    f = 0.3 + X - 2 * Y * Z + Z * Z + X * X * Y
    kw = dict(N=N, n=8, Q=10, b=2, nD=ND)
    a = O.mlc_solve(O.Params(s=12, beta=3.0, **kw), f, G1=G10)
    b = O.mlc_solve(O.Params(s=16, mode="mlc0", **kw), f, G1=G10)
    assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()
    f2 = f + 40 * (X - 0.5) ** 4
    a2 = O.mlc_solve(O.Params(s=12, beta=3.0, **kw), f2, G1=G10)
    b2 = O.mlc_solve(O.Params(s=16, mode="mlc0", **kw), f2, G1=G10)
    assert np.abs(a2 - b2).max() > 1e-9 * np.abs(b2).max()


def test_q10_mlc0_barrier_falls_with_beta(G10):
    # MLC-0 barrier O((H/R)^q beta^-q) (eq. finemesherrorMLCaeqabar) with q = 10
    N = 32
    f = I.sample_bumps(N, I.single_bump(radius=0.3), nodes=N + 1)
    prm0 = O.Params(N=N, n=8, s=8, Q=10, b=2, nD=ND)
    plain = O.plain_solution(prm0, f, G1=G10)
    errs = []
    for s in (12, 16, 20):
        phi = O.mlc_solve(O.Params(N=N, n=8, s=s, Q=10, b=2, nD=ND, mode="mlc0"), f, G1=G10)
        errs.append(np.abs(phi - plain).max() / np.abs(plain).max())
    assert errs[0] > 5 * errs[1] > 25 * errs[2], errs
