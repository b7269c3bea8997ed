"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks one component of oracle/mlc_oracle.py against something
other than itself: exact identities of the stencils (App. A.1), the defining
equations of the DGF (Sec. 2 eq. dgf), a library convolution, exactness of
Boole's rule and of Lagrange interpolation, closed-form potentials (Sec. 7.1),
and the error behaviour the analysis predicts (Sec. 4.2, eq. finemesherrorMLC).
"""
import math

import numpy as np
import pytest
import scipy.signal

from oracle import closed_forms as CF
from oracle import mlc_oracle as O
from paper_1702_08111_gb300 import inputs as I

ND = 32  # small DGF tables keep the CPU suite fast


@pytest.fixture(scope="module")
def G4():
    return O.dgf_octant(4, ND, 2)


@pytest.fixture(scope="module")
def G6():
    return O.dgf_octant(6, ND, 2)


# ---------------------------------------------------------------- stencils

@pytest.mark.parametrize("Q", [4, 6])
def test_stencil_sums_and_quadratics(Q):
    st = O.stencil(Q)
    assert len(st) == (19 if Q == 4 else 27)
    assert abs(sum(c for _, c in st)) < 1e-14
    h = 0.1
    x = np.arange(7) * h
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    # Mehrstellen operators are exact on quadratics: Delta x^2 = 2, Delta xy = 0
    assert np.allclose(O.apply_laplacian(X * X, Q, h), 2.0, atol=1e-11)
    assert np.allclose(O.apply_laplacian(Z * Z + Y * Y, Q, h), 4.0, atol=1e-11)
    assert np.allclose(O.apply_laplacian(X * Y, Q, h), 0.0, atol=1e-11)


@pytest.mark.parametrize("Q", [4, 6])
def test_symbol_expansion(Q):
    # along an axis: lambda(theta) = -theta^2 + theta^4/12 + O(theta^6) (C2 = 1/12, Sec. 2)
    for th in [1e-2, 2e-2]:
        lam = O.symbol(Q, math.cos(th), 1.0, 1.0)
        assert abs(lam - (-th ** 2 + th ** 4 / 12)) < 5e-3 * th ** 6 * 100


@pytest.mark.parametrize("Q", [4, 6])
def test_fourth_order_truncation_error_is_c2_term(Q):
    # tau = (h^2/12) Delta Delta phi + O(h^4) (App. A.1): check on phi = x^4
    for h in [0.05, 0.025]:
        x = np.arange(5) * h + 0.3
        X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
        L = O.apply_laplacian(X ** 4, Q, h)
        tau = L - 12 * X[1:-1, 1:-1, 1:-1] ** 2
        assert np.allclose(tau, (h * h / 12) * 24, rtol=1e-6, atol=1e-9)


# ---------------------------------------------------------------- DGF

@pytest.mark.parametrize("Q", [4, 6])
def test_dgf_residual_is_delta(Q, G4, G6):
    G = G4 if Q == 4 else G6
    # even extension of the octant to [-ND, ND]^3
    full = np.concatenate([G[:0:-1], G], axis=0)
    full = np.concatenate([full[:, :0:-1], full], axis=1)
    full = np.concatenate([full[:, :, :0:-1], full], axis=2)
    r = O.apply_laplacian(full, Q, 1.0)
    c = ND - 1
    r[c, c, c] -= 1.0
    assert np.abs(r).max() <= 1e-12


def test_dgf_symmetry_and_far_field(G4, G6):
    for G in (G4, G6):
        assert np.array_equal(G, np.transpose(G, (1, 0, 2))) or np.allclose(G, np.transpose(G, (1, 0, 2)), rtol=0, atol=1e-15)
        assert np.allclose(G, np.transpose(G, (2, 1, 0)), rtol=0, atol=1e-15)
        # G -> -1/(4 pi |g|): relative deviation shrinks with distance
        dev = [abs(G[k, 0, 0] * 4 * math.pi * k + 1.0) for k in (4, 8, 16)]
        assert dev[0] > dev[1] > dev[2] and dev[2] < 2e-3


def test_dgf_boundary_error_order():
    # App. A.1: replacing the discrete BCs by the exact kernel costs O((zeta n)^-4);
    # compare tables at nD = 8, 16, 32 on the common octant [0, 4]^3
    a = O.dgf_octant(4, 8, 2)[:5, :5, :5]
    b = O.dgf_octant(4, 16, 2)[:5, :5, :5]
    c = O.dgf_octant(4, ND, 2)[:5, :5, :5]
    e1 = np.abs(a - c).max()
    e2 = np.abs(b - c).max()
    assert e1 / e2 > 8.0


# ---------------------------------------------------------------- direct sums

def test_direct_sum_matches_library_convolution(G4):
    rng = np.random.default_rng(0)
    src = rng.standard_normal((5, 6, 7))
    full = np.concatenate([G4[:0:-1], G4], axis=0)
    full = np.concatenate([full[:, :0:-1], full], axis=1)
    full = np.concatenate([full[:, :, :0:-1], full], axis=2)
    ref = scipy.signal.fftconvolve(src, full, mode="full")  # index of lag 0 at ND
    out = O.direct_sum(G4, src, (3, -2, 1), (0, -4, 2), (6, 5, 4), 0.5)
    for a in range(6):
        for b in range(5):
            for c in range(4):
                o = (0 + a, -4 + b, 2 + c)
                idx = (o[0] - 3 + ND, o[1] + 2 + ND, o[2] - 1 + ND)
                assert abs(out[a, b, c] - 0.5 * ref[idx]) < 1e-12


def test_green_matrix_matches_direct_sum(G4):
    rng = np.random.default_rng(1)
    src = rng.standard_normal((3, 4, 5))
    pts = rng.integers(-6, 9, size=(40, 3))
    sp = O.box_points(0, 0)  # placeholder for shape
    s0, s1, s2 = np.meshgrid(np.arange(3), np.arange(4), np.arange(5), indexing="ij")
    sp = np.stack([s0, s1, s2], -1).reshape(-1, 3)
    v = O.green_matrix(G4, pts, sp) @ src.reshape(-1)
    for a, p in enumerate(pts):
        d = O.direct_sum(G4, src, (0, 0, 0), tuple(p), (1, 1, 1), 1.0)[0, 0, 0]
        assert abs(v[a] - d) < 1e-13


# ---------------------------------------------------------------- quadrature & Legendre

def test_boole_exact_to_degree_five():
    n, h = 16, 0.01
    w = O.boole_weights_1d(n, h)
    x = np.arange(n + 1) * h
    Lx = n * h
    for k in range(6):
        assert abs(w @ x ** k - Lx ** (k + 1) / (k + 1)) < 1e-14 * max(1, Lx ** (k + 1))
    assert abs(w @ x ** 6 - Lx ** 7 / 7) > 1e-18


def test_legendre_orthonormal():
    prm = O.Params(N=32, n=8, s=8)
    xs, ws = np.polynomial.legendre.leggauss(12)
    idx = O.legendre_index(4)
    assert len(idx) == 20
    # exact inner products on [-R, R]^3 by tensor Gauss rule
    vals = {k: O.legendre_1d(k, xs) for k in range(4)}
    for p in idx:
        for q in idx:
            ip = 1.0
            for d in range(3):
                ip *= np.sum(ws * vals[p[d]] * vals[q[d]])
            assert abs(ip - (1.0 if p == q else 0.0)) < 1e-13
    # the R^{-3/2} factor makes the Boole-rule moment of Q^0 itself equal 1
    M = O.moment_matrix(prm)
    Lp = O.legendre_patch(prm)
    assert abs(M[0] @ Lp[0] - 1.0) < 1e-12


def test_projection_reproduces_quadratics():
    # P(pi) = pi for polynomials of degree < P (Sec. 3.2); Boole is exact here
    prm = O.Params(N=32, n=8, s=8)
    m = O.box_points(0, prm.n) * prm.h
    f = 0.7 - 2 * m[:, 0] + m[:, 1] * m[:, 2] + 3 * m[:, 2] ** 2
    c = O.moment_matrix(prm) @ f
    back = c @ O.legendre_patch(prm)
    assert np.abs(back - f).max() < 1e-12


# ---------------------------------------------------------------- interpolation

@pytest.mark.parametrize("b", [2, 3])
def test_interpolant_exact_on_degree_2b_plus_1(b):
    prm = O.Params(N=64, n=16, s=16, b=b, Q=4 if b == 2 else 6)
    rng = np.random.default_rng(b)
    nodes = np.array([[16, 5, 7], [32, 18, 33], [9, 16, 13], [22, 31, 48], [48, 48, 5], [0, 2, 16]])
    P, W = O.stencils_for(prm, nodes)
    coef = rng.standard_normal((2 * b + 2, 2 * b + 2))

    def poly(p):  # per-axis degree <= 2b+1 in two in-plane coordinates, linear in the third
        x, y, z = p[..., 0] / 64.0, p[..., 1] / 64.0, p[..., 2] / 64.0
        s = 0.0
        for i in range(2 * b + 2):
            for j in range(2 * b + 2):
                s = s + coef[i, j] * (x + 0.1 * z) ** i * (y - 0.2 * z) ** j
        return s

    for a, g in enumerate(nodes):
        # the interpolated function restricted to the face plane of g
        val = np.sum(W[a] * poly(4 * P[a]))
        assert abs(val - poly(g)) < 1e-9 * max(1.0, abs(poly(g)))
        assert abs(W[a].sum() - 1.0) < 1e-13
        p1, w1 = O.face_stencil(g, b)
        assert abs(np.sum(w1 * poly(4 * p1)) - val) < 1e-11


# ---------------------------------------------------------------- Dirichlet solve

@pytest.mark.parametrize("Q", [4, 6])
def test_dirichlet_solve_recovers_discrete_solution(Q):
    prm = O.Params(N=32, n=8, s=12, Q=Q)
    rng = np.random.default_rng(3)
    psi = rng.standard_normal((2,) + (prm.n + 1,) * 3)
    f = np.zeros_like(psi)
    for p in range(2):
        f[p, 1:-1, 1:-1, 1:-1] = O.apply_laplacian(psi[p], Q, prm.h)
    U = psi.copy()
    U[:, 1:-1, 1:-1, 1:-1] = 0.0
    out = O.dirichlet_solve(prm, U, f)
    assert np.abs(out - psi).max() < 1e-12 * np.abs(psi).max()


# ---------------------------------------------------------------- closed forms

def test_closed_form_bump_laplacian():
    sp = pytest.importorskip("sympy")
    r, a, A = sp.symbols("r a A", positive=True)
    rho = r / a
    phi_in = a ** 2 * A * (rho ** 2 / 6 - rho ** 4 / 5 + rho ** 6 / 7 - rho ** 8 / 18 + rho ** 10 / 110 - sp.Rational(1, 10))
    phi_out = -sp.Rational(128, 3465) * a ** 2 * A / rho
    lap = sp.simplify(sp.diff(r ** 2 * sp.diff(phi_in, r), r) / r ** 2 - A * (1 - rho ** 2) ** 4)
    assert lap == 0
    assert sp.simplify(sp.diff(r ** 2 * sp.diff(phi_out, r), r)) == 0
    assert sp.simplify((phi_in - phi_out).subs(r, a)) == 0
    assert sp.simplify((sp.diff(phi_in, r) - sp.diff(phi_out, r)).subs(r, a)) == 0
    v = CF.bump_potential_radial(np.array([0.5, 2.0]), 0.3, -0.7)
    assert abs(v[0] - float(phi_in.subs({r: 0.15, a: 0.3, A: -0.7}))) < 1e-15
    assert abs(v[1] - float(phi_out.subs({r: 0.6, a: 0.3, A: -0.7}))) < 1e-15


def test_closed_form_smooth_charge_sec71():
    sp = pytest.importorskip("sympy")
    r = sp.symbols("r", positive=True)
    phi_in = r ** 6 / 42 - r ** 7 / 14 + r ** 8 / 12 - 2 * r ** 9 / 45 + r ** 10 / 110 - sp.Rational(1, 1260)
    phi_out = -1 / (2310 * r)
    assert sp.simplify(sp.diff(r ** 2 * sp.diff(phi_in, r), r) / r ** 2 - (r - r ** 2) ** 4) == 0
    assert sp.simplify((phi_in - phi_out).subs(r, 1)) == 0
    assert sp.simplify((sp.diff(phi_in, r) - sp.diff(phi_out, r)).subs(r, 1)) == 0


def test_closed_form_oscillatory_charge_sec73():
    # Sec. 7.2: the radial Laplacian of the interior potential is the charge,
    # value and slope match the monopole at r = 1 (gamma = 28 pi), the centre
    # value is the r -> 0 limit, and the monopole strength is minus the charge
    # over 4 pi; then the oracle's numpy form against the symbolic one
    sp = pytest.importorskip("sympy")
    r, g = sp.symbols("r gamma", positive=True)
    phi_in = (r ** 6 / 84 - r ** 5 / 30 + r ** 4 / 40 + 60 / g ** 6 - 9 / g ** 4 - sp.Rational(1, 120)
              + 120 / (g ** 6 * r)
              + (-120 / (g ** 6 * r) - 9 / g ** 4 + 300 / g ** 6 + 36 * r / g ** 4 + r ** 2 / (2 * g ** 2)
                 - 30 * r ** 2 / g ** 4 - r ** 3 / g ** 2 + r ** 4 / (2 * g ** 2)) * sp.cos(g * r)
              + (12 / (g ** 5 * r) - 360 / (g ** 7 * r) - 96 / g ** 5 + 120 * r / g ** 5 - 3 * r / g ** 3
                 + 8 * r ** 2 / g ** 3 - 5 * r ** 3 / g ** 3) * sp.sin(g * r))
    phi_out = (-sp.Rational(1, 210) - 12 / g ** 4 + 360 / g ** 6) / r
    f = (r - r ** 2) ** 2 * sp.sin(g * r / 2) ** 2
    lap = sp.diff(r ** 2 * sp.diff(phi_in, r), r) / r ** 2 - f
    assert sp.simplify(sp.expand(sp.expand_trig(lap.rewrite(sp.exp)))) == 0
    gam = 28 * sp.pi
    assert sp.simplify((phi_in - phi_out).subs(r, 1).subs(g, gam)) == 0
    assert sp.simplify((sp.diff(phi_in, r) - sp.diff(phi_out, r)).subs(r, 1).subs(g, gam)) == 0
    assert sp.simplify(sp.limit(phi_in, r, 0) - (-sp.Rational(1, 120) - 6 / g ** 4)) == 0
    q = sp.integrate(r ** 2 * f, (r, 0, 1))  # total charge / (4 pi) in scaled units
    assert sp.simplify((phi_out * r + q).subs(g, gam)) == 0
    Ro = 0.05
    rr = np.array([0.0, 0.013, 0.37, 0.9, 1.0, 1.6])
    v = CF.oscillatory_potential(rr, Ro)
    for k, x in enumerate(rr):
        expr = phi_in.subs(g, gam) if 0 < x < 1 else phi_out.subs(g, gam)
        want = float(-sp.Rational(1, 120) - 6 / gam ** 4) if x == 0 else float(expr.subs(r, x))
        assert abs(v[k] - want / Ro) <= 1e-13 * abs(want / Ro), (x, v[k], want / Ro)


def test_paper_charges_sample_the_sec7_densities():
    # the shared input module's samplers of the Sec. 7.1 / 7.3 charges at
    # hand-picked nodes, and the closed-form potentials on the same grid
    N = 64
    fs = I.paper_smooth_charge(N)
    assert fs[32, 32, 32] == 0.0                                    # r = 0
    r = (8 / 64) / 0.25                                             # node 8 h from the centre
    assert abs(fs[40, 32, 32] - (r - r * r) ** 4) < 1e-16
    assert fs[0, 0, 0] == 0.0
    fo = I.paper_oscillatory_charge(N)
    c = (12, 28, 52)                                                # 3/16, 7/16, 13/16 at N = 64
    assert fo[c] == 0.0
    r = (1 / 64) / 0.05
    want = (r - r * r) ** 2 * np.sin(14 * np.pi * r) ** 2 / 0.05 ** 3
    assert abs(fo[13, 28, 52] - want) <= 1e-12 * abs(want)
    ps = CF.smooth_potential_grid(N)
    assert abs(ps[32, 32, 32] - 0.25 ** 2 * (-1 / 1260)) < 1e-18
    po = CF.oscillatory_potential_grid(N)
    # a centre node: its own charge's centre value plus the other two (exterior) charges
    others = sum(CF.oscillatory_potential(np.array([np.linalg.norm(np.array(c) / 64 - np.array(e)) / 0.05]), 0.05)[0]
                 for e in CF.OSC_CENTRES[1:])
    assert abs(po[c] - ((-1 / 120 - 6 / CF.OSC_GAMMA ** 4) / 0.05 + others)) < 1e-12


# ---------------------------------------------------------------- local field and whole solve

def test_local_field_solves_patch_problem(G4):
    # Delta^h (G^h * f^{i,h}) = f^{i,h} (eq. dgf) everywhere inside the evaluation box
    prm = O.Params(N=32, n=8, s=8, nD=ND)
    rng = np.random.default_rng(5)
    f = rng.standard_normal((prm.n + 1,) * 3)
    src = O.box_points(0, prm.n)
    chi = O.chi_patch(prm.n)
    out = O.box_points(-3, prm.n + 3)
    phi = (O.green_matrix(G4, out, src) * prm.h ** 2 * chi[None, :]) @ f.reshape(-1)
    phi = phi.reshape((prm.n + 7,) * 3)
    lap = O.apply_laplacian(phi, 4, prm.h)
    fx = np.zeros((prm.n + 5,) * 3)
    fx[2:-2, 2:-2, 2:-2] = (chi * f.reshape(-1)).reshape((prm.n + 1,) * 3)
    assert np.abs(lap - fx).max() < 1e-10 * np.abs(fx).max()


@pytest.fixture(scope="module")
def bump32():
    N = 32
    bumps = I.single_bump(radius=0.3)
    return N, bumps, I.sample_bumps(N, bumps, nodes=N + 1)


def test_plain_definition_converges_fourth_order(G4):
    # eq. msCorr4: G^h * f + h^2/12 f = phi + O(h^4)
    errs = []
    for N in (8, 16, 32):
        bumps = I.single_bump(radius=0.45)
        f = I.sample_bumps(N, bumps, nodes=N + 1)
        prm = O.Params(N=N, n=8, s=8, nD=ND)
        phi = O.plain_solution(prm, f, G1=G4)
        ex = CF.bumps_potential(N, bumps, nodes=N + 1)
        errs.append(np.abs(phi - ex).max() / np.abs(ex).max())
    assert 10.0 < errs[1] / errs[2] < 24.0


def test_mlc0_barrier_falls_with_beta(G4, bump32):
    # MLC-0 barrier error O((H/R)^q beta^-q) (eq. finemesherrorMLCaeqabar)
    N, bumps, f = bump32
    plain = O.plain_solution(O.Params(N=N, n=8, s=8, nD=ND), f, G1=G4)
    errs = []
    for s in (12, 16, 24):
        phi = O.mlc_solve(O.Params(N=N, n=8, s=s, nD=ND, mode="mlc0"), f, G1=G4)
        errs.append(np.abs(phi - plain).max() / np.abs(plain).max())
    assert errs[0] > 5 * errs[1] > 25 * errs[2]
    assert errs[2] < 1e-5


@pytest.mark.parametrize("Q", [4, 6])
def test_ring_field_is_exact_for_quadratic_charges(Q, G4, G6):
    # For f of degree <= 2 the Boole moments are exact, P^h(f^{i,h}) = f^{i,h}, so the
    # Legendre ring field equals the local field: MLC(alpha<beta) == MLC-0(beta).
    G = G4 if Q == 4 else G6
    N = 32
    x = np.arange(N + 1) / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    f = 0.3 + X - 2 * Y * Z + Z * Z + X * X * Y
    a = O.mlc_solve(O.Params(N=N, n=8, s=12, Q=Q, b=2, beta=3.0, nD=ND), f, G1=G)
    b = O.mlc_solve(O.Params(N=N, n=8, s=16, Q=Q, b=2, nD=ND, mode="mlc0"), f, G1=G)
    assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()
    # and a charge with a degree-4 part breaks it (the pin can fail)
    f2 = f + 40 * (X - 0.5) ** 4
    a2 = O.mlc_solve(O.Params(N=N, n=8, s=12, Q=Q, b=2, beta=3.0, nD=ND), f2, G1=G)
    b2 = O.mlc_solve(O.Params(N=N, n=8, s=16, Q=Q, b=2, nD=ND, mode="mlc0"), f2, G1=G)
    assert np.abs(a2 - b2).max() > 1e-9 * np.abs(b2).max()


def test_mlc_symmetries_and_linearity(G4, bump32):
    N, bumps, f = bump32
    prm = O.Params(N=N, n=8, s=8, nD=ND)
    phi = O.mlc_solve(prm, f, G1=G4)
    scale = np.abs(phi).max()
    # a centred bump: phi invariant under axis permutations and g -> N - g
    assert np.abs(phi - np.transpose(phi, (1, 0, 2))).max() < 1e-13 * scale
    assert np.abs(phi - np.transpose(phi, (2, 1, 0))).max() < 1e-13 * scale
    assert np.abs(phi - phi[::-1, :, :]).max() < 1e-13 * scale
    assert np.abs(phi - phi[:, :, ::-1]).max() < 1e-13 * scale
    # linearity
    rng = np.random.default_rng(9)
    g = I.sample_bumps(N, I.draw_bumps(3, 11), nodes=N + 1)
    pg = O.mlc_solve(prm, g, G1=G4)
    pfg = O.mlc_solve(prm, f - 0.5 * g, G1=G4)
    assert np.abs(pfg - (phi - 0.5 * pg)).max() < 1e-13 * scale


def test_mlc_close_to_plain_definition(G4):
    # the whole two-level solve with the ring (P=4) stays at the barrier level of Sec. 4.2
    N = 32
    bumps = I.single_bump(radius=0.3)
    f = I.sample_bumps(N, bumps, nodes=N + 1)
    plain = O.plain_solution(O.Params(N=N, n=8, s=8, nD=ND), f, G1=G4)
    phi = O.mlc_solve(O.Params(N=N, n=8, s=12, nD=ND), f, G1=G4)
    err = np.abs(phi - plain).max() / np.abs(plain).max()
    assert err < 2e-3
    phi1 = O.mlc_solve(O.Params(N=N, n=8, s=12, nD=ND, P=1), f, G1=G4)
    err1 = np.abs(phi1 - plain).max() / np.abs(plain).max()
    assert err < err1  # P = 4 improves on the monopole-only P = 1


def test_moments_stage_is_boole_of_charge(G4, bump32):
    N, bumps, f = bump32
    prm = O.Params(N=N, n=8, s=8, nD=ND)
    st = {}
    O.mlc_solve(prm, f, G1=G4, stages=st)
    M = O.moment_matrix(prm)
    i = 21
    o = O.patch_origin(prm, i)
    fp = f[o[0]:o[0] + 9, o[1]:o[1] + 9, o[2]:o[2] + 9].reshape(-1)
    assert np.allclose(st["moments"][i], M @ fp, rtol=0, atol=1e-15)
    # Q^0 moment = total patch charge / sqrt(volume) (Boole)
    w = O.boole_weights_1d(prm.n, prm.h)
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).reshape(-1)
    assert abs(st["moments"][i][0] - (W @ fp) / (2 * prm.R) ** 1.5) < 1e-15


# ---------------------------------------------------------------- patch indexing
def test_face_patch_index_worked_example():
    """N = 32, n = 8, s = 8, Q = 4: g_alpha = 0, g_beta = 8.  Node (8, 3, 4):
    per axis Omega_alpha(i) = [8i, 8i+8] holds 8 for i in {0, 1}, 3 and 4 for
    i = 0; Omega_beta(i) = [8i-8, 8i+16] holds 8 for i in {0, 1, 2}, 3 and 4
    for i in {0, 1}.  So 12 patches, of which (0,0,0) and (1,0,0) in alpha."""
    prm = O.Params(N=32, n=8, s=8, Q=4)
    off, ent = O.face_patch_index(prm, np.array([[8, 3, 4]]))
    assert list(off) == [0, 12]
    # linear index (i0 * 4 + i1) * 4 + i2; entry 2 i + (0 alpha, 1 ring)
    assert list(ent) == [0, 3, 9, 11, 32, 35, 41, 43, 65, 67, 73, 75]


def test_face_patch_index_counts_closed_form():
    """N = 128, n = s = 16, Q = 4: g_alpha = 8, g_beta = 16.  Node (64, 40, 72):
    beta holds it for i0 in 2..5, i1 in 1..3, i2 in 3..5 (36 patches), alpha
    for i0 in 3..4, i1 in 1..3, i2 in 3..5 (18 patches)."""
    prm = O.Params(N=128, n=16, s=16, Q=4)
    off, ent = O.face_patch_index(prm, np.array([[64, 40, 72], [0, 0, 0]]))
    e = ent[off[0]:off[1]]
    assert len(e) == 36 and int((e % 2 == 0).sum()) == 18
    assert np.all(np.diff(e // 2) > 0)  # ascending patch index
    # corner node 0: beta holds it for i in {0, 1} on every axis (16 i - 16 <= 0),
    # alpha only for i = 0 (16 i - 8 <= 0); linear index (i0 * 8 + i1) * 8 + i2
    assert list(ent[off[1]:off[2]]) == [0, 3, 17, 19, 129, 131, 145, 147]


def test_coarse_patch_index_worked_example():
    """N = 32, n = 8, Q = 4: C(Omega_alpha) = [0, 2], C(Omega_beta) = [-2, 4]
    relative to n i / 4 = 2 i; F^H on [-2, 10].  Coarse node (3, 0, -2): beta
    for i0 in {0, 1, 2}, i1 in {0, 1}, i2 = 0; alpha needs 2 i2 <= -2: none."""
    prm = O.Params(N=32, n=8, s=8, Q=4)
    off, ent = O.coarse_patch_index(prm)
    node = ((3 + 2) * 13 + (0 + 2)) * 13 + (-2 + 2)
    assert list(ent[off[node]:off[node + 1]]) == [1, 9, 33, 41, 65, 73]
    assert len(off) == 13 ** 3 + 1


# ---------------------------------------------------------------- multilevel (Sec. 5)

def test_coarse_level_params_worked_example():
    # N = 32, n = 8, Q = 4 (b = 2), MLC-0: s = 12 -> g_alpha = 4, F^H on
    # [floor(-4/4), 3*2 + ceil(12/4)] = [-1, 9], phi^H on [-2, 10]: the coarse
    # problem starts at -2 and needs 13 nodes -> two patches of 8 (N = 16).
    # s = 24 -> g_alpha = 16: F^H on [-4, 12], phi^H on [-2, 10] -> c0 = -4,
    # 17 nodes -> 24.
    for s, c0_want, N_want in ((12, -2, 16), (24, -4, 24)):
        prm = O.Params(N=32, n=8, s=s, nD=ND, mode="mlc0", levels=3)
        c0, child = O.coarse_level_params(prm)
        assert (c0, child.N) == (c0_want, N_want)
        assert child.h == prm.H and child.levels == 2 and not child.correction
        assert (child.g_alpha, child.g_beta, child.b) == (prm.g_alpha, prm.g_beta, prm.b)


def test_multilevel_mlc0_error_insensitive_to_levels(G4, bump32):
    # Sec. 7.1.2: the MLC-0 error does not depend on the number of levels (Table 8
    # against Table 4); and it still falls with the correction radius
    N, bumps, f = bump32
    plain = O.plain_solution(O.Params(N=N, n=8, s=8, nD=ND), f, G1=G4)
    errs = {}
    for s in (16, 24):
        for L in (2, 3, 4):
            phi = O.mlc_solve(O.Params(N=N, n=8, s=s, nD=ND, mode="mlc0", levels=L), f, G1=G4)
            errs[s, L] = np.abs(phi - plain).max() / np.abs(plain).max()
    for s in (16, 24):
        for L in (3, 4):
            assert errs[s, 2] / 1.5 < errs[s, L] < 1.5 * errs[s, 2], (s, L, errs)
    assert errs[24, 3] < errs[16, 3] / 50


def test_coarse_level_solve_approximates_coarse_convolution(G4, bump32):
    # the level below solves Delta^H phi = F^H by MLC: against the direct sum
    # G^H * F^H its error is that level's own barrier, falling with s
    N, bumps, f = bump32
    diffs = []
    for s in (16, 24):
        prm = O.Params(N=N, n=8, s=s, nD=ND, mode="mlc0", levels=3)
        st = {}
        O.mlc_solve(prm, f, G1=G4, stages=st)
        flo, (olo, ohi) = st["FH_lo"], prm.phih_extent
        no = ohi - olo + 1
        direct = O.direct_sum(G4, st["FH"], (flo,) * 3, (olo,) * 3, (no,) * 3, prm.H * prm.H)
        assert np.array_equal(st["phiH"], O.coarse_level_solve(prm, st["FH"], G4))
        diffs.append(np.abs(st["phiH"] - direct).max() / np.abs(direct).max())
    assert diffs[0] < 1e-4 and diffs[1] < diffs[0] / 5, diffs


def test_coarse_level_takes_coarse_support(G4, bump32):
    # coarse_s sets the coarser levels' support (their inner radius): the
    # coarse problem's parameters carry it, and with coarse_s = s the solve is
    # the same as without it; a larger coarse radius brings the coarse-level
    # solve closer to the direct coarse convolution
    N, bumps, f = bump32
    base = O.Params(N=N, n=8, s=12, nD=ND, mode="mlc0", levels=3)
    same = O.Params(N=N, n=8, s=12, nD=ND, mode="mlc0", levels=3, coarse_s=12)
    wide = O.Params(N=N, n=8, s=12, nD=ND, mode="mlc0", levels=3, coarse_s=24)
    _, child = O.coarse_level_params(wide)
    assert (child.s, child.g_alpha, child.coarse_s) == (24, 16, 24)
    assert np.array_equal(O.mlc_solve(base, f, G1=G4), O.mlc_solve(same, f, G1=G4))
    diffs = []
    for prm in (base, wide):
        st = {}
        O.mlc_solve(prm, f, G1=G4, stages=st)
        olo, ohi = prm.phih_extent
        no = ohi - olo + 1
        direct = O.direct_sum(G4, st["FH"], (st["FH_lo"],) * 3, (olo,) * 3, (no,) * 3, prm.H * prm.H)
        diffs.append(np.abs(st["phiH"] - direct).max() / np.abs(direct).max())
    assert diffs[1] < diffs[0] / 5, diffs
