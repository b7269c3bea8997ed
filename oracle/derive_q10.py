"""Derivation of the q = 10 Mehrstellen operator of the oracle (R18, Sec. 8).

TEST INFRASTRUCTURE (oracle): run by tests/test_oracle_pins.py only.

Sec. 2 states that operators with q = 10 exist in the 5 x 5 x 5 block.  An
operator with the cube's symmetries has one coefficient per orbit of offsets
(named by the sorted absolute components).  Its truncation error on a
harmonic function is the sum over even k of h^(k-2) (1/k!) sum_j a_j (j.grad)^k
phi, and (j.grad)^k p = k! p(j) for a homogeneous polynomial p of degree k, so
q = 10 asks for sum_j a_j p(j) = 0 for every harmonic homogeneous p of degree
4, 6, 8 and 10; with the cube's symmetries only the symmetric harmonic
polynomial of each degree (one each) gives a condition.  With consistency
(sum a_j = 0, sum a_j j_0^2 = 2) that is six linear conditions; this script
solves them exactly on the six orbits with the smallest offsets.
"""
from __future__ import annotations

import itertools

ORBITS = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1), (2, 0, 0), (2, 1, 0)]


def symmetric_harmonics(k: int):
    """The cube-symmetric harmonic homogeneous polynomials of degree k (sympy)."""
    import sympy as sp
    x, y, z = sp.symbols("x y z")
    exps = sorted({tuple(sorted(e, reverse=True)) for e in itertools.product(range(0, k + 1, 2), repeat=3)
                   if sum(e) == k})
    cs = sp.symbols(f"c0:{len(exps)}")
    P = 0
    for c, e in zip(cs, exps):
        P += c * sum(x ** p[0] * y ** p[1] * z ** p[2] for p in set(itertools.permutations(e)))
    lap = sp.diff(P, x, 2) + sp.diff(P, y, 2) + sp.diff(P, z, 2)
    sol = sp.solve(sp.Poly(sp.expand(lap), x, y, z).coeffs(), cs, dict=True)[0]
    Ph = sp.expand(P.subs(sol))
    return [sp.expand(Ph.diff(c)) for c in cs if c not in sol], (x, y, z)


def derive(orbits=ORBITS):
    """Exact coefficients {orbit: Rational} of the q = 10 operator on the orbits."""
    import sympy as sp
    a = sp.symbols(f"a0:{len(orbits)}")
    pts = {o: [p for p in itertools.product(range(-2, 3), repeat=3)
               if tuple(sorted(map(abs, p), reverse=True)) == o] for o in orbits}

    def moment(poly, xyz):
        return sum(a[i] * sum(poly.subs(dict(zip(xyz, p))) for p in pts[o]) for i, o in enumerate(orbits))

    _, xyz = symmetric_harmonics(4)
    conds = [moment(sp.Integer(1), xyz), moment(xyz[0] ** 2, xyz) - 2]
    for k in (4, 6, 8, 10):
        hs, xyz = symmetric_harmonics(k)
        conds += [moment(hp, xyz) for hp in hs]
    sol = sp.solve(conds, a, dict=True)
    if len(sol) != 1 or len(sol[0]) != len(orbits):
        raise ValueError("no unique solution on these orbits")
    return {o: sol[0][a[i]] for i, o in enumerate(orbits)}


if __name__ == "__main__":
    for o, v in derive().items():
        print(o, v)
