"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

FP64-accurate tiers (MLC_TIER_FP64: FP64 arithmetic; MLC_TIER_DF:
double-float arithmetic): relative max-norm difference <= 1e-12 per stage and
for the final potential (the tolerance stated for the FP64 path).  Split
tiers (FP32 local convolutions): <= 1e-6 against the oracle and the FP64 GPU
path.  Both sides build their own DGF for the same (Q, nD = 128, zeta = 2);
the tables are compared first.
"""
import numpy as np
import pytest

from oracle import mlc_oracle as O
from paper_1702_08111_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12


def relmax(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    return torch


def _phiB_from_planes(planes, nodes, n):
    out = np.empty(len(nodes))
    for a, g in enumerate(nodes):
        for d in range(3):
            if g[d] % n == 0:
                u, v = [g[e] for e in range(3) if e != d]
                out[a] = planes[d, g[d] // n, u, v]
                break
    return out


def _check_plane_duplicates(planes, N, n):
    # a node on several face planes must carry one value (computed from g alone)
    np_ = N // n
    for j0 in range(np_ + 1):
        for j1 in range(np_ + 1):
            # edge along axis 2: g0 = j0 n, g1 = j1 n
            a = planes[0, j0, j1 * n, :]
            b = planes[1, j1, j0 * n, :]
            assert np.array_equal(a, b)


FP64, SPLIT, DF, SPLIT_DF = 0, 1, 2, 3
EXACT_TIERS = [FP64, DF]  # FP64-accurate: the 1e-12 bar

_ORACLE = {}


def _oracle(key, prm, f_open, G1):
    """Oracle solve (and its stages) once per case, shared by the tiers."""
    if key not in _ORACLE:
        st = {}
        phi = O.solve_open(prm, f_open, G1=G1, stages=st)
        _ORACLE[key] = (phi, st)
    return _ORACLE[key]


def _run(torch, prm_kw, f_open, stages=True, **plan_kw):
    from paper_1702_08111_gb300 import mlc
    plan = mlc.Plan(**prm_kw, **plan_kw)
    f = torch.from_numpy(f_open).cuda()
    phi = plan.solve(f)
    torch.cuda.synchronize()
    plan.status()  # no kernel-side bounded wait gave up
    res = {"phi": phi.cpu().numpy()}
    if stages:
        res["moments"] = plan.export(mlc.STAGE_MOMENTS)
        res["FH"] = plan.export(mlc.STAGE_FH)
        res["phiH"] = plan.export(mlc.STAGE_PHIH)
        res["phiB"] = plan.export(mlc.STAGE_PHIB)
    res["plan"] = plan
    return res


def _compare(res, prm, f_open, G1, key=None):
    if key is None:
        st = {}
        phi_o = O.solve_open(prm, f_open, G1=G1, stages=st)
    else:
        phi_o, st = _oracle(key, prm, f_open, G1)
    assert relmax(res["moments"], st["moments"]) <= TOL
    assert relmax(res["FH"], st["FH"]) <= TOL
    assert relmax(res["phiH"], st["phiH"]) <= TOL
    pb = _phiB_from_planes(res["phiB"], st["face_nodes"], prm.n)
    assert relmax(pb, st["phiB"]) <= TOL
    _check_plane_duplicates(res["phiB"], prm.N, prm.n)
    err = relmax(res["phi"], phi_o)
    assert err <= TOL, err
    return err


@pytest.fixture(scope="module")
def G4():
    return O.dgf_octant(4, 128, 2)


@pytest.fixture(scope="module")
def G6():
    return O.dgf_octant(6, 128, 2)


@pytest.mark.parametrize("Q", [4, 6])
def test_dgf_table_matches_oracle(torch_cuda, Q, G4, G6):
    from paper_1702_08111_gb300 import mlc
    plan = mlc.Plan(32, 8, 12, 4, Q, b=2)
    T = plan.export(mlc.STAGE_DGF)
    G = G4 if Q == 4 else G6
    L = min(T.shape[0], G.shape[0])
    assert relmax(T[:L, :L, :L], G[:L, :L, :L]) <= 1e-13


@pytest.mark.parametrize("tier", EXACT_TIERS)
def test_single_bump_32(torch_cuda, G4, tier):
    w = I.workload("single_bump_32")
    f = w.charge()
    res = _run(torch_cuda, dict(N=32, n=8, s=8, P=4, Q=4), f, tier=tier)
    _compare(res, O.Params(N=32, n=8, s=8, Q=4), f, G4, key="single_bump_32")


@pytest.mark.parametrize("tier", EXACT_TIERS)
def test_bumps8_128(torch_cuda, G4, tier):
    w = I.workload("bumps8_128")
    f = w.charge()
    res = _run(torch_cuda, dict(N=128, n=16, s=16, P=4, Q=4), f, tier=tier)
    _compare(res, O.Params(N=128, n=16, s=16, Q=4), f, G4, key="bumps8_128")


@pytest.mark.parametrize("tier", EXACT_TIERS)
def test_q6_reduced_64(torch_cuda, G6, tier):
    w = I.workload("bumps8_64_q6")
    f = w.charge()
    res = _run(torch_cuda, dict(N=64, n=16, s=16, P=4, Q=6), f, tier=tier)
    _compare(res, O.Params(N=64, n=16, s=16, Q=6), f, G6, key="bumps8_64_q6")


@pytest.mark.parametrize("tier", EXACT_TIERS)
@pytest.mark.parametrize("kw", [
    dict(N=48, n=16, s=16, P=4, Q=4),            # odd patch count per axis
    dict(N=32, n=8, s=12, P=1, Q=4),             # monopole-only ring (P = 1)
    dict(N=32, n=8, s=16, P=4, Q=4, mode=1),     # MLC-0 (no ring)
    dict(N=40, n=8, s=12, P=3, Q=6, b=2),        # 27-point, b = 2, P = 3
])
def test_variants(torch_cuda, G4, G6, kw, tier):
    kw = dict(kw)
    key = repr(sorted(kw.items()))
    N = kw["N"]
    f = I.sample_bumps(N, I.draw_bumps(5, 100 + N))
    mode = kw.pop("mode", 0)
    b = kw.get("b", None)
    res = _run(torch_cuda, kw, f, mode=mode, tier=tier)
    prm = O.Params(N=N, n=kw["n"], s=kw["s"], P=kw["P"], Q=kw["Q"], b=b,
                   mode="mlc0" if mode else "mlc")
    _compare(res, prm, f, G4 if kw["Q"] == 4 else G6, key=key)


@pytest.mark.parametrize("kw", [
    dict(N=32, n=8, s=8, P=4, Q=4),
    dict(N=128, n=16, s=16, P=4, Q=4),
    dict(N=256, n=16, s=16, P=4, Q=6),
    dict(N=40, n=8, s=12, P=3, Q=6, b=2),
    dict(N=32, n=8, s=16, P=4, Q=4, mode=1),
])
def test_plan_geometry_matches_oracle(torch_cuda, kw):
    # patch decomposition and coarse extents, integer for integer (Sec. 4:
    # g_alpha = s - C b, g_beta = ceil((beta - 1) n / 2), F^H on the union of
    # C(Omega_beta), phi^H on [-b, N/4 + b], Hockney length M >= 2 (n + s))
    from paper_1702_08111_gb300 import mlc
    kw = dict(kw)
    mode = kw.pop("mode", 0)
    b = kw.get("b", None)
    plan = mlc.Plan(**kw, mode=mode)
    info = plan.info
    prm = O.Params(N=kw["N"], n=kw["n"], s=kw["s"], P=kw["P"], Q=kw["Q"], b=b,
                   mode="mlc0" if mode else "mlc")
    assert (info.N, info.n, info.s, info.b) == (prm.N, prm.n, prm.s, prm.b)
    assert (info.g_alpha, info.g_beta) == (prm.g_alpha, prm.g_beta)
    assert (info.fh_lo, info.fh_hi) == tuple(prm.fh_extent)
    assert (info.phih_lo, info.phih_hi) == tuple(prm.phih_extent)
    assert info.npoly == prm.P * (prm.P + 1) * (prm.P + 2) // 6  # |p|_1 <= P - 1 in 3D
    M = 1
    while M < 2 * (prm.n + prm.s):
        M *= 2
    assert info.M == M


def test_zero_charge_gives_zero(torch_cuda):
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    plan = mlc.Plan(32, 8, 8, 4, 4)
    f = torch.zeros((32, 32, 32), dtype=torch.float64, device="cuda")
    phi = plan.solve(f)
    torch.cuda.synchronize()
    assert float(phi.abs().max()) == 0.0


def test_repeat_and_host_path_identical(torch_cuda):
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    w = I.workload("single_bump_32")
    f = torch.from_numpy(w.charge()).cuda()
    plan = mlc.Plan(32, 8, 8, 4, 4)
    a = plan.solve(f).clone()
    b = plan.solve(f).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    fh = f.cpu().pin_memory()
    ph = torch.empty((32, 32, 32), dtype=torch.float64).pin_memory()
    plan.solve_host(fh, ph)
    assert torch.equal(ph, a.cpu())


def test_invalid_arguments(torch_cuda):
    from paper_1702_08111_gb300 import mlc
    for kw in [dict(N=30, n=8, s=8), dict(N=32, n=6, s=8), dict(N=32, n=8, s=4),
               dict(N=32, n=8, s=8, Q=5), dict(N=32, n=8, s=8, C=2)]:
        with pytest.raises(mlc.MLCError) as e:
            mlc.Plan(**kw)
        assert e.value.status == 1
    # legal for the method, not built: a local period above 128, a patch size
    # without a Dirichlet kernel
    for kw in [dict(N=64, n=32, s=36), dict(N=40, n=20, s=8)]:
        with pytest.raises(mlc.MLCError) as e:
            mlc.Plan(**kw)
        assert e.value.status == 2


# ------------------------------------------------------------------ split tiers
SPLIT_TOL = 1e-6


@pytest.mark.parametrize("tier", [SPLIT, SPLIT_DF])
def test_split_tier_matches_fp64_and_oracle(torch_cuda, G6, tier):
    """Split tiers (FP32 charge, FP32 local convolutions and ring sums; FP64 or
    double-float after them) within 1e-6 relative max-norm of the FP64 GPU
    path and of the oracle."""
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    w = I.workload("bumps8_64_q6")
    f32 = w.charge().astype(np.float32)
    f64 = f32.astype(np.float64)
    ps = mlc.Plan(64, 16, 16, 4, 6, tier=tier)
    pd = mlc.Plan(64, 16, 16, 4, 6, tier=FP64)
    a = ps.solve(torch.from_numpy(f32).cuda())
    b = pd.solve(torch.from_numpy(f64).cuda())
    torch.cuda.synchronize()
    a, b = a.cpu().numpy(), b.cpu().numpy()
    e_gpu = relmax(a, b)
    ref = O.solve_open(O.Params(N=64, n=16, s=16, Q=6), f64, G1=G6)
    assert relmax(b, ref) <= TOL
    assert e_gpu <= SPLIT_TOL, e_gpu
    assert relmax(a, ref) <= SPLIT_TOL


@pytest.mark.parametrize("tier", [SPLIT, SPLIT_DF])
def test_split_tier_small_patches_vs_oracle(torch_cuda, G4, tier):
    """n = 8 patches (M = 32 transforms) in the split tiers against the oracle."""
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    w = I.workload("single_bump_32")
    f32 = w.charge().astype(np.float32)
    a = mlc.Plan(32, 8, 8, 4, 4, tier=tier).solve(torch.from_numpy(f32).cuda())
    torch.cuda.synchronize()
    ref = O.solve_open(O.Params(N=32, n=8, s=8, Q=4), f32.astype(np.float64), G1=G4)
    assert relmax(a.cpu().numpy(), ref) <= SPLIT_TOL


def test_split_tier_256_below_discretisation_error(torch_cuda):
    """256^3, 4096 patches, Q = 6, 32 bumps, FP32 charge: both split tiers and
    the double-float tier against the FP64 GPU path (<= 1e-6; <= 1e-12 for
    double-float), the split tiers below the FP64 path's error against the
    closed-form potential."""
    from oracle import closed_forms as CF
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    w = I.workload("bumps32_256_q6")
    f32 = w.charge()
    f64 = f32.astype(np.float64)
    out = {}
    for tier in (FP64, DF, SPLIT, SPLIT_DF):
        p = mlc.Plan(256, 16, 16, 4, 6, tier=tier)
        f = torch.from_numpy(f32 if tier in (SPLIT, SPLIT_DF) else f64).cuda()
        out[tier] = p.solve(f).cpu().numpy()
        del p, f
    b = out[FP64]
    ex = CF.bumps_potential(256, w.bumps)
    e_disc = relmax(b, ex)
    assert relmax(out[DF], b) <= TOL
    for tier in (SPLIT, SPLIT_DF):
        e_split = relmax(out[tier], b)
        assert e_split <= SPLIT_TOL, (tier, e_split)
        assert e_split < e_disc, (tier, e_split, e_disc)


# ------------------------------------------------------------ indexing, failures
def _plane_order_nodes(N, n):
    """Face-plane nodes in the library's [axis][plane][u][v] order."""
    npl = N // n + 1
    u, v = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    u, v = u.reshape(-1), v.reshape(-1)
    out = []
    for axis in range(3):
        for j in range(npl):
            c = np.full_like(u, j * n)
            out.append(np.stack([c, u, v], 1) if axis == 0 else
                       (np.stack([u, c, v], 1) if axis == 1 else np.stack([u, v, c], 1)))
    return np.concatenate(out)


@pytest.mark.parametrize("kw", [dict(N=32, n=8, s=8, Q=4), dict(N=48, n=16, s=16, Q=4),
                                dict(N=128, n=16, s=16, Q=4), dict(N=64, n=16, s=16, Q=6)])
def test_index_arrays_match_oracle(torch_cuda, kw):
    """The patch indexing the boundary and coarse-charge kernels run (per
    face-plane node and per coarse node: the patches whose Omega_beta or
    C(Omega_beta) holds it, ascending, alpha / ring class) equals the oracle's
    membership tests bit for bit."""
    from paper_1702_08111_gb300 import mlc
    plan = mlc.Plan(kw["N"], kw["n"], kw["s"], 4, kw["Q"])
    prm = O.Params(N=kw["N"], n=kw["n"], s=kw["s"], Q=kw["Q"])
    off, ent = plan.export(mlc.STAGE_FACE_INDEX)
    o_off, o_ent = O.face_patch_index(prm, _plane_order_nodes(kw["N"], kw["n"]))
    assert np.array_equal(off, o_off)
    assert np.array_equal(ent, o_ent)
    off, ent = plan.export(mlc.STAGE_COARSE_INDEX)
    o_off, o_ent = O.coarse_patch_index(prm)
    assert np.array_equal(off, o_off)
    assert np.array_equal(ent, o_ent)


@pytest.mark.parametrize("tier", EXACT_TIERS)
def test_coarse_samples_match_oracle(torch_cuda, G4, tier):
    """Local fields phi^{i,h} at the coarse points of every field box (the
    samples Delta^H and the interpolation read) against the oracle's."""
    from paper_1702_08111_gb300 import mlc
    w = I.workload("single_bump_32")
    f = w.charge()
    plan = mlc.Plan(32, 8, 8, 4, 4, tier=tier)
    plan.solve(torch_cuda.from_numpy(f).cuda())
    got = plan.export(mlc.STAGE_COARSE_SAMPLES)
    _, st = _oracle("single_bump_32", O.Params(N=32, n=8, s=8, Q=4), f, G4)
    ref = st["coarse_samples"].reshape(got.shape)
    assert relmax(got, ref) <= TOL


def test_bounded_wait_runs_out_and_reports_timeout(torch_cuda):
    """With the test hook on, the inverse-x kernels' bulk copies are not
    issued: every bounded wait runs out (64 tests), the kernels record it and
    return, and the plan reports TIMEOUT; the next normal solve is correct."""
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    f = torch.from_numpy(I.workload("single_bump_32").charge()).cuda()
    for N, n, s in ((32, 8, 8), (48, 16, 16)):  # M = 32 and M = 64 kernels
        fN = torch.from_numpy(I.sample_bumps(N, I.draw_bumps(2, 5))).cuda() if N != 32 else f
        plan = mlc.Plan(N, n, s, 4, 4)
        ref = plan.solve(fN).clone()
        plan.status()
        plan.set_fault(1)
        plan.solve(fN)
        with pytest.raises(mlc.MLCError) as e:
            plan.status()
        assert e.value.status == 6
        plan.set_fault(0)
        out = plan.solve(fN)
        plan.status()
        assert torch.equal(out, ref)
    with pytest.raises(mlc.MLCError):
        plan.set_fault(7)


def _golden_256():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_bumps32_256_q6_samples.txt")
    scale = None
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#"):
                if "max |phi| =" in line:
                    scale = float(line.split("max |phi| =")[1])
                continue
            a = line.split()
            rows.append((int(a[0]), int(a[1]), int(a[2]), float(a[3])))
    g = np.array([r[:3] for r in rows])
    return g, np.array([r[3] for r in rows]), scale


@pytest.mark.parametrize("tier", [FP64, DF, SPLIT, SPLIT_DF])
def test_full_size_256_against_oracle_samples(torch_cuda, tier):
    """The bench workload at full size (256^3, 4096 patches, Q = 6, FP32-rounded
    charge) in every tier, in the launch configuration bench.py times, against
    the oracle's potential at 4096 seeded nodes (tests/golden, written by
    make_oracle_256_samples.py from oracle/ alone); errors relative to the
    oracle's max |phi| over the whole grid."""
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    g, ref, scale = _golden_256()
    w = I.workload("bumps32_256_q6")
    f32 = w.charge()
    f = f32 if tier in (SPLIT, SPLIT_DF) else f32.astype(np.float64)
    plan = mlc.Plan(256, 16, 16, 4, 6, tier=tier)
    phi = plan.solve(torch.from_numpy(f).cuda())
    torch.cuda.synchronize()
    plan.status()
    got = phi[g[:, 0], g[:, 1], g[:, 2]].cpu().numpy()
    err = float(np.abs(got - ref).max() / scale)
    assert err <= (TOL if tier in EXACT_TIERS else SPLIT_TOL), (tier, err)


def test_set_dgf_uses_the_injected_table(torch_cuda, G4):
    """mlc_plan_set_dgf: the oracle's DGF table injected as data gives the
    oracle's result; a doubled table gives the oracle's result for the doubled
    table (so the injected table, not the library's own, is what the solve
    uses); a table too small for the plan is rejected and leaves it intact."""
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    w = I.workload("single_bump_32")
    f = w.charge()
    ft = torch.from_numpy(f).cuda()
    prm = O.Params(N=32, n=8, s=8, Q=4)
    plan = mlc.Plan(32, 8, 8, 4, 4)
    base = plan.solve(ft).clone()
    L = plan.info.L
    G = np.ascontiguousarray(G4[:L + 1, :L + 1, :L + 1])
    plan.set_dgf(G)
    a = plan.solve(ft).cpu().numpy()
    assert relmax(a, O.solve_open(prm, f, G1=G4)) <= TOL
    plan.set_dgf(2.0 * G)
    b = plan.solve(ft).cpu().numpy()
    ref2 = O.solve_open(prm, f, G1=2.0 * G4)
    assert relmax(b, ref2) <= TOL
    assert relmax(b, a) > 0.5
    with pytest.raises(mlc.MLCError) as e:
        plan.set_dgf(G[:9, :9, :9])
    assert e.value.status == 1
    plan.set_dgf(G)
    assert relmax(plan.solve(ft).cpu().numpy(), base.cpu().numpy()) <= TOL


# ------------------------------------------------------------------ other patch sizes
_SIZES = [
    dict(N=48, n=24, s=12, P=4, Q=4),            # n = 24, local period 128, Legendre ring
    dict(N=48, n=24, s=8, P=4, Q=4, mode=1),     # n = 24, local period 64, MLC-0
    dict(N=48, n=12, s=12, P=4, Q=4),            # n = 12 (generic Dirichlet lines)
    dict(N=16, n=4, s=8, P=2, Q=4),              # n = 4, local period 32
]


@pytest.mark.parametrize("tier", [FP64, DF, SPLIT])
@pytest.mark.parametrize("kw", _SIZES, ids=["n24_ring", "n24_mlc0", "n12", "n4"])
def test_patch_sizes_against_oracle(torch_cuda, G4, kw, tier):
    """Patch sizes 4, 12 and 24 (every Dirichlet instantiation besides 16 and
    32) in the FP64, double-float and split tiers, every stage against the
    oracle (1e-12; 1e-6 for the split tier)."""
    from paper_1702_08111_gb300 import mlc
    kw = dict(kw)
    key = "sizes" + repr(sorted(kw.items()))
    N = kw["N"]
    mode = kw.pop("mode", 0)
    f64 = I.sample_bumps(N, I.draw_bumps(4, 500 + N + kw["n"]))
    if tier == SPLIT:
        f64 = f64.astype(np.float32).astype(np.float64)
        key += "f32"
    torch = torch_cuda
    plan = mlc.Plan(**kw, mode=mode, tier=tier)
    f = torch.from_numpy(f64.astype(np.float32) if tier == SPLIT else f64).cuda()
    phi = plan.solve(f)
    torch.cuda.synchronize()
    plan.status()
    prm = O.Params(N=N, n=kw["n"], s=kw["s"], P=kw["P"], Q=kw["Q"], mode="mlc0" if mode else "mlc")
    phi_o, st = _oracle(key, prm, f64, G4)
    tol = SPLIT_TOL if tier == SPLIT else TOL
    assert relmax(plan.export(mlc.STAGE_MOMENTS), st["moments"]) <= tol
    assert relmax(plan.export(mlc.STAGE_FH), st["FH"]) <= tol
    assert relmax(plan.export(mlc.STAGE_PHIH), st["phiH"]) <= tol
    pb = _phiB_from_planes(plan.export(mlc.STAGE_PHIB), st["face_nodes"], prm.n)
    assert relmax(pb, st["phiB"]) <= tol
    _check_plane_duplicates(plan.export(mlc.STAGE_PHIB), N, prm.n)
    assert relmax(phi.cpu().numpy(), phi_o) <= tol
