"""GPU tests of the batched entry point and the continuous-batching server.

Batch: problems of several patch geometries and tiers in one mlc_batch_solve
call (per-patch steps of each geometry group share launches, captured in a
CUDA graph).  Each result must equal the problem's standalone solve exactly
(same kernels, same tables) and match the CPU oracle: relative max-norm
<= 1e-12 for the FP64-accurate tiers, <= 1e-6 for the split tiers.  Server:
requests of both operators and all tiers are merged into batched launches;
each result is the same alone and in the mix, and matches the oracle within
the same tolerances.
"""
import numpy as np
import pytest

from oracle import mlc_oracle as O
from paper_1702_08111_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64, SPLIT, DF, SPLIT_DF = 0, 1, 2, 3
F32_TIERS = (SPLIT, SPLIT_DF)


def tol_of(tier):
    return 1e-6 if tier in F32_TIERS else 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def G():
    return {4: O.dgf_octant(4, 128, 2), 6: O.dgf_octant(6, 128, 2)}


_ORACLE = {}


def oracle_phi(G, N, n, s, Q, seed, nb):
    """Oracle solve of the seeded bump charge (FP64 samples; the split tiers
    solve the same samples rounded to FP32)."""
    key = (N, n, s, Q, seed, nb)
    if key not in _ORACLE:
        f = I.sample_bumps(N, I.draw_bumps(nb, seed))
        _ORACLE[key] = O.solve_open(O.Params(N=N, n=n, s=s, Q=Q), f, G1=G[Q])
    return _ORACLE[key]


def charge(torch, N, seed, nb, tier):
    f = I.sample_bumps(N, I.draw_bumps(nb, seed))
    return torch.from_numpy(f.astype(np.float32) if tier in F32_TIERS else f).cuda()


def relmax(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("tier", [FP64, SPLIT, DF, SPLIT_DF])
def test_batch_equals_standalone(torch_cuda, tier):
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    sides = [32, 64, 48, 96, 32, 80]
    plans = [mlc.Plan(N, 16, 16, 4, 4, tier=tier) for N in sides]
    fs = [charge(torch, N, 900 + k, 1 + k % 5, tier) for k, N in enumerate(sides)]
    alone = [p.solve(f).clone() for p, f in zip(plans, fs)]
    phis = [torch.empty_like(a) for a in alone]
    mlc.batch_solve(plans, fs, phis)
    mlc.batch_solve(plans, fs, phis)  # graph replay
    torch.cuda.synchronize()
    for a, b in zip(alone, phis):
        assert torch.equal(a, b)
    for p in plans:
        p.status()
    ch = mlc.batch_choice(plans, fs, phis)
    assert ch["branches"] in (1, 4, 16)


# config 4's shape: uneven problems, patch 8 for side 32, 16 otherwise,
# support = patch side, Q = 4, 1..16 bumps per problem
MIXED = [(32, 8, 8, 4001, 3), (64, 16, 16, 4002, 9), (48, 16, 16, 4003, 1), (96, 16, 16, 4004, 16),
         (32, 8, 8, 4005, 7), (64, 16, 16, 4006, 5)]


@pytest.mark.parametrize("tier", [FP64, SPLIT, DF, SPLIT_DF])
def test_batch_mixed_geometry_vs_oracle(torch_cuda, G, tier):
    """n = 8 and n = 16 problems (two geometry groups) in one batch call:
    every problem against the oracle element by element, and bit-identical
    to its standalone solve."""
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    plans = [mlc.Plan(N, n, s, 4, 4, tier=tier) for N, n, s, _, _ in MIXED]
    fs = [charge(torch, N, seed, nb, tier) for N, _, _, seed, nb in MIXED]
    phis = [torch.empty((N,) * 3, dtype=torch.float64, device="cuda") for N, *_ in MIXED]
    mlc.batch_solve(plans, fs, phis)
    torch.cuda.synchronize()
    for p in plans:
        p.status()
    for (N, n, s, seed, nb), p, f, phi in zip(MIXED, plans, fs, phis):
        ref = oracle_phi(G, N, n, s, 4, seed, nb)
        err = relmax(phi.cpu().numpy(), ref)
        assert err <= tol_of(tier), (N, n, tier, err)
        assert torch.equal(p.solve(f), phi)


def test_batch_mixed_tiers_and_errors(torch_cuda):
    """Problems of different tiers share one call (one group per tier); a plan
    may appear only once per call."""
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    specs = [(32, FP64), (40, SPLIT), (32, DF), (48, SPLIT_DF)]
    plans = [mlc.Plan(N, 8, 8, 4, 4, tier=t) for N, t in specs]
    fs = [charge(torch, N, 300 + k, 2, t) for k, (N, t) in enumerate(specs)]
    alone = [p.solve(f).clone() for p, f in zip(plans, fs)]
    phis = [torch.empty_like(a) for a in alone]
    mlc.batch_solve(plans, fs, phis)
    torch.cuda.synchronize()
    for a, b in zip(alone, phis):
        assert torch.equal(a, b)
    with pytest.raises(mlc.MLCError) as e:
        mlc.batch_solve([plans[0], plans[0]], [fs[0], fs[0]], [phis[0], torch.empty_like(phis[0])])
    assert e.value.status == 1


# (N, Q, tier, bumps): both operators, all tiers; oracle-sized problems first
SERVE = [(64, 4, FP64, 3), (48, 6, SPLIT, 5), (64, 6, DF, 2), (32, 4, SPLIT_DF, 1), (48, 4, DF, 4),
         (64, 4, SPLIT, 6), (48, 6, FP64, 2), (64, 6, SPLIT_DF, 8),
         (96, 4, SPLIT_DF, 7), (80, 4, DF, 3), (112, 6, FP64, 2), (96, 6, SPLIT, 4)]


def test_server_results_same_alone_and_in_mix(torch_cuda, G):
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    reqs = []
    for k, (N, Q, tier, nb) in enumerate(SERVE):
        reqs.append((N, Q, tier, nb, 20 + k, charge(torch, N, 20 + k, nb, tier)))
    srv = mlc.Server(64 << 30, max_batch=4)
    outs, tickets = [], []
    for N, Q, tier, nb, seed, f in reqs:
        phi = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
        outs.append(phi)
        tickets.append(srv.enqueue(f, phi, N, 16, 16, 4, Q, tier=tier))
    for t in tickets:
        st, l, q = srv.wait(t, 120000)
        assert st == 0
        assert l >= q >= 0
    srv.close()
    for (N, Q, tier, nb, seed, f), phi in zip(reqs, outs):
        alone = mlc.Plan(N, 16, 16, 4, Q, tier=tier).solve(f)
        torch.cuda.synchronize()
        assert torch.equal(phi, alone)
        if N <= 64:  # oracle-sized requests: against the oracle
            ref = oracle_phi(G, N, 16, 16, Q, seed, nb)
            err = relmax(phi.cpu().numpy(), ref)
            assert err <= tol_of(tier), (N, Q, tier, err)


def test_server_admission_and_timeout(torch_cuda):
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    srv = mlc.Server(1 << 20, max_batch=2)  # 1 MiB: nothing fits
    f = charge(torch, 64, 5, 2, FP64)
    phi = torch.empty_like(f)
    with pytest.raises(mlc.MLCError) as e:
        srv.enqueue(f, phi, 64, 16, 16, 4, 4)
    assert e.value.status == 5
    with pytest.raises(mlc.MLCError) as e:
        srv.wait(12345, 20)  # never issued: the wait runs out
    assert e.value.status == 6
    srv.close()


def test_caller_scratch_and_small_launch_groups(torch_cuda):
    """A plan solving with caller-owned scratch, and with local convolutions
    in launch groups of 5 patches (a ragged last group), equals the default
    solve bit for bit."""
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    f = charge(torch, 64, 77, 4, FP64)
    ref = mlc.Plan(64, 16, 16, 4, 4).solve(f).clone()
    p = mlc.Plan(64, 16, 16, 4, 4, conv_chunk=5)
    buf = torch.empty(p.scratch_bytes() // 8 + 64, dtype=torch.float64, device="cuda")
    p.set_scratch(buf)
    out = p.solve(f)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    with pytest.raises(mlc.MLCError) as e:
        p.set_scratch(buf[:8])
    assert e.value.status == 1
    p.set_scratch(None)
    assert torch.equal(p.solve(f), ref)


def test_batch_new_arrays_reuse_the_graph(torch_cuda):
    """A batch solved again with other f / phi arrays for the same plans
    replays the tuned graph with rewritten problem records: every result
    equals the standalone solve of the new charge, on another stream too."""
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    plans = [mlc.Plan(32, 8, 8, 4, 4), mlc.Plan(64, 16, 16, 4, 6, tier=SPLIT)]
    tiers = [FP64, SPLIT]
    Ns = [32, 64]
    for rnd, stream in enumerate([None, torch.cuda.Stream(), None]):
        fs = [charge(torch, N, 40 + 10 * rnd + k, 3, t) for k, (N, t) in enumerate(zip(Ns, tiers))]
        phis = [torch.empty((N,) * 3, dtype=torch.float64, device="cuda") for N in Ns]
        mlc.batch_solve(plans, fs, phis, stream=stream)
        torch.cuda.synchronize()
        choice = mlc.batch_choice(plans, fs, phis)
        if rnd == 0:
            first = choice
        assert choice == first  # tuned once for the set of plans
        for p, f, ph in zip(plans, fs, phis):
            assert torch.equal(ph, p.solve(f).clone())
