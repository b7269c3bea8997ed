"""GPU tests of the batched entry point and the continuous-batching server.

Batch: the per-patch steps of several problems share launches (captured in a
CUDA graph); each result must equal the problem's standalone solve exactly
(same kernels, same tables).  Server: each result is the same alone and in
the mix, within the stated tolerance (exact equality is expected and
checked; the bar is 1e-12 relative for FP64 and 1e-6 for the split tier).
"""
import numpy as np
import pytest

from paper_1702_08111_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    return torch


def _charge(torch, N, seed, f32=False):
    f = I.sample_bumps(N, I.draw_bumps(1 + seed % 5, 900 + seed))
    t = torch.from_numpy(f.astype(np.float32) if f32 else f).cuda()
    return t


@pytest.mark.parametrize("tier", [0, 1, 2, 3])
def test_batch_equals_standalone(torch_cuda, tier):
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    sides = [32, 64, 48, 96, 32, 80]
    plans = [mlc.Plan(N, 16, 16, 4, 4, tier=tier) for N in sides]
    fs = [_charge(torch, N, k, f32=(tier in (1, 3))) for k, N in enumerate(sides)]
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


def test_batch_small_patches_and_errors(torch_cuda):
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    plans = [mlc.Plan(32, 8, 8, 4, 4), mlc.Plan(40, 8, 8, 4, 4)]
    fs = [_charge(torch, 32, 1), _charge(torch, 40, 2)]
    alone = [p.solve(f).clone() for p, f in zip(plans, fs)]
    phis = [torch.empty_like(a) for a in alone]
    mlc.batch_solve(plans, fs, phis)
    torch.cuda.synchronize()
    for a, b in zip(alone, phis):
        assert torch.equal(a, b)
    other = mlc.Plan(64, 16, 16, 4, 4)
    with pytest.raises(mlc.MLCError) as e:
        mlc.batch_solve([plans[0], other], [fs[0], _charge(torch, 64, 3)],
                        [phis[0], torch.empty((64,) * 3, dtype=torch.float64, device="cuda")])
    assert e.value.status == 1
    with pytest.raises(mlc.MLCError) as e:
        mlc.batch_solve([plans[0], plans[0]], [fs[0], fs[0]], [phis[0], torch.empty_like(phis[0])])
    assert e.value.status == 1


def test_server_results_same_alone_and_in_mix(torch_cuda):
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    reqs = []
    for k, (N, Q, tier) in enumerate([(64, 4, 0), (48, 6, 1), (96, 4, 3), (64, 6, 2), (32, 4, 0),
                                      (80, 4, 2), (64, 4, 1), (48, 4, 0), (112, 6, 0), (64, 4, 3)]):
        f = _charge(torch, N, 20 + k, f32=(tier in (1, 3)))
        reqs.append((N, Q, tier, f))
    srv = mlc.Server(64 << 30, max_batch=4)
    outs, tickets = [], []
    for N, Q, tier, f in reqs:
        phi = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
        outs.append(phi)
        tickets.append(srv.enqueue(f, phi, N, 16, 16, 4, Q, tier=tier))
    lat = []
    for t in tickets:
        st, l, q = srv.wait(t, 120000)
        assert st == 0
        assert l >= q >= 0
        lat.append(l)
    srv.close()
    for (N, Q, tier, f), phi in zip(reqs, outs):
        alone = mlc.Plan(N, 16, 16, 4, Q, tier=tier).solve(f)
        torch.cuda.synchronize()
        tol = 1e-12 if tier in (0, 2) else 1e-6
        err = float((phi - alone).abs().max() / alone.abs().max())
        assert err <= tol
        assert torch.equal(phi, alone)


def test_server_admission_and_timeout(torch_cuda):
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    srv = mlc.Server(1 << 20, max_batch=2)  # 1 MiB: nothing fits
    f = _charge(torch, 64, 5)
    phi = torch.empty_like(f)
    with pytest.raises(mlc.MLCError) as e:
        srv.enqueue(f, phi, 64, 16, 16, 4, 4)
    assert e.value.status == 5
    with pytest.raises(mlc.MLCError) as e:
        srv.wait(12345, 20)  # never issued: the wait runs out
    assert e.value.status == 6
    srv.close()
