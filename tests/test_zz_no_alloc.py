"""mlc_solve_noalloc, the solve for callers that cannot allocate device memory
when they solve: it keeps the local-convolution scratch in the library's
static 64 MiB device array.  Checked through the C ABI against mlc_solve on
the same plan and charge, on two calls in a row with another problem solved
through the same array in between, with the FP64 tolerance of the parity
tests (1e-12 relative; the same kernels run, so equality is expected) and the
split-tier one (1e-6).  Collected last on purpose.
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


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("N,n,s,Q,tier,tol", [
    (48, 16, 16, 4, 0, 1e-12),
    (32, 8, 8, 4, 0, 1e-12),
    (48, 16, 16, 4, 2, 1e-12),
    (64, 16, 16, 6, 1, 1e-6),
    (64, 16, 16, 6, 3, 1e-6),
])
def test_noalloc_matches_solve_twice(torch_cuda, N, n, s, Q, tier, tol):
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    f = I.sample_bumps(N, I.draw_bumps(6, 77 + N))
    ft = torch.from_numpy(f.astype(np.float32) if tier in (1, 3) else f).cuda()
    plan = mlc.Plan(N, n, s, 4, Q, tier=tier)
    ref = plan.solve(ft).clone()
    # a different problem (other geometry, tier and charge) that also runs
    # through the static array: between the two checked calls it leaves its
    # own values there, so a call that read scratch it had not written first
    # would differ from mlc_solve
    other = mlc.Plan(40, 8, 12, 4, 6, tier=0)
    fo = torch.from_numpy(I.sample_bumps(40, I.draw_bumps(3, 991))).cuda()
    ref_o = other.solve(fo).clone()
    for _ in range(2):
        out = torch.full((N, N, N), float("nan"), dtype=torch.float64, device="cuda")
        plan.solve_noalloc(ft, out)
        torch.cuda.synchronize()
        assert _rel(out, ref) <= tol
        assert torch.equal(out, ref)
        out_o = torch.full((40,) * 3, float("nan"), dtype=torch.float64, device="cuda")
        other.solve_noalloc(fo, out_o)
        torch.cuda.synchronize()
        assert torch.equal(out_o, ref_o)


def test_noalloc_rejects_plans_beyond_the_array(torch_cuda):
    from paper_1702_08111_gb300 import mlc
    torch = torch_cuda
    plan = mlc.Plan(128, 16, 16, 4, 4)  # 512 patches: spectra far above 64 MiB
    f = torch.zeros((128,) * 3, dtype=torch.float64, device="cuda")
    out = torch.empty_like(f)
    with pytest.raises(mlc.MLCError) as e:
        plan.solve_noalloc(f, out)
    assert e.value.status == 1
