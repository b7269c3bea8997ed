"""The checked debugging build (-DMLC_CHECKED): every kernel tests its
computed indices into the plan's arrays before use and records a bad one in
the plan's error word (mlc_plan_status -> MLC_ERR_INDEX) instead of touching
memory.  Solves covering every kernel family (local convolutions at 32-, 64-
and 128-point periods, the ring GEMM, residuals, coarse charge, coarse solve,
the coarser level of a multilevel plan, boundary values, Dirichlet solves of
four patch sizes, the q = 10 operator's second layer and two-layer Dirichlet
solves) run on the checked library in a child process: no check may
fire, and every result must carry the bits of the normal build (the checks
change no arithmetic)."""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from paper_1702_08111_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [
    dict(N=64, n=16, s=16, P=4, Q=6, tier=1),                 # split, ring GEMM, 64-point slab
    dict(N=48, n=16, s=16, P=4, Q=4, tier=0),                 # FP64
    dict(N=32, n=8, s=8, P=4, Q=4, tier=2),                   # double-float, 32-point period
    dict(N=64, n=32, s=20, P=4, Q=6, tier=1, g_beta=16),      # n = 32, 128-point register slab
    dict(N=64, n=32, s=20, P=4, Q=6, tier=0, mode=1),         # n = 32, FP64 row-streamed slab
    dict(N=48, n=24, s=8, P=4, Q=4, tier=0, mode=1),          # n = 24
    dict(N=32, n=8, s=12, P=4, Q=4, tier=0, levels=3),        # coarser level
    dict(N=16, n=4, s=8, P=2, Q=4, tier=3),                   # n = 4, split with double-float
    dict(N=32, n=8, s=16, P=4, Q=10, tier=0),                 # q = 10: second layer, ring, period 64
    dict(N=64, n=32, s=12, P=4, Q=10, tier=1, b=3, mode=1),   # q = 10, n = 32: workspace Dirichlet
]

CHILD = r"""
import json, os, sys
import numpy as np, torch
from paper_1702_08111_gb300 import inputs as I, mlc
cases, out = json.loads(sys.argv[1]), sys.argv[2]
for k, kw in enumerate(cases):
    kw = dict(kw)
    N = kw.pop("N"); n = kw.pop("n"); s = kw.pop("s"); P = kw.pop("P"); Q = kw.pop("Q")
    f64 = I.sample_bumps(N, I.draw_bumps(3, 1200 + k))
    f = torch.from_numpy(f64.astype(np.float32) if kw["tier"] in (1, 3) else f64).cuda()
    plan = mlc.Plan(N, n, s, P, Q, **kw)
    phi = plan.solve(f)
    torch.cuda.synchronize()
    plan.status()
    np.save(os.path.join(out, "%d.npy" % k), phi.cpu().numpy())
print("ok")
"""


def test_checked_build_runs_clean_and_bit_identical():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1702_08111_gb300 import build, mlc
    lib = build.build(checked=True)
    with tempfile.TemporaryDirectory() as tmp:
        env = dict(os.environ, MLC_GB300_LIBRARY=lib, PYTHONPATH=ROOT)
        r = subprocess.run([sys.executable, "-c", CHILD, json.dumps(CASES), tmp], env=env, cwd=ROOT,
                           capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stderr[-2000:]
        for k, kw in enumerate(CASES):
            kw = dict(kw)
            N, n, s, P, Q = (kw.pop(x) for x in ("N", "n", "s", "P", "Q"))
            f64 = I.sample_bumps(N, I.draw_bumps(3, 1200 + k))
            f = torch.from_numpy(f64.astype(np.float32) if kw["tier"] in (1, 3) else f64).cuda()
            ref = mlc.Plan(N, n, s, P, Q, **kw).solve(f).cpu().numpy()
            got = np.load(os.path.join(tmp, "%d.npy" % k))
            assert np.array_equal(got, ref), (k, float(np.abs(got - ref).max()))
