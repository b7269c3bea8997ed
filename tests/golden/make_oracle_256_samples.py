"""Write tests/golden/oracle_bumps32_256_q6_samples.txt: the CPU oracle's
two-level MLC potential for the 256^3 precision-form workload (4096 patches
of 16^3, support 16, Q = 6, P = 4; 32 bumps from seed 3, sampled in FP64 and
rounded to FP32 as the split tiers read them) at 4096 seeded sample nodes.

The full-size oracle solve takes many minutes on the host cores, so the GPU
parity test at this size compares against these stored samples.  This script
calls only the oracle and the seeded input generators.

    python tests/golden/make_oracle_256_samples.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import mlc_oracle as O  # noqa: E402
from paper_1702_08111_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "oracle_bumps32_256_q6_samples.txt")


def sample_nodes(N, count, seed):
    """Seeded sample: count distinct nodes of [0, N)^3, half of them on patch
    faces (where the boundary values enter) and half anywhere."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, N, size=(count // 2, 3))
    b = rng.integers(0, N, size=(count - count // 2, 3))
    b[np.arange(len(b)), rng.integers(0, 3, size=len(b))] = 16 * rng.integers(0, N // 16, size=len(b))
    g = np.unique(np.concatenate([a, b]), axis=0)
    return g


def main():
    w = I.workload("bumps32_256_q6")
    f = w.charge().astype(np.float64)  # FP32 samples, exactly representable
    prm = O.Params(N=w.N, n=w.n, s=w.s, Q=w.Q, P=w.P)
    G1 = O.dgf_octant(w.Q, 128, 2)
    t0 = time.time()
    phi = O.solve_open(prm, f, G1=G1)
    dt = time.time() - t0
    g = sample_nodes(w.N, 4096, 256)
    with open(OUT, "w") as fh:
        fh.write("# CPU oracle (oracle/mlc_oracle.py, two-level MLC of Sec. 4) at 256^3, n = s = 16, Q = 6, P = 4,\n")
        fh.write("# charge: 32 bumps from seed 3 sampled at the nodes and rounded to FP32 (inputs.workload\n")
        fh.write("# 'bumps32_256_q6'); DGF nD = 128, zeta = 2.  Written by make_oracle_256_samples.py\n")
        fh.write(f"# (oracle solve {dt:.0f} s).  Columns: g0 g1 g2 phi; max |phi| = {np.abs(phi).max():.17e}\n")
        for k in range(len(g)):
            fh.write(f"{g[k, 0]} {g[k, 1]} {g[k, 2]} {phi[g[k, 0], g[k, 1], g[k, 2]]:.17e}\n")
    print(f"wrote {len(g)} samples to {OUT} ({dt:.0f} s)")


if __name__ == "__main__":
    main()
