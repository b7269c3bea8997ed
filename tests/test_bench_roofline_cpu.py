"""The roofline arithmetic of bench.py, recounted by enumerating the slab
kernels' transform schedules (host logic only; no GPU)."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _radix2_fp32_count(nin=None):
    """FP32 instructions of a 64-point radix-2 line transform, counted butterfly
    by butterfly: 4 adds per butterfly with two live inputs, 4 instructions per
    twiddle other than 1 and -i.  nin: inputs nin..63 are zero (forward passes)."""
    live = np.ones(64, bool) if nin is None else np.arange(64) < nin
    inst = 0
    for st in range(5, -1, -1):  # decimation in frequency, half size 2^st
        hs = 1 << st
        new = live.copy()
        for g in range(0, 64, 2 * hs):
            for j in range(hs):
                i0, i1 = g + j, g + j + hs
                k = j << (5 - st)
                if live[i0] and live[i1]:
                    inst += 4
                if k not in (0, 16):
                    inst += 4
                new[i0] = new[i1] = live[i0] or live[i1]
        live = new
    return inst


def test_split_schedule_counts_match_enumeration():
    b = _bench()
    assert b.fft64_schedule_inst("split", False) == _radix2_fp32_count()
    assert b.fft64_schedule_inst("split", True, 17) == _radix2_fp32_count(17)


def test_radix8_schedule_counts():
    # radix 8 x 8: 16 butterflies of 52 adds + 4 multiplies, 56 twiddle
    # products (4 multiplies + 2 adds); double-float add = 8, multiply = 4
    b = _bench()
    adds, muls = 16 * 52 + 56 * 2, 16 * 4 + 56 * 4
    assert b.fft64_schedule_inst("df", False) == adds * 8 + muls * 4
    adds_s, muls_s = 8 * 26 + 8 * 52 + 56 * 2, 8 * 2 + 8 * 4 + 56 * 4
    assert b.fft64_schedule_inst("df", True) == adds_s * 8 + muls_s * 4
    # FP64: one instruction per add and multiply, a twiddle product is
    # 2 multiplies + 2 FMAs
    assert b.fft64_schedule_inst("fp64", False) == 16 * 52 + 16 * 4 + 56 * 4
    assert b.fft64_schedule_inst("fp64", True) == 8 * 26 + 8 * 52 + 8 * 2 + 8 * 4 + 56 * 4


def test_dirichlet_counts_closed_form():
    """Boundary terms of the Dirichlet right-hand side for n = 16: every
    neighbour of the 15^3 interior nodes lies in [0, 16]^3, so the terms are
    15^3 x (neighbours) minus the ordered interior-interior pairs, which number
    prod_d (15 - |s_d|) per stencil offset s."""
    b = _bench()
    inter = {1: 3 * 2 * 14 * 15 * 15, 2: 3 * 4 * 14 * 14 * 15, 3: 8 * 14 ** 3}
    t6 = 15 ** 3 * 26 - (inter[1] + inter[2] + inter[3])   # 27-point: all 26 offsets
    t4 = 15 ** 3 * 18 - (inter[1] + inter[2])              # 19-point: no corner offsets
    assert (t6, t4) == (11618, 6570)
    for Q, t in ((6, t6), (4, t4)):
        flops, inst = b.dirichlet_counts(16, Q)
        dst = 6 * 15 * 15 * 97
        assert flops == 2 * t + dst + 15 ** 3 + 2 * 16 ** 3
        assert inst == t + dst + 15 ** 3 + 16 ** 3
    # n = 32, 27-point: 31^3 x 26 neighbours minus the interior pairs
    inter32 = {1: 3 * 2 * 30 * 31 * 31, 2: 3 * 4 * 30 * 30 * 31, 3: 8 * 30 ** 3}
    t32 = 31 ** 3 * 26 - (inter32[1] + inter32[2] + inter32[3])
    assert t32 == 50786
    flops, inst = b.dirichlet_counts(32, 6)
    line_f, line_i = 30 + 97 + 8 * 34, 30 + 97 + 8 * 19  # sums/differences, DST-15, 8 odd pairs
    assert flops == 2 * t32 + 6 * 31 * 31 * line_f + 31 ** 3 + 2 * 32 ** 3
    assert inst == t32 + 6 * 31 * 31 * line_i + 31 ** 3 + 32 ** 3
    assert b.dirichlet_counts(24, 6) is None



def test_slab_rows_and_fp32_peak():
    b = _bench()

    class W:
        n, s = 16, 16
    # z rows of the field box read later: Omega_alpha rows plus coarse rows
    assert b.slab_rows(W, 8) == 37   # Q = 4, g_alpha = 8
    assert b.slab_rows(W, 4) == 31   # Q = 6, g_alpha = 4
    assert abs(b.FP32_LANE_INST_PER_S - 152 * 128 * 2.07e9) < 1.0
    assert abs(b.FP64_INST_PER_S - 0.625e12) < 1.0


def test_dirichlet_wide_counts_closed_form():
    """The q = 10 Dirichlet counts (bench.py dirichlet_wide_counts) against
    closed forms: a stencil offset s leaves the interior [1, n-1]^3 from
    m^3 - prod_d (m - |s_d|) nodes (m = n - 1), so that many boundary terms;
    an offset with one component of size 2 reaches the outer layer from the
    nodes next to the face, and its mirror image is interior from
    prod_{e != d} (m - |s_e|) of them (the fixed-point corrections)."""
    import itertools
    b = _bench()
    orbits = {(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1), (2, 0, 0), (2, 1, 0)}
    offs = [s for s in itertools.product(range(-2, 3), repeat=3)
            if tuple(sorted(map(abs, s), reverse=True)) in orbits]
    assert len(offs) == 57
    for n in (8, 16, 32):
        m = n - 1
        tb = sum(m ** 3 - np.prod([m - abs(c) for c in s]) for s in offs)
        tc = 0
        for s in offs:
            two = [d for d in range(3) if abs(s[d]) == 2]
            if len(two) == 1:
                tc += np.prod([m - abs(s[e]) for e in range(3) if e != two[0]])
        it = b.WIDE_DIRICHLET_ITERS
        if n == 16:
            lf = li = 97
        elif n == 32:
            li, lf = 30 + 97 + 8 * 19, 30 + 97 + 8 * 34
        else:
            lf, li = 2 * m * m, m * m
        flops = 2 * tb + (1 + it) * (6 * m * m * lf + m ** 3) + it * 2 * tc + 2 * n ** 3
        inst = 2 * tb + (1 + it) * (6 * m * m * li + m ** 3) + it * 2 * tc + n ** 3
        assert b.dirichlet_wide_counts(n) == (flops, inst), n
