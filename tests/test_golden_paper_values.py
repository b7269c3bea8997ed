"""Pins of the oracle against values the paper prints (fixtures under
tests/golden/, each citing its passage)."""
import os
from fractions import Fraction

from oracle import mlc_oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def test_stencil_weights_are_the_printed_ones():
    seen = set()
    for row in _rows("mehrstellen_stencils.txt"):
        if row[0] in ("4", "6"):
            Q = int(row[0])
            printed = [Fraction(v) for v in row[1:5]]
            for got, want in zip(O.STENCIL_B[Q], printed):
                assert abs(float(got) - float(want)) <= 1e-15
            seen.add(Q)
        elif row[0] == "C2":
            assert abs(O.C2 - float(Fraction(row[1]))) <= 1e-17
            seen.add("C2")
    assert seen == {4, 6, "C2"}


def test_quoted_barrier_ratio():
    # the printed 18.4 is (3.25 / 2)^6 to the digits shown
    for row in _rows("mehrstellen_stencils.txt"):
        if row[0] == "barrier_ratio_q6":
            assert round((3.25 / 2.0) ** 6, 1) == float(row[1])
            return
    raise AssertionError("fixture row missing")
