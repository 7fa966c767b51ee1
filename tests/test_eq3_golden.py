"""Eq. 3 pinned: synth.delta_z_for(vfov, hlines) feeds both the oracle and the
CUDA path, so a slip in it would pass every parity test. It is checked here
against the closed form tan(vfov / hlines degrees), written out in
tests/golden/eq3_delta_z.txt and recomputed with exact rational arithmetic
(pi from Machin's formula, sine and cosine from their Taylor series)."""
import os
from fractions import Fraction

import numpy as np

from paper_2310_05766_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eq3_delta_z.txt")


def _arctan_inv(n: int, terms: int) -> Fraction:
    """arctan(1/n) by its alternating series."""
    s, x2 = Fraction(0), Fraction(1, n * n)
    p = Fraction(1, n)
    for k in range(terms):
        s += (-1) ** k * p / (2 * k + 1)
        p *= x2
    return s


def _tan_deg(angle: Fraction) -> Fraction:
    pi = 16 * _arctan_inv(5, 40) - 4 * _arctan_inv(239, 15)   # Machin; error far below 1e-40
    x = angle * pi / 180
    sin, cos, term = Fraction(0), Fraction(0), Fraction(1)
    for k in range(30):   # term = x^k / k!
        if k % 4 == 0:
            cos += term
        elif k % 4 == 1:
            sin += term
        elif k % 4 == 2:
            cos -= term
        else:
            sin -= term
        term = term * x / (k + 1)
    return sin / cos


def _rows():
    out = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            v, h, t = line.split()
            out.append((int(v), int(h), t))
    return out


def test_golden_rows_are_the_closed_form():
    rows = _rows()
    assert len(rows) == 5
    for v, h, t in rows:
        exact = _tan_deg(Fraction(v, h))
        assert abs(exact - Fraction(t)) < Fraction(1, 10 ** 25), (v, h)   # rows are truncated after 26 decimals


def test_delta_z_for_rounds_the_closed_form_to_float32():
    for v, h, t in _rows():
        assert synth.delta_z_for(float(v), h) == float(np.float32(float(Fraction(t)))), (v, h)
    # the two workload values, as float32 literals
    assert synth.delta_z_for(30.0, 16) == float(np.float32(0.03273661))
    assert synth.delta_z_for(45.0, 128) == float(np.float32(0.006136))
