"""Pin of the oracle's error norms on a hand-worked example.  The norms are
the reference of the library's FP64 reduction (hermite_error), so they are
checked here against values computed by hand, not against a second coding
of the same formulas."""
from math import sqrt

import numpy as np
import pytest

from oracle import hermite


def _example():
    """m = 1 on a 1 x 1 x 2 grid: 2 fields x 2^3 orders x 2 nodes = 32 values.
    ref is all ones except the u value at node z = 1, which is 5.  The state
    differs from ref by +3 in the u value at node z = 0 and by -4 in the v
    derivative of orders (i1, i2, i3) = (1, 0, 1) at node z = 1."""
    shape = (2, 2, 2, 2, 2, 1, 1)            # [f][i3][i2][i1][z][y][x]
    ref = np.ones(shape)
    ref[0, 0, 0, 0, 1, 0, 0] = 5.0
    d = np.zeros(shape)
    d[0, 0, 0, 0, 0, 0, 0] = 3.0
    d[1, 1, 0, 1, 1, 0, 0] = -4.0
    return ref + d, ref


# (mask, max_abs, max_rel, l2_abs, l2_rel), worked by hand from _example:
#   0b111: all 32 values; differences 3 and -4; max|ref| = 5; sum ref^2 = 31 + 25.
#   0b011: the values of u and v (4 entries); the -4 is a derivative, not selected.
#   0b110: every order of v (16 entries); max|ref| = 1.
#   0b001: the values of u (2 entries: ref 1 and 5).
CASES = [
    (0b111, 4.0, 4.0 / 5.0, 5.0, 5.0 / sqrt(56.0)),
    (0b011, 3.0, 3.0 / 5.0, 3.0, 3.0 / sqrt(28.0)),
    (0b110, 4.0, 4.0, 4.0, 4.0 / sqrt(16.0)),
    (0b001, 3.0, 3.0 / 5.0, 3.0, 3.0 / sqrt(26.0)),
]


@pytest.mark.parametrize("mask,max_abs,max_rel,l2_abs,l2_rel", CASES)
def test_error_norms_on_a_hand_worked_example(mask, max_abs, max_rel, l2_abs, l2_rel):
    a, b = _example()
    got = hermite.error_norms(a, b, mask)
    assert got == pytest.approx((max_abs, max_rel, l2_abs, l2_rel), rel=1e-15, abs=0)


def test_error_norms_of_equal_states_are_zero():
    a, b = _example()
    assert hermite.error_norms(b, b, 0b111) == (0.0, 0.0, 0.0, 0.0)
    assert hermite.error_norms(a, a, 0b010)[0] == 0.0
