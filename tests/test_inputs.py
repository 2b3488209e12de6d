"""The shared seeded input generators agree with the oracle's closed forms
(two independent samplings of the same initial data, Eq. 2)."""
import numpy as np
import pytest

import hermite_inputs as HI
from oracle import exact


@pytest.mark.parametrize("m", [1, 2, 3])
def test_gaussian_pulse_matches_oracle(m):
    n, h = (12, 10, 8), (1 / 12, 1 / 10, 1 / 8)
    a = HI.gaussian_pulse(m, n, h, centre=(0.3, 0.55, 0.7), sigma=0.08)
    b = exact.gaussian_pulse(m, n, h, centre=(0.3, 0.55, 0.7), sigma=0.08)
    assert np.max(np.abs(a - b)) <= 1e-14


@pytest.mark.parametrize("m", [1, 3])
def test_standing_modes_match_oracle(m):
    n, h = (8, 8, 8), (1 / 8,) * 3
    a = HI.standing_modes(m, n, h, seed=1609)
    ks, amps = HI.standing_mode_draw(1609)
    b = exact.plane_modes(m, n, h, 1.0, 0.0, ks, amps)
    assert np.max(np.abs(a - b)) <= 1e-12
    c = HI.product_standing_mode(m, n, h)
    d = exact.product_mode(m, n, h, 1.0, 0.0)
    assert np.max(np.abs(c - d)) <= 1e-14


def test_draws_are_seeded():
    assert HI.batch_draw(3) == HI.batch_draw(3)
    r = HI.receiver_draw(5, (64, 64, 64))
    assert len(np.unique(r)) == 32 and np.array_equal(r, HI.receiver_draw(5, (64, 64, 64)))
