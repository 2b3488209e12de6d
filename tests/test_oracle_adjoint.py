"""Pins of the oracle's discrete adjoint of the half step."""
import numpy as np
import pytest

from oracle import hermite


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("parity", [0, 1])
def test_dot_product_identity(m, parity):
    """<S x, y> = <x, S^T y> for random x, y (exact identity of a transpose)."""
    n = (3, 4, 5)
    h = (1 / 3, 1 / 4, 1 / 5)
    rng = np.random.default_rng(21)
    shape = (2, m + 1, m + 1, m + 1, n[2], n[1], n[0])
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    Sx = hermite.half_step(x, m, h, 1.2, 0.06, parity)
    STy = hermite.adjoint_half_step(y, m, h, 1.2, 0.06, parity)
    lhs, rhs = np.sum(Sx * y), np.sum(x * STy)
    assert abs(lhs - rhs) <= 1e-13 * (np.linalg.norm(Sx) * np.linalg.norm(y))


@pytest.mark.parametrize("m", [1, 2])
@pytest.mark.parametrize("parity", [0, 1])
def test_gather_adjoint_equals_scatter(m, parity):
    n = (3, 2, 4)
    h = (1 / 3, 1 / 2, 1 / 4)
    rng = np.random.default_rng(22)
    G = rng.standard_normal((2, m + 1, m + 1, m + 1, n[2], n[1], n[0]))
    a = hermite.adjoint_half_step(G, m, h, 1.0, 0.05, parity)
    b = hermite.adjoint_half_step_literal(G, m, h, 1.0, 0.05, parity)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
