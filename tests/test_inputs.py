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


def _sympy_scaled(f, xyz, node, h, i):
    """h1^i1 h2^i2 h3^i3 / (i1! i2! i3!) d^i f at `node`, by symbolic
    differentiation (independent of both hand-written derivative formulas)."""
    sympy = pytest.importorskip("sympy")
    from math import factorial
    x, y, z = xyz
    d = sympy.diff(f, x, i[0], y, i[1], z, i[2]) if any(i) else f
    val = float(d.subs({x: node[0], y: node[1], z: node[2]}).evalf(30))
    return val * np.prod([h[k] ** i[k] / factorial(i[k]) for k in range(3)])


@pytest.mark.parametrize("m", [1, 3])
def test_gaussian_pulse_derivatives_are_the_symbolic_ones(m):
    """Eq. 2 scaling and the periodic image sum of the Gaussian pulse, against
    SymPy's derivatives of the same function at sampled nodes."""
    sympy = pytest.importorskip("sympy")
    n, h, centre, sigma = (6, 5, 4), (1 / 6, 1 / 5, 1 / 4), (0.3, 0.55, 0.7), 0.2
    x, y, z = sympy.symbols("x y z")

    def g(v, c):
        return sum(sympy.exp(-(v - c - p) ** 2 / (2 * sympy.Rational(1, 5) ** 2)) for p in (-1, 0, 1))
    f = g(x, sympy.Rational(3, 10)) * g(y, sympy.Rational(11, 20)) * g(z, sympy.Rational(7, 10))
    S = HI.gaussian_pulse(m, n, h, centre=centre, sigma=sigma)
    rng = np.random.default_rng(m)
    M = m + 1
    for _ in range(6):
        ix, iy, iz = (int(rng.integers(0, nn)) for nn in n)
        i = tuple(int(v) for v in rng.integers(0, M, 3))
        node = (ix * h[0], iy * h[1], iz * h[2])
        want = _sympy_scaled(f, (x, y, z), node, h, i)
        got = S[0, i[2], i[1], i[0], iz, iy, ix]
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (i, node, got, want)
    assert np.all(S[1] == 0.0)


def test_standing_mode_derivatives_are_the_symbolic_ones():
    """A plane standing mode sum_r A_r sin(2 pi k_r . x) (seeded draw) against
    SymPy's derivatives at sampled nodes, every derivative order of m = 2."""
    sympy = pytest.importorskip("sympy")
    m, n, h = 2, (5, 4, 3), (1 / 5, 1 / 4, 1 / 3)
    ks, amps = HI.standing_mode_draw(7, count=3, kmax=3)
    x, y, z = sympy.symbols("x y z")
    f = sum(float(a) * sympy.sin(2 * sympy.pi * (int(k[0]) * x + int(k[1]) * y + int(k[2]) * z))
            for k, a in zip(ks, amps))
    S = HI.standing_modes(m, n, h, seed=7, count=3, kmax=3)
    for node_idx in ((0, 0, 0), (3, 1, 2), (4, 3, 1)):
        node = tuple(node_idx[k] * h[k] for k in range(3))
        for i3 in range(m + 1):
            for i2 in range(m + 1):
                for i1 in range(m + 1):
                    want = _sympy_scaled(f, (x, y, z), node, h, (i1, i2, i3))
                    got = S[0, i3, i2, i1, node_idx[2], node_idx[1], node_idx[0]]
                    assert abs(got - want) <= 1e-12, ((i1, i2, i3), node, got, want)


@pytest.mark.parametrize("grid", [0, 1])
def test_advection_plane_wave_derivatives_are_the_symbolic_ones(grid):
    """The one-field plane wave sin(2 pi k . x + phase) of the advection tests,
    on the primal and the dual grid (nodes at (i + 1/2) h), against SymPy."""
    sympy = pytest.importorskip("sympy")
    m, n, h, k, phase = 3, (4, 3, 5), (1 / 4, 1 / 3, 1 / 5), (1, 2, 1), 0.4
    x, y, z = sympy.symbols("x y z")
    f = sympy.sin(2 * sympy.pi * (k[0] * x + k[1] * y + k[2] * z) + sympy.Rational(2, 5))
    A = HI.plane_wave(m, n, h, k, phase, grid)
    off = 0.5 if grid else 0.0
    for node_idx in ((0, 0, 0), (3, 2, 4), (1, 1, 2)):
        node = tuple((node_idx[d] + off) * h[d] for d in range(3))
        for i in ((0, 0, 0), (1, 0, 2), (3, 1, 0), (2, 3, 3)):
            want = _sympy_scaled(f, (x, y, z), node, h, i)
            got = A[i[2], i[1], i[0], node_idx[2], node_idx[1], node_idx[0]]
            assert abs(got - want) <= 1e-12, (i, node, got, want)
