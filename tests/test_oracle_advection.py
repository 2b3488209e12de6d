"""Pins of the advection oracle (Eq. 1 with a constant velocity a, Sec. 2,
Alg. 4, Eq. 5) to facts that do not come from the oracle itself."""
from math import factorial, pi

import numpy as np
import numpy.polynomial.polynomial as npp
import pytest

import hermite_inputs as HI
from oracle import advection as adv


def _poly_corner_tensor(C, m, h):
    """Local tensor (1, P, P, P) [tz, ty, tx] of the tensor polynomial with
    coefficients C[j1, j2, j3] in (y1, y2, y3) = x - x_centre: at each corner,
    h^i / i! D^i p, via numpy's polynomial derivatives (no Hermite operator)."""
    M, P = m + 1, 2 * m + 2
    U = np.zeros((1, P, P, P))
    for sz in (0, 1):
        for sy in (0, 1):
            for sx in (0, 1):
                y = ((sx - 0.5) * h[0], (sy - 0.5) * h[1], (sz - 0.5) * h[2])
                for i3 in range(M):
                    for i2 in range(M):
                        for i1 in range(M):
                            D = npp.polyder(npp.polyder(npp.polyder(C, i1, axis=0), i2, axis=1), i3, axis=2)
                            w = h[0] ** i1 * h[1] ** i2 * h[2] ** i3 / (factorial(i1) * factorial(i2) * factorial(i3))
                            U[0, sz * M + i3, sy * M + i2, sx * M + i1] = w * npp.polyval3d(*y, D)
    return U


def _scaled_derivs_at(C, m, h, y):
    M = m + 1
    out = np.zeros((M, M, M))
    for i3 in range(M):
        for i2 in range(M):
            for i1 in range(M):
                D = npp.polyder(npp.polyder(npp.polyder(C, i1, axis=0), i2, axis=1), i3, axis=2)
                w = h[0] ** i1 * h[1] ** i2 * h[2] ** i3 / (factorial(i1) * factorial(i2) * factorial(i3))
                out[i3, i2, i1] = w * npp.polyval3d(*y, D)
    return out


def _directional(C, a):
    """(a . grad) p on coefficient arrays, with numpy's polyder."""
    P = C.shape[0]
    out = np.zeros_like(C)
    for k in range(3):
        d = npp.polyder(C, 1, axis=k)
        pad = [(0, 0)] * 3
        pad[k] = (0, 1)
        out += a[k] * np.pad(d, pad)
    return out


CASES = [(1, 1), (1, 4), (1, 9), (2, 3), (2, 15), (3, 6), (3, 21), (3, 25)]


@pytest.mark.parametrize("m,q", CASES)
def test_polynomial_data_gives_truncated_exponential(m, q):
    """For data of a degree-(2m+1) tensor polynomial the interpolant is the
    polynomial, so the half step returns the scaled derivatives at the centre
    of sum_{s <= q} tau^s / s! (a . grad)^s p; for q >= 3(2m+1) that is the
    translated polynomial p(y + a tau), the exact solution of Eq. 1."""
    rng = np.random.default_rng(40 + 7 * m + q)
    P = 2 * m + 2
    C = rng.standard_normal((P, P, P))
    h = (0.11, 0.07, 0.09)
    a = (1.0, -0.6, 0.8)
    tau = 0.3 * min(h)
    U = _poly_corner_tensor(C, m, h)
    got = adv.cell_map(U, m, h, a, tau, q)[0]
    acc, term = np.zeros_like(C), C.copy()
    for s in range(q + 1):
        acc += term * tau ** s / factorial(s)
        term = _directional(term, a)
    want = _scaled_derivs_at(acc, m, h, (0.0, 0.0, 0.0))
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 1e-11 * scale
    if q >= adv.full_q(m):
        shifted = _scaled_derivs_at(C, m, h, tuple(a[k] * tau for k in range(3)))
        assert np.max(np.abs(got - shifted)) <= 1e-11 * scale


@pytest.mark.parametrize("q", [1, 2, 5, 9, 15])
def test_horner_form_equals_coefficient_recursion(q):
    """Alg. 4 (Horner loop over the stages) and Eq. 5 (recursion of the
    space-time coefficients, evaluated at t_{n+1/2}) are the same series."""
    rng = np.random.default_rng(q)
    B = rng.standard_normal((4, 6, 6, 6))
    h, a, dt = (0.1, 0.13, 0.07), (1.0, -0.5, 0.7), 0.04
    x = adv.evolve_taylor(B, 0.5 * dt, a, h, q)
    y = adv.evolve_recursion(B, dt, a, h, q)
    assert np.max(np.abs(x - y)) <= 1e-14 * np.max(np.abs(x))


@pytest.mark.parametrize("m", [1, 2, 3])
def test_constant_state_is_invariant(m):
    M = m + 1
    n = (5, 4, 3)
    A = np.zeros((M, M, M, n[2], n[1], n[0]))
    A[0, 0, 0] = 2.5
    for parity in (0, 1):
        out = adv.half_step(A, m, (0.2, 0.25, 1 / 3), (1.0, 1.0, 1.0), 0.1, parity)
        assert np.max(np.abs(out - A)) <= 1e-14


@pytest.mark.parametrize("m", [1, 2, 3])
def test_one_dimensional_stability_limit_is_half_a_cell(m):
    """Sec. 2: with the full series the method is stable while a wave moves at
    most from the cell boundary to its centre in a half step (|a| tau <= h/2),
    whatever the order.  The symbol of a mode along x1 with a = (a1, 0, 0) has
    spectral radius 1 at lam = a1 tau / h = 0.5 and above 1 just past it."""
    assert adv.max_spectral_radius(m, 0.5, npts=9, dims=1) <= 1.0 + 1e-12
    assert adv.max_spectral_radius(m, 0.45, npts=9, dims=1) <= 1.0 + 1e-12
    assert adv.max_spectral_radius(m, 0.52, npts=9, dims=1) > 1.01


@pytest.mark.parametrize("m,n0", [(1, 8), (2, 6), (3, 4)])
def test_plane_wave_converges_at_order_2m_plus_1(m, n0):
    """Sec. 2: the global error for smooth solutions is O(h^(2m+1)).  A plane
    wave sin(2 pi (x1 + x2 + x3)) advected with a = (1, 1, 1) to t = 0.25 at a
    fixed lam = 0.25 on n0^3 and (2 n0)^3 grids."""
    errs = []
    for n in (n0, 2 * n0):
        h = (1.0 / n,) * 3
        dt = 0.5 * h[0]                       # lam = a tau / h = 0.25
        nfull = int(round(0.25 / dt))
        A0 = HI.plane_wave(m, (n,) * 3, h)
        A = adv.run(A0, m, h, (1.0, 1.0, 1.0), dt, 2 * nfull)
        exact = HI.plane_wave(m, (n,) * 3, h, phase=2 * pi * 3 * 0.25)
        errs.append(np.max(np.abs(A[0, 0, 0] - exact[0, 0, 0])))
    order = np.log2(errs[0] / errs[1])
    assert order >= 2 * m + 1 - 0.5, (errs, order)
