"""Pins of the oracle's evolution and truncation (Eq. 4, Alg. 3/4, Sec. 2).

Exact polynomial solutions of u_t = v, v_t = c^2 Delta u are built here in
physical coordinates (an independent representation from the oracle's scaled
coefficient tensors): for polynomials p, q with Delta^3 p = 0 and
Delta^2 q = 0 the solution

    u(t) = p + t q + t^2/2 c^2 Dp + t^3/6 c^2 Dq + t^4/24 c^4 D^2 p,  v = u_t,

has degree <= 4 in t, so one RK4 (= Taylor q = 4) half step reproduces it
exactly once its degree per variable is at most 2m+1.
"""
from itertools import product
from math import factorial

import numpy as np
import pytest

from oracle import exact, hermite, symbol


def _lap(C):
    """Laplacian of sum C[a,b,c] x^a y^b z^c (physical coordinates)."""
    out = np.zeros_like(C)
    n = C.shape[0]
    for a, b, c in product(range(n), repeat=3):
        v = C[a, b, c]
        if v == 0:
            continue
        if a >= 2:
            out[a - 2, b, c] += a * (a - 1) * v
        if b >= 2:
            out[a, b - 2, c] += b * (b - 1) * v
        if c >= 2:
            out[a, b, c - 2] += c * (c - 1) * v
    return out


def _random_poly(rng, P, max_total, max_each):
    C = np.zeros((P, P, P))
    for a, b, c in product(range(P), repeat=3):
        if a + b + c <= max_total and max(a, b, c) <= max_each:
            C[a, b, c] = rng.standard_normal()
    return C


def _solution(p, q, c, t):
    Lp, Lq = _lap(p), _lap(q)
    LLp = _lap(Lp)
    assert np.all(_lap(LLp) == 0) and np.all(_lap(Lq) == 0)
    u = p + t * q + t ** 2 / 2 * c ** 2 * Lp + t ** 3 / 6 * c ** 2 * Lq + t ** 4 / 24 * c ** 4 * LLp
    v = q + t * c ** 2 * Lp + t ** 2 / 2 * c ** 2 * Lq + t ** 3 / 6 * c ** 4 * LLp
    return u, v


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("evolve", ["rk4", "taylor"])
def test_polynomial_wave_solution_advanced_exactly(m, evolve):
    M, P = m + 1, 2 * m + 2
    rng = np.random.default_rng(100 + m)
    h = (0.11, 0.07, 0.09)
    c = 1.7
    tau = 0.25 * min(h) / c        # c tau / h_k <= 0.25, inside the stable range
    xc = (0.2, -0.1, 0.3)
    p = _random_poly(rng, P, max_total=5, max_each=2 * m + 1)
    q = _random_poly(rng, P, max_total=3, max_each=2 * m + 1)
    U = exact.poly_cell_data(m, p, q, h, xc)
    out = hermite.cell_map(U[None], m, h, c, tau, evolve)[0]
    u1, v1 = _solution(p, q, c, tau)
    for f, C in enumerate((u1, v1)):
        ref = np.array([[[exact.poly_scaled_derivative(C, (i1, i2, i3), xc, h) for i1 in range(M)]
                         for i2 in range(M)] for i3 in range(M)])
        # rounding only: H has 2-norm condition 7 / 39 / 273 per dimension
        scale = max(1.0, np.max(np.abs(ref)), np.max(np.abs(U)))
        assert np.max(np.abs(out[f] - ref)) <= {1: 1e-12, 2: 1e-11, 3: 1e-10}[m] * scale


@pytest.mark.parametrize("m", [1, 2, 3])
def test_rk4_equals_taylor_q4(m):
    P = 2 * m + 2
    rng = np.random.default_rng(5)
    Bu, Bv = rng.standard_normal((2, 3, P, P, P))
    h, c, tau = (0.1, 0.13, 0.08), 1.1, 0.02
    a = hermite.evolve_rk4(Bu, Bv, tau, c, h)
    b = hermite.evolve_taylor(Bu, Bv, tau, c, h, q=4)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) <= 1e-13 * np.max(np.abs(x))


def test_second_derivative_matches_monomial_rule():
    """d^2/dxi^2 xi^j = j (j-1) xi^(j-2) written on coefficient vectors."""
    P = 6
    for j in range(P):
        e = np.zeros(P)
        e[j] = 1.0
        d = hermite.second_derivative(e, 0)
        ref = np.zeros(P)
        if j >= 2:
            ref[j - 2] = j * (j - 1)
        assert np.array_equal(d, ref)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_zero_and_constant_states(m):
    n = (3, 4, 2)
    h = (1 / 3, 1 / 4, 1 / 2)
    S = np.zeros((2, m + 1, m + 1, m + 1) + n[::-1])
    for p in (0, 1):
        assert np.all(hermite.half_step(S, m, h, 1.0, 0.05, p) == 0)
    S[0, 0, 0, 0] = 2.5           # u = const, v = 0 is a steady solution
    for p in (0, 1):
        out = hermite.half_step(S, m, h, 1.0, 0.05, p)
        assert np.max(np.abs(out - S)) <= 1e-13


@pytest.mark.parametrize("m", [1, 2])
def test_full_taylor_equals_matrix_exponential(m):
    """With q = d(2m+1) stages (Alg. 4's largest step, Sec. 3.2) the local
    evolution is exact: L = [[0, I], [c^2 Delta, 0]] is nilpotent on the
    polynomials of degree <= 2m+1 per variable (Delta lowers the total degree
    by 2), so the q-term Taylor series equals exp(tau L), computed here by
    scipy's Pade-based expm of the explicit matrix of L."""
    from scipy.linalg import expm
    P = 2 * m + 2
    h, c, tau = (0.1, 0.13, 0.09), 1.1, 0.02
    n = 2 * P ** 3
    E = np.eye(n).reshape(n, 2, P, P, P)
    Lu, Lv = hermite.wave_operator(E[:, 0], E[:, 1], c, h)
    L = np.concatenate([Lu.reshape(n, -1), Lv.reshape(n, -1)], axis=1).T      # column k = L e_k
    rng = np.random.default_rng(7)
    B = rng.standard_normal((2, P, P, P))
    q = 3 * (2 * m + 1)
    wu, wv = hermite.evolve_taylor(B[0][None], B[1][None], tau, c, h, q=q)
    ref = expm(tau * L) @ B.reshape(-1)
    got = np.concatenate([wu.reshape(-1), wv.reshape(-1)])
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
    # and fewer stages are not exact
    wu4, wv4 = hermite.evolve_taylor(B[0][None], B[1][None], tau, c, h, q=4)
    assert np.max(np.abs(np.concatenate([wu4.reshape(-1), wv4.reshape(-1)]) - ref)) > 1e-8 * np.max(np.abs(ref))


@pytest.mark.parametrize("m", [1, 2, 3])
def test_polynomial_solution_full_taylor(m):
    """Any polynomial solution of degree <= 2m+1 per variable is advanced
    exactly by the full-order Taylor evolution (here p of total degree 2m+1
    per the tensor space, with its exact time dependence from the series of
    Delta^k p)."""
    M, P = m + 1, 2 * m + 2
    rng = np.random.default_rng(300 + m)
    h = (0.11, 0.07, 0.09)
    c = 1.3
    tau = 0.2 * min(h) / c
    xc = (0.05, -0.1, 0.2)
    p = _random_poly(rng, P, max_total=3 * (2 * m + 1), max_each=2 * m + 1)
    q0 = np.zeros_like(p)
    # u(t) = sum_k t^(2k)/(2k)! c^(2k) Delta^k p,  v = u_t
    u1, v1, D, k = np.zeros_like(p), np.zeros_like(p), p.copy(), 0
    while np.any(D != 0):
        u1 += tau ** (2 * k) / factorial(2 * k) * c ** (2 * k) * D
        D = _lap(D)
        k += 1
        if np.any(D != 0):
            v1 += tau ** (2 * k - 1) / factorial(2 * k - 1) * c ** (2 * k) * D
    U = exact.poly_cell_data(m, p, q0, h, xc)
    out = hermite.cell_map(U[None], m, h, c, tau, "taylor", q=3 * (2 * m + 1))[0]
    for f, C in enumerate((u1, v1)):
        ref = np.array([[[exact.poly_scaled_derivative(C, (i1, i2, i3), xc, h) for i1 in range(M)]
                         for i2 in range(M)] for i3 in range(M)])
        scale = max(1.0, np.max(np.abs(ref)), np.max(np.abs(U)))
        assert np.max(np.abs(out[f] - ref)) <= {1: 1e-12, 2: 1e-11, 3: 1e-9}[m] * scale


def test_full_taylor_is_stable_beyond_rk4_limit():
    """Sec. 2: with the full series the step is limited only by the geometric
    condition, so at m = 2 a half step with lam = 0.38 is stable for
    q = 3(2m+1) and unstable for q = 4 (RK4)."""
    assert symbol.max_spectral_radius(2, 0.38, npts=5, evolve="taylor", q=15) <= 1.0 + 1e-10
    assert symbol.max_spectral_radius(2, 0.38, npts=5) > 1.0 + 1e-6
