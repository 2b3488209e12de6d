"""The library's stability tool (Fourier symbol of the half step, largest
stable step) against the oracle's symbol (no GPU needed)."""
import ctypes
import itertools

import numpy as np
import pytest

from oracle import advection as adv
from oracle import hermite as oh
from oracle import symbol as osym


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1609_09841_gb300 as pkg
    return pkg


def _oracle_wave_radius(m, h, c, dt, theta, q):
    evolve = "rk4" if q == 4 else "taylor"
    blocks = oh.corner_blocks(oh.cell_matrix(m, h, c, dt, evolve, q), m)
    G = sum(W * np.exp(1j * (theta[0] * (a - 0.5) + theta[1] * (b - 0.5) + theta[2] * (cc - 0.5)))
            for (a, b, cc), W in blocks.items())
    return float(np.max(np.abs(np.linalg.eigvals(G))))


def _oracle_adv_radius(m, h, a, dt, theta, q):
    M = m + 1
    W = adv.cell_matrix(m, h, a, dt, q).reshape(M ** 3, 2, M, 2, M, 2, M)
    G = 0
    for cz, cy, cx in itertools.product((0, 1), repeat=3):
        G = G + W[:, cz, :, cy, :, cx, :].reshape(M ** 3, M ** 3) * np.exp(
            1j * (theta[0] * (cx - 0.5) + theta[1] * (cy - 0.5) + theta[2] * (cz - 0.5)))
    return float(np.max(np.abs(np.linalg.eigvals(G))))


@pytest.mark.parametrize("m,q", [(1, 4), (1, 9), (2, 4), (2, 7), (2, 15), (3, 4), (3, 21)])
def test_wave_symbol_radius_matches_oracle(lib, m, q):
    """The symbol assembled from the kernels' tables has the oracle's
    spectral radius (anisotropic spacings, several modes)."""
    h, c = (0.11, 0.07, 0.09), 1.3
    dt = 2 * 0.3 * min(h) / c
    rng = np.random.default_rng(m * 31 + q)
    for theta in [(0.0, 0.0, 0.0), (np.pi, np.pi, np.pi)] + [tuple(rng.uniform(0, np.pi, 3)) for _ in range(3)]:
        got = lib.symbol_radius(m, h, c, dt, theta, q=q)
        want = _oracle_wave_radius(m, h, c, dt, theta, q)
        assert abs(got - want) <= 1e-8 * max(1.0, want), (theta, got, want)


@pytest.mark.parametrize("m,q", [(1, 3), (1, 0), (2, 5), (2, 0), (3, 4), (3, 0)])
def test_advection_symbol_radius_matches_oracle(lib, m, q):
    h, a = (0.1, 0.12, 0.08), (1.0, -0.6, 0.4)
    qq = q or adv.full_q(m)
    dt = 0.4 * min(hk / abs(ak) for hk, ak in zip(h, a))
    rng = np.random.default_rng(7 * m + q)
    for theta in [(np.pi, 0.0, np.pi / 2)] + [tuple(rng.uniform(0, np.pi, 3)) for _ in range(3)]:
        got = lib.adv_symbol_radius(m, h, a, dt, theta, q=q)
        want = _oracle_adv_radius(m, h, a, dt, theta, qq)
        assert abs(got - want) <= 1e-9 * max(1.0, want), (theta, got, want)


def test_max_dt_isotropic_matches_oracle_limits(lib):
    """For h1 = h2 = h3 the bound is the oracle's isotropic RK4 limit (0.4518
    and 0.3010 for m = 1, 2) and at least the plan's rounded table entry."""
    h = (1 / 16,) * 3
    for m, want in ((1, 0.4518), (2, 0.3010)):
        lam = lib.max_dt(m, h, 1.0) / 2 / h[0]
        assert abs(lam - want) <= 2e-3, (m, lam)
        assert lam >= lib.stability_limit(m)


def test_max_dt_anisotropic_checked_by_the_oracle(lib):
    """An anisotropic grid (aspect ratios 1 : 1.6 : 0.7): the oracle's symbol
    is stable at the returned step and unstable 2 % above it."""
    m, c = 1, 1.0
    h = (0.1, 0.16, 0.07)
    dt = lib.max_dt(m, h, c)
    th = np.linspace(0, np.pi, 7)

    def rho(d):
        return max(_oracle_wave_radius(m, h, c, d, t, 4) for t in itertools.product(th, th, th))
    assert rho(dt) <= 1 + 1e-10
    assert rho(1.02 * dt) > 1 + 1e-10
    # the finest spacing sets the step: larger than the isotropic bound on h = 0.07
    assert dt > 2 * lib.stability_limit(m) * 0.07 / c


def test_full_series_has_an_instability_window_at_m3(lib):
    """m = 3, q = 21: the oracle's symbol is stable at lam = 0.36 and 0.40
    but weakly unstable at 0.38, so the set of stable steps is not an
    interval; the library's radius agrees there, and the plan's bound stays
    below the window."""
    assert osym.max_spectral_radius(3, 0.38, npts=7, evolve="taylor", q=21) > 1 + 1e-9
    assert osym.max_spectral_radius(3, 0.40, npts=7, evolve="taylor", q=21) <= 1 + 1e-10
    h = (1.0, 1.0, 1.0)
    assert lib.max_radius(3, h, 1.0, 2 * 0.38, q=21) > 1 + 1e-9
    assert lib.max_radius(3, h, 1.0, 2 * 0.36, q=21) <= 1 + 1e-10
    assert lib.stability_limit(3, 21) < 0.375


def test_advection_bound_is_half_a_cell(lib):
    """Sec. 2, whole series: |a_k| tau / h_k <= 1/2 in every dimension."""
    h, a = (0.1, 0.2, 0.05), (1.0, 0.3, -0.2)
    dt = lib.adv_max_dt(2, h, a)
    lam = max(abs(ak) * dt / 2 / hk for ak, hk in zip(a, h))
    assert abs(lam - 0.5) <= 1e-3


def test_tool_argument_checks(lib):
    c = lib.capi
    d3 = (ctypes.c_double * 3)
    out = ctypes.c_double()
    assert c.lib.hermite_symbol_radius(0, 4, 1.0, d3(1, 1, 1), 0.1, d3(0, 0, 0), ctypes.byref(out)) == -1
    assert c.lib.hermite_symbol_radius(2, 3, 1.0, d3(1, 1, 1), 0.1, d3(0, 0, 0), ctypes.byref(out)) == -1
    assert c.lib.hermite_symbol_radius(2, 4, -1.0, d3(1, 1, 1), 0.1, d3(0, 0, 0), ctypes.byref(out)) == -1
    assert c.lib.hermite_max_dt(2, 4, 1.0, d3(1, 0, 1), 7, ctypes.byref(out)) == -1
    assert c.lib.hermite_max_dt(2, 4, 1.0, d3(1, 1, 1), 1, ctypes.byref(out)) == -1
    assert c.lib.hermite_adv_max_dt(2, 0, d3(0, 0, 0), d3(1, 1, 1), 7, ctypes.byref(out)) == -1
    assert c.lib.hermite_adv_symbol_radius(2, 16, d3(1, 0, 0), d3(1, 1, 1), 0.1, d3(0, 0, 0),
                                           ctypes.byref(out)) == -1
    assert c.lib.hermite_max_radius(2, 4, 1.0, d3(1, 1, 1), 0.5, 0, ctypes.byref(out)) == -1
