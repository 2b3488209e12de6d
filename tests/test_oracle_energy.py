"""Pins of the oracle's energy E = sum over cells of the integral of
B_v^2 + c^2 |grad B_u|^2 over the cell, B the tensor-product Hermite
interpolant of the node data (Eq. 3).

Nothing here reuses the oracle's arithmetic:
* the brute-force pin builds each cell's interpolant in physical coordinates
  from SciPy's Hermite (Bernstein-form) basis with unscaled derivatives,
  gathers the corners with its own periodic indexing, and integrates with
  Gauss-Legendre quadrature, exact for these polynomial degrees;
* the closed-form pin compares with the continuous energy of a product
  standing mode on the unit torus, which the interpolant approaches at the
  method's order (Sec. 3.1).
"""
from math import factorial, pi

import numpy as np
import pytest
from scipy.interpolate import BPoly

import hermite_inputs as HI
from oracle import hermite as oh


def _basis_1d(m, h, xq):
    """Values and first derivatives at the points xq (in [0, h]) of the 1-D
    Hermite basis on the cell [0, h] that takes SCALED data d_i = h^i/i!
    u^(i) at the two ends.  Columns are t = side * M + i."""
    M = m + 1
    val = np.zeros((len(xq), 2 * M))
    der = np.zeros((len(xq), 2 * M))
    for side in (0, 1):
        for i in range(M):
            data = [np.zeros(M), np.zeros(M)]
            data[side][i] = 1.0
            phi = BPoly.from_derivatives([0.0, h], [list(data[0]), list(data[1])])
            scale = factorial(i) / h ** i     # d_i -> u^(i)
            val[:, side * M + i] = scale * phi(xq)
            der[:, side * M + i] = scale * phi.derivative()(xq)
    return val, der


def _energy_brute(S, m, h, c, shift=0):
    """Sum over the cells of a periodic grid of the Gauss-Legendre integral
    of B_v^2 + c^2 |grad B_u|^2; cell (z, y, x) has its corners at the nodes
    (z + shift + {0,1}, y + shift + {0,1}, x + shift + {0,1}) mod n."""
    M = m + 1
    nz, ny, nx = S.shape[-3:]
    nq = 2 * M + 1
    gx, gw = np.polynomial.legendre.leggauss(nq)
    wts, V, D = [], [], []
    for d in range(3):
        xq = 0.5 * h[d] * (gx + 1.0)
        wts.append(0.5 * h[d] * gw)
        v, dv = _basis_1d(m, h[d], xq)
        V.append(v)
        D.append(dv)
    W = np.einsum("a,b,c->abc", wts[2], wts[1], wts[0])   # [qz, qy, qx]
    E = 0.0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                loc = np.empty((2, 2 * M, 2 * M, 2 * M))   # [f, tz, ty, tx]
                for cz in (0, 1):
                    for by in (0, 1):
                        for ax in (0, 1):
                            node = S[:, :, :, :, (z + shift + cz) % nz, (y + shift + by) % ny,
                                     (x + shift + ax) % nx]            # [f, i3, i2, i1]
                            loc[:, cz * M:(cz + 1) * M, by * M:(by + 1) * M, ax * M:(ax + 1) * M] = node

                def ev(A, bz, by_, bx):
                    return np.einsum("ZT,YU,XV,TUV->ZYX", bz, by_, bx, A)
                bv = ev(loc[1], V[2], V[1], V[0])
                ux = ev(loc[0], V[2], V[1], D[0])
                uy = ev(loc[0], V[2], D[1], V[0])
                uz = ev(loc[0], D[2], V[1], V[0])
                E += float(np.sum(W * (bv * bv + c * c * (ux * ux + uy * uy + uz * uz))))
    return E


@pytest.mark.parametrize("m", [1, 2, 3])
def test_energy_matches_quadrature_of_the_interpolant(m):
    """Random data on 2^3 and 3x2x2 grids with unequal spacings and c != 1:
    the oracle's moment-matrix energy equals the brute-force integral."""
    c = 1.7
    for n, h in (((2, 2, 2), (0.3, 0.5, 0.7)), ((3, 2, 2), (0.2, 0.45, 0.35))):
        S = HI.random_state(m, n, seed=40 + m)
        want = _energy_brute(S, m, h, c)
        got = oh.energy(S, m, h, c)
        assert abs(got - want) <= 1e-12 * abs(want), (n, got, want)


def test_energy_separates_its_terms():
    """Each term alone: v only gives the B_v^2 integral; u only with c = 0
    gives zero; u only scales with c^2.  A dropped or swapped term fails one."""
    m, n, h = 2, (2, 3, 2), (0.4, 0.3, 0.6)
    S = HI.random_state(m, n, seed=7)
    Sv = S.copy()
    Sv[0] = 0.0
    Su = S.copy()
    Su[1] = 0.0
    ev = oh.energy(Sv, m, h, 2.0)
    assert abs(ev - _energy_brute(Sv, m, h, 0.0)) <= 1e-12 * ev
    assert abs(oh.energy(Su, m, h, 0.0)) <= 1e-14 * ev
    e1, e3 = oh.energy(Su, m, h, 1.0), oh.energy(Su, m, h, 3.0)
    assert abs(e3 - 9.0 * e1) <= 1e-12 * e3
    assert abs(oh.energy(S, m, h, 3.0) - (ev + e3)) <= 1e-12 * (ev + e3)


def test_energy_is_the_same_on_either_cell_set():
    """On a periodic grid the cells with corners offset by 0 or -1 are the
    same cells relabelled, so both parities give one energy."""
    m, n, h = 1, (3, 2, 4), (0.25, 0.5, 0.2)
    S = HI.random_state(m, n, seed=3)
    e0, e1 = oh.energy(S, m, h, 1.3, 0), oh.energy(S, m, h, 1.3, 1)
    assert abs(e0 - e1) <= 1e-13 * e0
    assert abs(e0 - _energy_brute(S, m, h, 1.3, shift=-1)) <= 1e-12 * e0


@pytest.mark.parametrize("m", [1, 2, 3])
def test_energy_of_a_standing_mode_converges_to_the_closed_form(m):
    """u = B sin(2 pi k1 x) sin(2 pi k2 y) sin(2 pi k3 z), v = A times the same
    product, on the unit torus with unequal node counts per axis: the
    continuous energy is (A^2 + c^2 B^2 (2 pi)^2 |k|^2) / 8.  The interpolant's
    energy approaches it, and the error falls at least as h^(2m+1) (the order
    of the gradient's interpolation error; order 2m+2 is observed) when every
    spacing halves."""
    k, c, A, B = (1, 2, 1), 0.8, 0.6, 1.1
    exact = (A * A + c * c * B * B * (2 * pi) ** 2 * sum(kk * kk for kk in k)) / 8.0
    errs = []
    for base in ((6, 8, 5), (12, 16, 10)):
        n = base
        h = tuple(1.0 / nn for nn in n)
        S0 = HI.product_standing_mode(m, n, h, k)
        S = np.empty_like(S0)
        S[0] = B * S0[0]
        S[1] = A * S0[0]
        errs.append(abs(oh.energy(S, m, h, c) - exact) / exact)
    assert errs[1] <= errs[0] / 2 ** (2 * m + 1), errs
    assert errs[1] <= (3e-3, 1e-5, 3e-8)[m - 1], errs


@pytest.mark.parametrize("m,sides", [(1, (6, 12)), (2, (6, 8))])
def test_energy_drift_of_the_scheme_vanishes_under_refinement(m, sides):
    """The wave equation conserves the continuous energy, and the half steps
    converge (Sec. 2), so the drift |E(t) - E(0)| / E(0) of the oracle's
    scheme over a fixed stretch of time must shrink as h does; at least as
    h^(2m) is asserted (orders 2.6 and 5.0 are observed for m = 1 and 2, and
    the energy falls in almost every half step: the method dissipates).  Standing mode
    k = (1, 1, 1), lam = 0.2, 12 half steps at the coarse spacing and the
    same simulated time at the fine one."""
    c, lam, k = 1.0, 0.2, (1, 1, 1)
    t_end = 12 * lam * 2 / sides[0] / 2        # 12 half steps of the coarse grid
    drift = []
    for nn in sides:
        n, h = (nn,) * 3, (1.0 / nn,) * 3
        nhalf = int(round(t_end / (lam * h[0])))
        dt = 2 * t_end / nhalf                 # tau = dt / 2 = t_end / nhalf
        S = HI.product_standing_mode(m, n, h, k)
        e0 = oh.energy(S, m, h, c)
        S = oh.run(S, m, h, c, dt, nhalf)
        drift.append(abs(oh.energy(S, m, h, c) - e0) / e0)
    assert drift[1] <= drift[0] * (sides[0] / sides[1]) ** (2 * m), drift
    assert drift[1] <= (5e-2, 5e-4)[m - 1], drift
