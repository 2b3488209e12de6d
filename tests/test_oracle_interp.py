"""Pins of the oracle's interpolation (Eq. 2, Eq. 3, Sec. 3.1, Alg. 1/2)."""
import os
from fractions import Fraction
from itertools import product
from math import comb

import numpy as np
import pytest

from oracle import exact, hermite

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fraction_matrix(path):
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([Fraction(tok) for tok in line.split()])
    return rows


def test_H_m1_matches_hand_derivation():
    H = hermite.hermite_matrix_exact(1)
    assert H == _read_fraction_matrix(os.path.join(GOLDEN, "H1_m1.txt"))


@pytest.mark.parametrize("m", [1, 2, 3])
def test_H_is_exact_inverse_of_conditions(m):
    A = hermite.hermite_conditions_exact(m)
    H = hermite.hermite_matrix_exact(m)
    P = 2 * m + 2
    for i in range(P):
        for j in range(P):
            assert sum(A[i][k] * H[k][j] for k in range(P)) == (1 if i == j else 0)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_H_reproduces_every_monomial_exactly(m):
    """For p = xi^d, d <= 2m+1, H applied to the node data gives the unit
    coefficient vector e_d (node data written out from the binomial rule)."""
    M, P = m + 1, 2 * m + 2
    H = hermite.hermite_matrix_exact(m)
    for d in range(P):
        data = []
        for xi0 in (Fraction(-1, 2), Fraction(1, 2)):
            for i in range(M):
                data.append(comb(d, i) * xi0 ** (d - i) if d >= i else Fraction(0))
        coeffs = [sum(H[j][k] * data[k] for k in range(P)) for j in range(P)]
        assert coeffs == [Fraction(int(j == d)) for j in range(P)]


@pytest.mark.parametrize("m", [1, 2, 3])
def test_H_norms(m):
    """max|H| and the 2-norm condition number quoted for the conditioning of
    the mixed-precision variants (2 / 6 / 21 and about 7.2 / 38.8 / 273)."""
    H = hermite.hermite_matrix(m)
    assert np.abs(H).max() == {1: 2.0, 2: 6.0, 3: 21.0}[m]
    assert np.linalg.cond(H) == pytest.approx({1: 7.17, 2: 38.8, 3: 273.3}[m], rel=2e-3)


@pytest.mark.parametrize("m", [1, 2])
def test_bruteforce_3d_interpolation_on_2cube(m):
    """Solve the full P^3 x P^3 Hermite conditions of one cell of a 2^3 grid
    directly (each row the scaled derivative of a monomial at a corner,
    evaluated by the generic polynomial rule), compare with Alg. 2."""
    M, P = m + 1, 2 * m + 2
    h = (0.5, 0.25, 0.4)
    rng = np.random.default_rng(7)
    U = rng.standard_normal((2, P, P, P))
    rows = []
    for cz, by, ax in product((0, 1), repeat=3):
        pt = ((ax - 0.5) * h[0], (by - 0.5) * h[1], (cz - 0.5) * h[2])
        for i3, i2, i1 in product(range(M), repeat=3):
            row = np.zeros((P, P, P))   # [jz, jy, jx]: monomial (x/h1)^jx (y/h2)^jy (z/h3)^jz
            for jz, jy, jx in product(range(P), repeat=3):
                C = np.zeros((P, P, P))
                C[jx, jy, jz] = 1.0 / (h[0] ** jx * h[1] ** jy * h[2] ** jz)
                row[jz, jy, jx] = exact.poly_scaled_derivative(C, (i1, i2, i3), pt, h)
            rows.append((cz * M + i3, by * M + i2, ax * M + i1, row.reshape(-1)))
    A = np.zeros((P ** 3, P ** 3))
    for r, (tz, ty, tx, row) in enumerate(rows):
        A[r] = row
    for f in range(2):
        rhs = np.array([U[f, tz, ty, tx] for tz, ty, tx, _ in rows])
        brute = np.linalg.solve(A, rhs).reshape(P, P, P)
        alg2 = hermite.reconstruct(U[f][None], hermite.hermite_matrix(m))[0]
        assert np.max(np.abs(brute - alg2)) <= 1e-12 * max(1.0, np.max(np.abs(brute)))


@pytest.mark.parametrize("m", [1, 2, 3])
def test_tensor_polynomials_reproduced_exactly(m):
    """A tensor polynomial of degree <= 2m+1 in each variable, sampled at the 8
    corners of a single (non-periodic) cell, is reconstructed exactly: the
    coefficients equal its scaled derivatives at the cell centre (Eq. 3)."""
    M, P = m + 1, 2 * m + 2
    rng = np.random.default_rng(11 + m)
    h = (0.3, 0.2, 0.25)
    xc = (0.1, -0.2, 0.05)
    C = rng.standard_normal((P, P, P))
    U = exact.poly_cell_data(m, C, np.zeros_like(C), h, xc)
    R = hermite.reconstruct(U[None], hermite.hermite_matrix(m))[0, 0]
    for jz, jy, jx in product(range(P), repeat=3):
        ref = exact.poly_scaled_derivative(C, (jx, jy, jz), xc, h)
        assert R[jz, jy, jx] == pytest.approx(ref, rel=1e-10, abs=1e-11)
