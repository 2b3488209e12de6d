"""Fourier symbol and stability limit of the half step (TEST INFRASTRUCTURE ONLY).

Sec. 2 states the stability condition of Hermite methods (waves must not
travel from the cell boundary to the cell centre in a half step).  For the
wave equation with RK4 inside the half step the limit is found here from the
symbol of the half step.  For a Fourier mode with phase theta_k per node along
dimension k, a half step maps its amplitude vector by

    G(theta) = sum_{abc} W_abc exp(i theta . ((a, b, c) - 1/2)),

W_abc the corner blocks of the per-cell matrix (the output node sits half a
cell from each of its corners on both parities).  The scheme is stable when
the spectral radius of G is at most one for every theta.
"""
import numpy as np

from . import hermite


def symbol(m, h, c, dt, theta):
    """G(theta) (2M^3 x 2M^3, complex) for theta = (theta1, theta2, theta3)."""
    blocks = hermite.corner_blocks(hermite.cell_matrix(m, h, c, dt), m)
    G = 0
    for (a, b, cc), Wb in blocks.items():
        G = G + Wb * np.exp(1j * (theta[0] * (a - 0.5) + theta[1] * (b - 0.5) + theta[2] * (cc - 0.5)))
    return G


def max_spectral_radius(m, lam, npts=7, dims=3, evolve="rk4", q=4):
    """max over a theta grid of rho(G(theta)) for the isotropic unit-spaced
    problem with c tau / h = lam (h = 1, c = 1, dt = 2 lam).  ``dims`` = 1
    keeps theta2 = theta3 = 0 (a mode varying along x1 only)."""
    h = (1.0, 1.0, 1.0)
    dt = 2.0 * lam
    blocks = hermite.corner_blocks(hermite.cell_matrix(m, h, 1.0, dt, evolve, q), m)
    th = np.linspace(0.0, np.pi, npts)
    grid2 = th if dims == 3 else [0.0]
    rho = 0.0
    for t1 in th:
        for t2 in grid2:
            for t3 in grid2:
                G = 0
                for (a, b, cc), Wb in blocks.items():
                    G = G + Wb * np.exp(1j * (t1 * (a - 0.5) + t2 * (b - 0.5) + t3 * (cc - 0.5)))
                rho = max(rho, float(np.max(np.abs(np.linalg.eigvals(G)))))
    return rho


def stability_limit(m, lo=0.05, hi=0.6, tol=1e-3, npts=7, dims=3, evolve="rk4", q=4):
    """Largest lam = c tau / h (bisection to ``tol``) with max rho <= 1 + 1e-10."""
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if max_spectral_radius(m, mid, npts, dims, evolve, q) <= 1.0 + 1e-10:
            lo = mid
        else:
            hi = mid
    return lo
