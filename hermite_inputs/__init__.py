"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

This module holds input generation only -- random states, initial data of the
workloads sampled as node data, the seeded draws of the batched and receiver
workloads -- and none of the half step's arithmetic (no interpolation,
evolution or truncation).  Arrays use the state layout
``S[f, i3, i2, i1, z, y, x]`` (field u/v, derivative orders along x3, x2, x1,
then the node with x fastest); entry i of a field at a node is
h1^i1 h2^i2 h3^i3 / (i1! i2! i3!) times the derivative d^i of the field
(Eq. 2 with the per-dimension spacings of Eq. 3).
"""
from math import factorial, pi

import numpy as np

__all__ = ["random_state", "gaussian_pulse", "standing_modes", "standing_mode_draw",
           "product_standing_mode", "batch_draw", "receiver_draw", "state_shape",
           "advection_random_state", "plane_wave"]


def state_shape(m, n):
    """Shape of a state for order m on an (n1, n2, n3) grid."""
    M = m + 1
    return (2, M, M, M, n[2], n[1], n[0])


def random_state(m, n, seed, decay=0.5):
    """Seeded N(0, 1) state, component i scaled by decay^|i| so that higher
    scaled derivatives are smaller, as they are for resolved data."""
    rng = np.random.default_rng(seed)
    M = m + 1
    S = rng.standard_normal(state_shape(m, n))
    i = np.arange(M)
    w = decay ** (i[:, None, None] + i[None, :, None] + i[None, None, :])
    return S * w[None, :, :, :, None, None, None]


def _coords(n, h, grid):
    return (np.arange(n) + (0.5 if grid else 0.0)) * h


def _gauss_1d(m, n, h, centre, sigma, grid, images):
    x = _coords(n, h, grid)
    rows = np.zeros((m + 1, n))
    for p in range(-images, images + 1):
        r = (x - centre - p) / sigma
        g = np.exp(-0.5 * r * r)
        # probabilists' Hermite polynomials He_i(r): d^i/dx^i g = (-1/sigma)^i He_i(r) g
        he_prev, he = np.zeros_like(r), np.ones_like(r)
        for i in range(m + 1):
            rows[i] += (h ** i / factorial(i)) * (-1.0 / sigma) ** i * he * g
            he_prev, he = he, r * he - i * he_prev
    return rows


def gaussian_pulse(m, n, h, centre=(0.5, 0.5, 0.5), sigma=0.05, grid=0, images=1):
    """u0 = exp(-|x - centre|^2 / (2 sigma^2)) over the 3^3 nearest periodic
    images, v0 = 0, sampled on the primal (grid 0) or dual (grid 1) grid."""
    g = [_gauss_1d(m, n[d], h[d], centre[d], sigma, grid, images) for d in range(3)]
    S = np.zeros(state_shape(m, n))
    S[0] = g[2][:, None, None, :, None, None] * g[1][None, :, None, None, :, None] \
        * g[0][None, None, :, None, None, :]
    return S


def product_standing_mode(m, n, h, k=(1, 1, 1)):
    """u0 = sin(2 pi k1 x) sin(2 pi k2 y) sin(2 pi k3 z), v0 = 0 on the
    primal grid."""
    rows = []
    for d in range(3):
        x = _coords(n[d], h[d], 0)
        rows.append(np.stack([(2 * pi * k[d] * h[d]) ** i / factorial(i)
                              * np.sin(2 * pi * k[d] * x + i * pi / 2) for i in range(m + 1)]))
    S = np.zeros(state_shape(m, n))
    S[0] = rows[2][:, None, None, :, None, None] * rows[1][None, :, None, None, :, None] \
        * rows[0][None, None, :, None, None, :]
    return S


def standing_mode_draw(seed, count=8, kmax=6):
    """Seeded wavenumbers k_r in {1..kmax}^3 and amplitudes A_r ~ U(-1, 1),
    drawn in that order."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(1, kmax + 1, size=(count, 3))
    amps = rng.uniform(-1.0, 1.0, size=count)
    return ks, amps


def standing_modes(m, n, h, seed, count=8, kmax=6):
    """u0 = sum_r A_r sin(2 pi k_r . x), v0 = 0 on the primal grid, with the
    seeded draw of ``standing_mode_draw``."""
    ks, amps = standing_mode_draw(seed, count, kmax)
    M = m + 1
    S = np.zeros(state_shape(m, n))
    X = [_coords(n[d], h[d], 0) for d in range(3)]
    z, y, x = np.meshgrid(X[2], X[1], X[0], indexing="ij")
    for k, A in zip(ks, amps):
        theta = 2 * pi * (k[0] * x + k[1] * y + k[2] * z)
        for i3 in range(M):
            for i2 in range(M):
                for i1 in range(M):
                    fac = ((2 * pi * k[0] * h[0]) ** i1 / factorial(i1)
                           * (2 * pi * k[1] * h[1]) ** i2 / factorial(i2)
                           * (2 * pi * k[2] * h[2]) ** i3 / factorial(i3))
                    S[0, i3, i2, i1] += A * fac * np.sin(theta + (i1 + i2 + i3) * pi / 2)
    return S


def batch_draw(seed, nsims=64, sides=(32, 48, 64, 96), orders=(1, 2, 3)):
    """Seeded batched workload: per simulation the grid sides (drawn per
    dimension from ``sides``), the order m, the pulse centre U(0.2, 0.8)^3 and
    width U(0.03, 0.08)."""
    rng = np.random.default_rng(seed)
    sims = []
    for _ in range(nsims):
        n = tuple(int(v) for v in rng.choice(sides, size=3))
        m = int(rng.choice(orders))
        centre = tuple(float(v) for v in rng.uniform(0.2, 0.8, size=3))
        sigma = float(rng.uniform(0.03, 0.08))
        sims.append({"m": m, "n": n, "h": tuple(1.0 / v for v in n), "centre": centre, "sigma": sigma})
    return sims


def receiver_draw(seed, n, count=32):
    """Seeded distinct receiver node indices (flat index z*n2*n1 + y*n1 + x)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n[0] * n[1] * n[2], size=count, replace=False)).astype(np.int64)


# ---------------------------------------------------------------------------
# Advection (Eq. 1): one field, layout A[i3, i2, i1, z, y, x].
# ---------------------------------------------------------------------------


def advection_random_state(m, n, seed, decay=0.5, dtype=np.float64):
    """Seeded one-field N(0, 1) state (shape (M, M, M, n3, n2, n1)), component
    i scaled by decay^|i| as in ``random_state``; drawn directly in ``dtype``."""
    rng = np.random.default_rng(seed)
    M = m + 1
    A = rng.standard_normal((M, M, M, n[2], n[1], n[0]), dtype=dtype)
    i = np.arange(M)
    w = (decay ** (i[:, None, None] + i[None, :, None] + i[None, None, :])).astype(dtype)
    A *= w[:, :, :, None, None, None]
    return A


def plane_wave(m, n, h, k=(1, 1, 1), phase=0.0, grid=0):
    """u = sin(2 pi k . x + phase) as one-field node data on the primal
    (grid 0) or dual (grid 1) grid.  Its scaled derivative of order i is
    prod_d (2 pi k_d h_d)^{i_d} / i_d! * sin(2 pi k . x + phase + |i| pi / 2)."""
    M = m + 1
    X = [_coords(n[d], h[d], grid) for d in range(3)]
    z, y, x = np.meshgrid(X[2], X[1], X[0], indexing="ij")
    arg = 2 * pi * (k[0] * x + k[1] * y + k[2] * z) + phase
    A = np.empty((M, M, M, n[2], n[1], n[0]))
    for i3 in range(M):
        for i2 in range(M):
            for i1 in range(M):
                w = ((2 * pi * k[0] * h[0]) ** i1 / factorial(i1) * (2 * pi * k[1] * h[1]) ** i2 / factorial(i2)
                     * (2 * pi * k[2] * h[2]) ** i3 / factorial(i3))
                A[i3, i2, i1] = w * np.sin(arg + (i1 + i2 + i3) * pi / 2)
    return A
