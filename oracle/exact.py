"""Closed-form solutions of u_t = v, v_t = c^2 Delta u on the periodic unit
cube, sampled as node data (Eq. 2 with the per-dimension spacings of Eq. 3).
TEST INFRASTRUCTURE ONLY.

Each function returns an array ``S[f, i3, i2, i1, z, y, x]`` whose entry is
h1^i1 h2^i2 h3^i3 / (i1! i2! i3!) d^i f(x_node, t), f = u or v, on the primal
grid (node x_k = i h_k) or the dual grid (x_k = (i + 1/2) h_k).
"""
from math import factorial, pi

import numpy as np


def node_coords(n, h, grid):
    """1-D node coordinates of the primal (grid = 0) or dual (grid = 1) grid."""
    return (np.arange(n) + (0.5 if grid else 0.0)) * h


def _scaled_sin_derivs(theta, k, h, m):
    """Rows i = 0..m of (h^i / i!) d^i/dx^i sin(2 pi k x + phase) evaluated as
    (2 pi k h)^i / i! * sin(theta + i pi / 2), theta the phase at the nodes."""
    return np.stack([(2 * pi * k * h) ** i / factorial(i) * np.sin(theta + i * pi / 2)
                     for i in range(m + 1)])


def product_mode(m, n, h, c, t, k=(1, 1, 1), amp=1.0, grid=0):
    """u = amp * sin(2 pi k1 x) sin(2 pi k2 y) sin(2 pi k3 z) cos(w t),
    v = u_t, w = 2 pi c |k|.  ``n`` and ``h`` are (n1, n2, n3), (h1, h2, h3)."""
    M = m + 1
    w = 2 * pi * c * np.sqrt(np.sum(np.square(k)))
    per = []
    for d in range(3):
        x = node_coords(n[d], h[d], grid)
        per.append(_scaled_sin_derivs(2 * pi * k[d] * x, k[d], h[d], m))     # (M, n_d)
    sx, sy, sz = per
    spatial = np.einsum("az,by,cx->abczyx", sz, sy, sx)          # (i3, i2, i1, z, y, x)
    S = np.empty((2, M, M, M, n[2], n[1], n[0]))
    S[0] = amp * np.cos(w * t) * spatial
    S[1] = -amp * w * np.sin(w * t) * spatial
    return S


def plane_modes(m, n, h, c, t, ks, amps, grid=0):
    """u = sum_r A_r sin(2 pi k_r . x) cos(2 pi |k_r| c t), v = u_t."""
    M = m + 1
    S = np.zeros((2, M, M, M, n[2], n[1], n[0]))
    X = [node_coords(n[d], h[d], grid) for d in range(3)]
    z, y, x = np.meshgrid(X[2], X[1], X[0], indexing="ij")
    for k, A in zip(ks, amps):
        w = 2 * pi * c * np.sqrt(np.sum(np.square(k)))
        theta = 2 * pi * (k[0] * x + k[1] * y + k[2] * z)
        for i3 in range(M):
            for i2 in range(M):
                for i1 in range(M):
                    fac = ((2 * pi * k[0] * h[0]) ** i1 / factorial(i1)
                           * (2 * pi * k[1] * h[1]) ** i2 / factorial(i2)
                           * (2 * pi * k[2] * h[2]) ** i3 / factorial(i3))
                    sp = fac * np.sin(theta + (i1 + i2 + i3) * pi / 2)
                    S[0, i3, i2, i1] += A * np.cos(w * t) * sp
                    S[1, i3, i2, i1] += -A * w * np.sin(w * t) * sp
    return S


def _hermite_he(nmax, x):
    """Probabilists' Hermite polynomials He_0..He_nmax at x
    (He_{n+1} = x He_n - n He_{n-1})."""
    out = [np.ones_like(x), x.copy()]
    for k in range(1, nmax):
        out.append(x * out[k] - k * out[k - 1])
    return out[:nmax + 1]


def gaussian_1d(m, n, h, centre, sigma, grid=0, images=1):
    """Rows i = 0..m of (h^i / i!) d^i/dx^i of sum_{p=-images..images}
    exp(-(x - centre - p)^2 / (2 sigma^2)); d^i g = (-1/sigma)^i He_i g."""
    x = node_coords(n, h, grid)
    out = np.zeros((m + 1, n))
    for p in range(-images, images + 1):
        r = (x - centre - p) / sigma
        g = np.exp(-0.5 * r * r)
        He = _hermite_he(m, r)
        for i in range(m + 1):
            out[i] += h ** i / factorial(i) * (-1.0 / sigma) ** i * He[i] * g
    return out


def gaussian_pulse(m, n, h, centre=(0.5, 0.5, 0.5), sigma=0.05, grid=0, images=1):
    """u0 = exp(-|x - centre|^2 / (2 sigma^2)) summed over the 3^3 nearest
    periodic images (a product of 1-D image sums), v0 = 0."""
    M = m + 1
    g = [gaussian_1d(m, n[d], h[d], centre[d], sigma, grid, images) for d in range(3)]
    S = np.zeros((2, M, M, M, n[2], n[1], n[0]))
    S[0] = np.einsum("az,by,cx->abczyx", g[2], g[1], g[0])
    return S


def poly_cell_data(m, coeffs_u, coeffs_v, h, xc=(0.0, 0.0, 0.0)):
    """Node data at the 8 corners of one cell for the polynomials
    u = sum coeffs_u[a,b,c] x^a y^b z^c (and v likewise) around corner
    coordinates xc +- h/2.  Returns u_loc of shape (2, P, P, P) indexed
    [f, tz, ty, tx] with t = side * M + i (side 0 at xc - h/2)."""
    M, P = m + 1, 2 * m + 2
    U = np.zeros((2, P, P, P))
    for f, C in enumerate((coeffs_u, coeffs_v)):
        C = np.asarray(C, dtype=float)
        for cz in range(2):
            for by in range(2):
                for ax in range(2):
                    pt = [xc[0] + (ax - 0.5) * h[0], xc[1] + (by - 0.5) * h[1], xc[2] + (cz - 0.5) * h[2]]
                    for i3 in range(M):
                        for i2 in range(M):
                            for i1 in range(M):
                                U[f, cz * M + i3, by * M + i2, ax * M + i1] = \
                                    poly_scaled_derivative(C, (i1, i2, i3), pt, h)
    return U


def poly_scaled_derivative(C, order, pt, h):
    """(h^i / i!) d^i p(pt) for p = sum C[a,b,c] x^a y^b z^c, i = order
    (i1, i2, i3)."""
    from math import comb
    val = 0.0
    for a in range(C.shape[0]):
        for b in range(C.shape[1]):
            for cc in range(C.shape[2]):
                if C[a, b, cc] == 0 or a < order[0] or b < order[1] or cc < order[2]:
                    continue
                term = C[a, b, cc]
                for e, i, x, hh in ((a, order[0], pt[0], h[0]), (b, order[1], pt[1], h[1]),
                                    (cc, order[2], pt[2], h[2])):
                    term *= comb(e, i) * x ** (e - i) * hh ** i
                val += term
    return val
