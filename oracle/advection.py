"""Plain FP64 oracle of the Hermite half step for the 3-D advection equation
(TEST INFRASTRUCTURE ONLY: only tests, the smoke check and the bench's CPU
baseline use it; the product path never does).

Sec. 2 introduces Hermite methods on the advection equation (Eq. 1)
u_t = u_x1 + u_x2 + u_x3.  Here it is taken with a general constant velocity,
u_t = a1 u_x1 + a2 u_x2 + a3 u_x3 (Eq. 1 is a = (1, 1, 1)), so the exact
solution is u(x, t) = u(x + a t, 0).

A state is one field of scaled derivatives A[i3, i2, i1, z, y, x] with the
layout, node convention and parities of ``oracle.hermite`` (one field instead
of the wave equation's two).  One half step, for every cell:

1. gathers the 8 corner nodes and builds the tensor Hermite interpolant of
   degree 2m+1 per variable (Eq. 3, Alg. 1/2);
2. evolves it over tau = dt / 2 with the q-stage Hermite-Taylor series
   (Alg. 4, in Horner form; ``evolve_recursion`` is the coefficient recursion
   of Eq. 5, the same polynomial);
3. keeps the coefficients of order <= m, the data of the dual node (Sec. 2).

q = 3(2m+1) = d(2N+1) stages (the default) is the paper's choice for the
largest time step; for the cell polynomial it is the whole series, so the
half step then equals the exact translation of the interpolant.
"""
import numpy as np

from . import hermite


def full_q(m):
    """d(2N+1) with d = 3 dimensions and N = m (Sec. 3.2)."""
    return 3 * (2 * m + 1)


# ---------------------------------------------------------------------------
# Alg. 3: the derivative of the coefficient tensor in one scaled variable.
# ---------------------------------------------------------------------------


def first_derivative(B, axis):
    """d/dxi along ``axis``: entry j becomes (j+1) B[j+1], the top entry 0
    (Alg. 3 with h = 1; the physical derivative divides by h_k)."""
    P = B.shape[axis]
    out = np.zeros_like(B)
    j = np.arange(P - 1, dtype=float)
    src = np.take(B, np.arange(1, P), axis=axis)
    shape = [1] * B.ndim
    shape[axis] = P - 1
    idx = [slice(None)] * B.ndim
    idx[axis] = slice(0, P - 1)
    out[tuple(idx)] = src * (j + 1).reshape(shape)
    return out


def advection_operator(B, a, h):
    """L B = sum_k a_k d/dx_k B for coefficient tensors (..., jz, jy, jx)
    (d/dx_k = h_k^{-1} d/dxi_k, scaled variables of Eq. 3)."""
    return (a[0] / h[0] * first_derivative(B, -1) + a[1] / h[1] * first_derivative(B, -2)
            + a[2] / h[2] * first_derivative(B, -3))


def evolve_taylor(B, tau, a, h, q):
    """Alg. 4: w <- Ru + (tau / k) L w for k = q, ..., 1 (Horner form of
    sum_{s <= q} (tau L)^s / s! Ru)."""
    w = B.copy()
    for k in range(q, 0, -1):
        w = B + tau / k * advection_operator(w, a, h)
    return w


def evolve_recursion(B, dt, a, h, q):
    """Eq. 4/5: space-time coefficients b_{j,s} in powers of (t - t_n)/dt,
    b_{j,s+1} = sum_k (j_k + 1)/(s + 1) * a_k dt / h_k * b_{j + e_k, s},
    then the series evaluated at t_{n+1/2}, i.e. sum_s b_{j,s} (1/2)^s."""
    b = B.copy()
    acc = B.copy()
    P = B.shape[-1]
    j = np.arange(P, dtype=float)
    for s in range(q):
        nxt = np.zeros_like(b)
        # along x1 (last axis), x2, x3: shift j + e_k down by one
        nxt[..., :, :, :P - 1] += (j[1:] / (s + 1) * a[0] * dt / h[0]) * b[..., :, :, 1:]
        nxt[..., :, :P - 1, :] += (j[1:, None] / (s + 1) * a[1] * dt / h[1]) * b[..., :, 1:, :]
        nxt[..., :P - 1, :, :] += (j[1:, None, None] / (s + 1) * a[2] * dt / h[2]) * b[..., 1:, :, :]
        b = nxt
        acc = acc + b * 0.5 ** (s + 1)
    return acc


# ---------------------------------------------------------------------------
# The half step.
# ---------------------------------------------------------------------------


def cell_map(U, m, h, a, tau, q=None):
    """Local tensors (ncell, P, P, P) -> new node data (ncell, M, M, M)."""
    M = m + 1
    q = full_q(m) if q is None else q
    R = hermite.reconstruct(U, hermite.hermite_matrix(m))
    R = evolve_taylor(R, tau, a, h, q)
    return R[:, :M, :M, :M]


def half_step(A, m, h, a, dt, parity, q=None, z_cells=None, chunk_cells=8192):
    """One half step of the whole grid; A has shape (M, M, M, nz, ny, nx).
    ``z_cells`` restricts the output to those z layers (the rest is NaN)."""
    A = np.asarray(A, dtype=np.float64)
    M = m + 1
    assert A.shape[:3] == (M, M, M), A.shape
    nz, ny, nx = A.shape[-3:]
    out = np.full_like(A, np.nan)
    zs = np.arange(nz) if z_cells is None else np.asarray(z_cells)
    per = max(1, chunk_cells // (ny * nx))
    for k in range(0, len(zs), per):
        zc = zs[k:k + per]
        U = hermite.gather_cells(A[None], m, parity, zc)[:, 0]
        V = cell_map(U, m, h, a, 0.5 * dt, q)
        out[..., zc, :, :] = V.reshape(len(zc), ny, nx, M, M, M).transpose(3, 4, 5, 0, 1, 2)
    return out


def run(A, m, h, a, dt, nhalf, parity0=0, q=None):
    """nhalf half steps alternating primal->dual and dual->primal."""
    p = parity0
    for _ in range(nhalf):
        A = half_step(A, m, h, a, dt, p, q)
        p ^= 1
    return A


# ---------------------------------------------------------------------------
# Fourier symbol (Sec. 2's stability condition).
# ---------------------------------------------------------------------------


def cell_matrix(m, h, a, dt, q=None):
    """Dense per-cell matrix (M^3 x P^3) of the half step."""
    P = 2 * m + 2
    E = np.eye(P ** 3).reshape(P ** 3, P, P, P)
    return cell_map(E, m, h, a, 0.5 * dt, q).reshape(P ** 3, -1).T


def max_spectral_radius(m, lam, q=None, npts=7, dims=3):
    """max over a theta grid of rho(G(theta)) for h = 1 and a = lam / tau in
    every dimension ``dims`` (1: a = (lam/tau, 0, 0), a mode along x1 only),
    so that a_k tau / h_k = lam."""
    M = m + 1
    tau = 0.5
    a = (lam / tau, lam / tau if dims == 3 else 0.0, lam / tau if dims == 3 else 0.0)
    W = cell_matrix(m, (1.0, 1.0, 1.0), a, 2 * tau, q).reshape(M ** 3, 2, M, 2, M, 2, M)
    th = np.linspace(0.0, np.pi, npts)
    grid2 = th if dims == 3 else [0.0]
    rho = 0.0
    for t1 in th:
        for t2 in grid2:
            for t3 in grid2:
                G = 0
                for cz in (0, 1):
                    for cy in (0, 1):
                        for cx in (0, 1):
                            blk = W[:, cz, :, cy, :, cx, :].reshape(M ** 3, M ** 3)
                            G = G + blk * np.exp(1j * (t1 * (cx - 0.5) + t2 * (cy - 0.5) + t3 * (cz - 0.5)))
                rho = max(rho, float(np.max(np.abs(np.linalg.eigvals(G)))))
    return rho
