"""Plain FP64 oracle of the Hermite half step (TEST INFRASTRUCTURE ONLY).

Notation.  m is the paper's N (number of scaled derivatives per dimension
minus one); M = m + 1 and P = 2m + 2.  A state lives on one of two periodic
grids (primal nodes x_k = i h_k, dual nodes x_k = (i + 1/2) h_k, Sec. 2) and
is stored as ``S[f, i3, i2, i1, z, y, x]`` -- field f in (u, v), derivative
orders (i3, i2, i1) <= m along (x3, x2, x1), then the node (x3, x2, x1) with
x1 fastest (the tensor u[m3][m2][m1][n3][n2][n1] of Sec. 3.1, one per field).
Entry ``S[f, i3, i2, i1, node]`` approximates
h1^i1 h2^i2 h3^i3 / (i1! i2! i3!) * d^i f / dx^i at the node (Eq. 2 with the
per-dimension spacings of Eq. 3).

``h`` is always given as (h1, h2, h3) = (hx, hy, hz); ``dt`` is the FULL time
step of Eq. 4, so one half step evolves over tau = dt / 2 (Sec. 2: evolution
from t_n to t_{n+1/2}).  ``parity`` 0 maps primal -> dual (a dual node i is the
centre of the cell with corners i and i+1), parity 1 maps dual -> primal (a
primal node i is the centre of the cell with dual corners i-1 and i).
"""
from fractions import Fraction
from math import comb

import numpy as np

# ---------------------------------------------------------------------------
# 1-D Hermite interpolation operator H (Sec. 3.1; construction of the operator
# is left by the paper to its reference on variations of Hermite methods; here
# it is built from the interpolation conditions themselves).
# ---------------------------------------------------------------------------


def _fraction_inverse(A):
    """Exact Gauss-Jordan inverse of a square matrix of Fractions."""
    n = len(A)
    aug = [list(row) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if aug[r][col] != 0)
        aug[col], aug[piv] = aug[piv], aug[col]
        p = aug[col][col]
        aug[col] = [v / p for v in aug[col]]
        for r in range(n):
            if r != col and aug[r][col] != 0:
                f = aug[r][col]
                aug[r] = [vr - f * vc for vr, vc in zip(aug[r], aug[col])]
    return [row[n:] for row in aug]


def hermite_conditions_exact(m):
    """Matrix A of the 1-D Hermite conditions, exact.

    Row (side, i) with side 0 = left node at xi = -1/2 and side 1 = right node
    at xi = +1/2, column j = monomial xi^j, j = 0..2m+1.  For p(xi) = sum c_j
    xi^j the scaled derivative (1/i!) p^(i)(xi0) equals
    sum_j C(j, i) xi0^(j-i) c_j, which is what the node stores (Eq. 2 written
    in the scaled variable of Eq. 3).
    """
    M, P = m + 1, 2 * m + 2
    A = [[Fraction(0)] * P for _ in range(P)]
    for side, xi0 in ((0, Fraction(-1, 2)), (1, Fraction(1, 2))):
        for i in range(M):
            for j in range(i, P):
                A[side * M + i][j] = comb(j, i) * xi0 ** (j - i)
    return A


def hermite_matrix_exact(m):
    """H = A^{-1} as Fractions: H[j][(side, i)] maps the 2M node values of a
    cell edge ([left i = 0..m, right i = 0..m]) to the P monomial coefficients
    of the interpolant in xi = (x - x_centre) / h (Eq. 3, Sec. 3.1)."""
    return _fraction_inverse(hermite_conditions_exact(m))


def hermite_matrix(m):
    """H as an FP64 array of shape (P, P)."""
    return np.array([[float(v) for v in row] for row in hermite_matrix_exact(m)])


# ---------------------------------------------------------------------------
# Gathering the cell neighbourhood (Sec. 3.1: the 8 vertices of the cell that
# encapsulates the target node) into the local tensor u_loc[tz][ty][tx].
# ---------------------------------------------------------------------------


def _offset(parity):
    if parity not in (0, 1):
        raise ValueError("parity must be 0 (primal->dual) or 1 (dual->primal)")
    return 0 if parity == 0 else -1


def gather_cells(S, m, parity, z_cells=None):
    """Local tensors u_loc of every target cell in an output z-range.

    Returns U of shape (ncell, F, P, P, P) indexed [cell, f, tz, ty, tx] with
    t = side * M + i along each dimension (side 0 = lower corner, 1 = upper),
    cells ordered (z, y, x) with x fastest, z in ``z_cells``; F = S.shape[0]
    fields (2 for the wave equation, 1 for advection).
    """
    M, P = m + 1, 2 * m + 2
    F = S.shape[0]
    nz, ny, nx = S.shape[-3:]
    s = _offset(parity)
    zs = np.arange(nz) if z_cells is None else np.asarray(z_cells)
    ys, xs = np.arange(ny), np.arange(nx)
    U = np.empty((len(zs), ny, nx, F, P, P, P))
    for c in (0, 1):
        zi = (zs + s + c) % nz
        for b in (0, 1):
            yi = (ys + s + b) % ny
            for a in (0, 1):
                xi = (xs + s + a) % nx
                blk = S[:, :, :, :][..., zi, :, :][..., yi, :][..., xi]  # (2,M,M,M,cz,ny,nx)
                U[:, :, :, :, c * M:(c + 1) * M, b * M:(b + 1) * M, a * M:(a + 1) * M] = \
                    blk.transpose(4, 5, 6, 0, 1, 2, 3)
    return U.reshape(len(zs) * ny * nx, F, P, P, P)


# ---------------------------------------------------------------------------
# Alg. 1 / Alg. 2: reconstruction in x1, then x2, then x3.
# ---------------------------------------------------------------------------


def reconstruct(U, H):
    """Ru = H_x3 H_x2 H_x1 u_loc for a batch of local tensors (..., P, P, P)
    indexed [tz, ty, tx]; the result is indexed [jz, jy, jx] (coefficient of
    xi3^jz xi2^jy xi1^jx)."""
    P = H.shape[0]
    R = U @ H.T                       # along x1:  Ru[tz][ty][jx] = sum_k H[jx][k] u[tz][ty][k]
    R = H @ R                         # along x2:  over the ty axis
    sh = R.shape
    R = (H @ R.reshape(-1, P, P * P)).reshape(sh)   # along x3: over the tz axis
    return R


# ---------------------------------------------------------------------------
# Alg. 3 applied twice: second derivative of the coefficient tensor in one
# scaled variable, and the Laplacian of the wave equation.
# ---------------------------------------------------------------------------


def second_derivative(B, axis):
    """d^2/dxi^2 along ``axis`` of the coefficient tensor: entry j becomes
    (j+1)(j+2) B[j+2], zero for the top two indices (Alg. 3 applied twice
    with h = 1)."""
    P = B.shape[axis]
    out = np.zeros_like(B)
    j = np.arange(P - 2, dtype=float)
    src = np.take(B, np.arange(2, P), axis=axis)
    shape = [1] * B.ndim
    shape[axis] = P - 2
    idx = [slice(None)] * B.ndim
    idx[axis] = slice(0, P - 2)
    out[tuple(idx)] = src * ((j + 1) * (j + 2)).reshape(shape)
    return out


def laplacian(B, h):
    """Delta B for coefficient tensors (..., jz, jy, jx): d^2/dx_k^2 =
    h_k^{-2} d^2/dxi_k^2 (scaled variables of Eq. 3)."""
    hx, hy, hz = h
    return (second_derivative(B, -1) / hx ** 2 + second_derivative(B, -2) / hy ** 2
            + second_derivative(B, -3) / hz ** 2)


def wave_operator(Bu, Bv, c, h):
    """L(u, v) = (v, c^2 Delta u): the first-order scalar wave equation."""
    return Bv, c * c * laplacian(Bu, h)


def evolve_rk4(Bu, Bv, tau, c, h):
    """Classical four-stage Runge-Kutta over one half step tau."""
    k1u, k1v = wave_operator(Bu, Bv, c, h)
    k2u, k2v = wave_operator(Bu + 0.5 * tau * k1u, Bv + 0.5 * tau * k1v, c, h)
    k3u, k3v = wave_operator(Bu + 0.5 * tau * k2u, Bv + 0.5 * tau * k2v, c, h)
    k4u, k4v = wave_operator(Bu + tau * k3u, Bv + tau * k3v, c, h)
    return (Bu + tau / 6.0 * (k1u + 2 * k2u + 2 * k3u + k4u),
            Bv + tau / 6.0 * (k1v + 2 * k2v + 2 * k3v + k4v))


def evolve_taylor(Bu, Bv, tau, c, h, q=4):
    """Alg. 4 (Horner form of the q-stage Taylor series) for the wave
    operator: w <- Ru + (tau / k) L w for k = q, ..., 1."""
    wu, wv = Bu.copy(), Bv.copy()
    for k in range(q, 0, -1):
        lu, lv = wave_operator(wu, wv, c, h)
        wu, wv = Bu + tau / k * lu, Bv + tau / k * lv
    return wu, wv


# ---------------------------------------------------------------------------
# The per-cell map: reconstruct, evolve, truncate to j <= m (Sec. 2: the
# coefficients of the cell polynomial are the scaled derivatives at the cell
# centre, i.e. the data of the dual node).
# ---------------------------------------------------------------------------


def cell_map(U, m, h, c, tau, evolve="rk4", q=4):
    """Map a batch of local tensors (ncell, 2, P, P, P) to the new node data
    (ncell, 2, M, M, M) [cell, f, i3, i2, i1].  evolve = "rk4" (classical
    RK4), "taylor" (Alg. 4 with q stages) or "none"."""
    M = m + 1
    H = hermite_matrix(m)
    R = reconstruct(U, H)
    Bu, Bv = R[:, 0], R[:, 1]
    if evolve == "rk4":
        Bu, Bv = evolve_rk4(Bu, Bv, tau, c, h)
    elif evolve == "taylor":
        Bu, Bv = evolve_taylor(Bu, Bv, tau, c, h, q)
    elif evolve == "none":
        pass
    else:
        raise ValueError(evolve)
    return np.stack([Bu[:, :M, :M, :M], Bv[:, :M, :M, :M]], axis=1)


def half_step(S, m, h, c, dt, parity, evolve="rk4", z_cells=None, chunk_cells=8192, q=4):
    """One half step of the whole grid (vectorised over cells).

    ``z_cells`` restricts the output to those z layers (the rest of the
    returned array is NaN); the work is done in batches of about
    ``chunk_cells`` cells, each batch independent of the others.
    """
    S = np.asarray(S, dtype=np.float64)
    M = m + 1
    assert S.shape[:4] == (2, M, M, M), S.shape
    nz, ny, nx = S.shape[-3:]
    tau = 0.5 * dt
    out = np.full_like(S, np.nan)
    zs = np.arange(nz) if z_cells is None else np.asarray(z_cells)
    per = max(1, chunk_cells // (ny * nx))
    for k in range(0, len(zs), per):
        zc = zs[k:k + per]
        U = gather_cells(S, m, parity, zc)
        V = cell_map(U, m, h, c, tau, evolve, q)          # (ncell, 2, M, M, M)
        out[..., zc, :, :] = V.reshape(len(zc), ny, nx, 2, M, M, M).transpose(3, 4, 5, 6, 0, 1, 2)
    return out


def run(S, m, h, c, dt, nhalf, parity0=0, evolve="rk4", q=4):
    """nhalf half steps alternating primal->dual and dual->primal (Sec. 2)."""
    p = parity0
    for _ in range(nhalf):
        S = half_step(S, m, h, c, dt, p, evolve, q=q)
        p ^= 1
    return S


# ---------------------------------------------------------------------------
# Literal version: plain loops over cells and the loops of Alg. 1 -- 4, for
# tiny grids.  Used to check the vectorised version.
# ---------------------------------------------------------------------------


def half_step_literal(S, m, h, c, dt, parity):
    S = np.asarray(S, dtype=np.float64)
    M, P = m + 1, 2 * m + 2
    nz, ny, nx = S.shape[-3:]
    s = _offset(parity)
    H = hermite_matrix(m)
    tau = 0.5 * dt
    hx, hy, hz = h
    out = np.zeros_like(S)

    def mode_product(A, axis):
        # Alg. 1 written with explicit loops along the chosen dimension.
        R = np.zeros((P, P, P))
        for tz in range(P):
            for ty in range(P):
                for tx in range(P):
                    acc = 0.0
                    for k in range(P):
                        if axis == 0:
                            acc += H[tx][k] * A[tz][ty][k]
                        elif axis == 1:
                            acc += H[ty][k] * A[tz][k][tx]
                        else:
                            acc += H[tz][k] * A[k][ty][tx]
                    R[tz][ty][tx] = acc
        return R

    def lap(B):
        L = np.zeros((P, P, P))
        for jz in range(P):
            for jy in range(P):
                for jx in range(P):
                    acc = 0.0
                    if jx + 2 < P:
                        acc += (jx + 1) * (jx + 2) * B[jz][jy][jx + 2] / hx ** 2
                    if jy + 2 < P:
                        acc += (jy + 1) * (jy + 2) * B[jz][jy + 2][jx] / hy ** 2
                    if jz + 2 < P:
                        acc += (jz + 1) * (jz + 2) * B[jz + 2][jy][jx] / hz ** 2
                    L[jz][jy][jx] = acc
        return L

    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                R = []
                for f in range(2):
                    u = np.zeros((P, P, P))
                    for cz in range(2):
                        for by in range(2):
                            for ax in range(2):
                                node = ((z + s + cz) % nz, (y + s + by) % ny, (x + s + ax) % nx)
                                for i3 in range(M):
                                    for i2 in range(M):
                                        for i1 in range(M):
                                            u[cz * M + i3][by * M + i2][ax * M + i1] = \
                                                S[(f, i3, i2, i1) + node]
                    R.append(mode_product(mode_product(mode_product(u, 0), 1), 2))
                Bu, Bv = R
                # classical RK4 with L(u, v) = (v, c^2 Delta u)
                k1u, k1v = Bv, c * c * lap(Bu)
                k2u, k2v = Bv + 0.5 * tau * k1v, c * c * lap(Bu + 0.5 * tau * k1u)
                k3u, k3v = Bv + 0.5 * tau * k2v, c * c * lap(Bu + 0.5 * tau * k2u)
                k4u, k4v = Bv + tau * k3v, c * c * lap(Bu + tau * k3u)
                Nu = Bu + tau / 6 * (k1u + 2 * k2u + 2 * k3u + k4u)
                Nv = Bv + tau / 6 * (k1v + 2 * k2v + 2 * k3v + k4v)
                for i3 in range(M):
                    for i2 in range(M):
                        for i1 in range(M):
                            out[0, i3, i2, i1, z, y, x] = Nu[i3][i2][i1]
                            out[1, i3, i2, i1, z, y, x] = Nv[i3][i2][i1]
    return out


# ---------------------------------------------------------------------------
# The half step as an explicit linear map, its transpose (discrete adjoint).
# ---------------------------------------------------------------------------


def cell_matrix(m, h, c, dt, evolve="rk4", q=4):
    """Dense per-cell matrix W (2 M^3 x 2 P^3) of the half step, built by
    applying the per-cell map to unit local tensors.  Column index (f, tz, ty,
    tx), row index (f, i3, i2, i1)."""
    M, P = m + 1, 2 * m + 2
    n_in = 2 * P ** 3
    E = np.eye(n_in).reshape(n_in, 2, P, P, P)
    out = cell_map(E, m, h, c, 0.5 * dt, evolve, q)
    return out.reshape(n_in, 2 * M ** 3).T.copy()


def corner_blocks(W, m):
    """Split W into the 8 corner blocks W[(a, b, c)] of shape (2M^3, 2M^3),
    (a, b, c) the corner offsets along (x1, x2, x3); the column index of a
    block is a node component (f, i3, i2, i1)."""
    M = m + 1
    W7 = W.reshape(2 * M ** 3, 2, 2, M, 2, M, 2, M)   # out, f, cz, i3, by, i2, ax, i1
    blocks = {}
    for a in (0, 1):
        for b in (0, 1):
            for cc in (0, 1):
                blocks[(a, b, cc)] = W7[:, :, cc, :, b, :, a, :].reshape(2 * M ** 3, 2 * M ** 3)
    return blocks


def half_step_matrix_form(S, m, h, c, dt, parity):
    """The forward half step written with the corner blocks: out(o) =
    sum_abc W_abc in(o + s + abc)."""
    M = m + 1
    s = _offset(parity)
    n = S.shape[-3:]
    X = S.reshape(2 * M ** 3, -1)
    out = np.zeros_like(X)
    for (a, b, cc), Wb in corner_blocks(cell_matrix(m, h, c, dt), m).items():
        sh = np.roll(S.reshape((2 * M ** 3,) + n), shift=(-(s + cc), -(s + b), -(s + a)), axis=(1, 2, 3))
        out += Wb @ sh.reshape(2 * M ** 3, -1)
    return out.reshape(S.shape)


def adjoint_half_step(G, m, h, c, dt, parity, evolve="rk4", q=4):
    """Transpose of the half step of the given parity: for an output-grid
    cotangent G, returns the input-grid cotangent sum over the 8 cells that
    contain each node of W_abc^T G(cell)."""
    M = m + 1
    s = _offset(parity)
    n = G.shape[-3:]
    Gf = G.reshape((2 * M ** 3,) + n)
    out = np.zeros((2 * M ** 3, int(np.prod(n))))
    for (a, b, cc), Wb in corner_blocks(cell_matrix(m, h, c, dt, evolve, q), m).items():
        sh = np.roll(Gf, shift=(s + cc, s + b, s + a), axis=(1, 2, 3))
        out += Wb.T @ sh.reshape(2 * M ** 3, -1)
    return out.reshape(G.shape)


def adjoint_half_step_literal(G, m, h, c, dt, parity):
    """The same transpose as an explicit scatter-add over cells."""
    M = m + 1
    s = _offset(parity)
    nz, ny, nx = G.shape[-3:]
    blocks = corner_blocks(cell_matrix(m, h, c, dt), m)
    out = np.zeros_like(G)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                g = G[..., z, y, x].reshape(-1)
                for (a, b, cc), Wb in blocks.items():
                    node = ((z + s + cc) % nz, (y + s + b) % ny, (x + s + a) % nx)
                    out[(Ellipsis,) + node] += (Wb.T @ g).reshape(2, M, M, M)
    return out


# ---------------------------------------------------------------------------
# Norms and energy.
# ---------------------------------------------------------------------------


def error_norms(a, b, component_mask=0b111):
    """(max_abs, max_rel, l2_abs, l2_rel) of a - b over the selected
    components: bit0 field u, bit1 field v, bit2 all derivative orders (else
    the values i = (0,0,0) only).  max_rel = max|a-b| / max|b|, l2_abs =
    ||a-b||_2, l2_rel = ||a-b||_2 / ||b||_2."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    fields = [f for f in (0, 1) if component_mask >> f & 1]
    if component_mask & 4:
        sa, sb = a[fields], b[fields]
    else:
        sa, sb = a[fields, 0, 0, 0], b[fields, 0, 0, 0]
    d = sa - sb
    max_abs = float(np.max(np.abs(d))) if d.size else 0.0
    max_b = float(np.max(np.abs(sb))) if d.size else 0.0
    l2 = float(np.sum(d * d))
    l2b = float(np.sum(sb * sb))
    return (max_abs, max_abs / max_b if max_b > 0 else np.inf,
            float(np.sqrt(l2)), float(np.sqrt(l2 / l2b)) if l2b > 0 else np.inf)


def energy(S, m, h, c, parity_of_grid=0):
    """E = sum over cells of the integral over the cell of B_v^2 + c^2 |grad B_u|^2,
    B the interpolant of the current data (Eq. 3) on each cell of the current
    grid.  The paper defines no energy; this is the natural quadratic
    invariant of the wave equation evaluated on the interpolants.  Pinned by
    a Gauss-Legendre quadrature of SciPy's Hermite interpolant and by the
    closed-form energy of a standing mode (tests/test_oracle_energy.py)."""
    M, P = m + 1, 2 * m + 2
    H = hermite_matrix(m)
    U = gather_cells(S, m, parity_of_grid)
    R = reconstruct(U, H)
    Bu, Bv = R[:, 0], R[:, 1]
    # monomial moments on [-1/2, 1/2]
    mom = np.array([0.0 if k % 2 else 2 * 0.5 ** (k + 1) / (k + 1) for k in range(2 * P)])
    G = np.array([[mom[j + k] for k in range(P)] for j in range(P)])
    D = np.zeros((P, P))
    for j in range(P - 1):
        D[j, j + 1] = j + 1            # d/dxi along one axis (Alg. 3, h = 1)

    def quad(A):
        # sum over cells of the integral of A^2, A indexed (cell, jz, jy, jx)
        return float(np.einsum("nzyx,zZ,yY,xX,nZYX->", A, G, G, G, A))

    hx, hy, hz = h
    vol = hx * hy * hz
    e = quad(Bv)
    e += c * c * quad(np.einsum("xX,nzyX->nzyx", D, Bu)) / hx ** 2
    e += c * c * quad(np.einsum("yY,nzYx->nzyx", D, Bu)) / hy ** 2
    e += c * c * quad(np.einsum("zZ,nZyx->nzyx", D, Bu)) / hz ** 2
    return e * vol
