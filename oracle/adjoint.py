"""Dense adjoint gradient of the solve-and-evaluate map -- test infrastructure.

Only tests/ (and the bench's reference leg) use this module; the product path never
imports it.  It shares no code with the CUDA library.

Variables: the planar node positions xi_j = X_j + i Y_j (Sec. 3) with the curve
derivatives xi'_j, xi''_j held fixed.  The oracle maps the nodes back to the sphere
(the inverse of Sec. 3's projection, differentiated along the curve), builds the
bordered matrix in the 3D form -- the double-layer kernel of Sec. 2 (Eq. kern1),
its diagonal limit (Appendix A) and 2 G (Eq. greens_func) -- and the evaluation
matrix of Eq. u_multi, solves densely (LAPACK), and differentiates every entry that
depends on xi_j by the complex step: for a real-analytic f, f(X + i h) =
f(X) + i h f'(X) + O(h^2), so Im f(X + i h) / h is f'(X) to rounding for tiny h.

For A z = b (b = [2 g; 0]), u = C z and a loss L(u) with ubar = dL/du:
    A^T lam = C^T ubar,   dL/dg = 2 lam_sigma,
    dL/dX_j = ubar^T (dC/dX_j) z - lam^T (dA/dX_j) z   (likewise Y_j),
where only row j, column j of A and column j of C depend on xi_j.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

_TWO_PI = 2.0 * np.pi
_STEP = 1e-30


def sphere_from_plane(X, Y, a, b, a2, b2):
    """x, x', x'' (alpha-derivatives) on the unit sphere of planar nodes
    xi = X + iY with xi' = a + ib and xi'' = a2 + i b2: x = (2X, 2Y, X^2 + Y^2 - 1)/D,
    D = 1 + X^2 + Y^2, differentiated twice along the curve.  Rational in X, Y, so it
    accepts complex-step arguments."""
    D = 1 + X * X + Y * Y
    D1 = 2 * (X * a + Y * b)
    D2 = 2 * (a * a + b * b + X * a2 + Y * b2)

    def first(U, u1):  # d/dalpha (2 U / D)
        return 2 * (u1 * D - U * D1) / D ** 2

    def second(U, u1, u2):  # d2/dalpha2 (2 U / D)
        return 2 * ((u2 * D - U * D2) / D ** 2 - 2 * D1 * (u1 * D - U * D1) / D ** 3)

    x = np.stack([2 * X / D, 2 * Y / D, 1 - 2 / D], axis=-1)
    dx = np.stack([first(X, a), first(Y, b), 2 * D1 / D ** 2], axis=-1)
    d2x = np.stack([second(X, a, a2), second(Y, b, b2), 2 * (D2 / D ** 2 - 2 * D1 * D1 / D ** 3)],
                   axis=-1)
    return x, dx, d2x


def _kernel(t, xs, dxs):
    """Double-layer kernel per unit alpha, -(1/2pi) (t - x)·(x × x')/|t - x|^2 (Eq. kern1),
    broadcast over t (.., 3) and sources (.., 3)."""
    n = np.cross(xs, dxs)
    d = t - xs
    return -np.sum(d * n, axis=-1) / (_TWO_PI * np.sum(d * d, axis=-1))


def _diag(x, dx, d2x):
    """Diagonal limit per unit alpha, -(1/4pi) x·(x' × x'')/|x'|^2 (Appendix A)."""
    return -np.sum(x * np.cross(dx, d2x), axis=-1) / (2 * _TWO_PI * np.sum(dx * dx, axis=-1))


def _green(t, c):
    """G = -(1/4pi) log|t - c|^2 + (1/4pi) log 2 (Eq. greens_func)."""
    d = t - c
    return (np.log(2.0) - np.log(np.sum(d * d, axis=-1))) / (2 * _TWO_PI)


def _h(ptr):
    ptr = np.asarray(ptr)
    return np.repeat(_TWO_PI / np.diff(ptr), np.diff(ptr))


def dense_system(ptr, x, dx, d2x, c):
    """The bordered matrix (Sec. 5, Eq. matrix_eqns; doubled scaling) in the 3D form."""
    ptr = np.asarray(ptr)
    N, M = int(ptr[-1]), len(ptr) - 1
    h = _h(ptr)
    A = np.zeros((N + M, N + M))
    with np.errstate(invalid="ignore", divide="ignore"):  # i == j, replaced below
        K = _kernel(x[:, None, :], x[None, :, :], dx[None, :, :])
    np.fill_diagonal(K, 0.0)
    A[:N, :N] = 2 * h[None, :] * K
    A[np.arange(N), np.arange(N)] = 1 + 2 * h * _diag(x, dx, d2x)
    A[:N, N:] = 2 * _green(x[:, None, :], c[None, :, :])
    for r in range(M - 1):
        A[N + r, ptr[r + 1]:ptr[r + 2]] = 1.0
    A[N + M - 1, N:] = 1.0
    return A


def evaluation_matrix(ptr, x, dx, c, t):
    """C with u = C [sigma; a] at the targets t (Eq. u_multi)."""
    h = _h(ptr)
    W = h[None, :] * _kernel(t[:, None, :], x[None, :, :], dx[None, :, :])
    return np.hstack([W, _green(t[:, None, :], c[None, :, :])])


def forward(ptr, xi, dxi, d2xi, c, t, g):
    """u at the targets for planar nodes (N x 2 each), sphere centres c and targets t."""
    x, dx, d2x = sphere_from_plane(xi[:, 0], xi[:, 1], dxi[:, 0], dxi[:, 1], d2xi[:, 0], d2xi[:, 1])
    N, M = len(xi), len(ptr) - 1
    A = dense_system(ptr, x, dx, d2x, c)
    z = sla.solve(A, np.concatenate([2 * np.asarray(g), np.zeros(M)]))
    return evaluation_matrix(ptr, x, dx, c, t) @ z


def gradient(ptr, xi, dxi, d2xi, c, t, g, loss_grad):
    """(L's gradient in g (N), gradient in xi (N x 2), u) for u = forward(...), with
    loss_grad(u) = dL/du."""
    ptr = np.asarray(ptr)
    N, M = len(xi), len(ptr) - 1
    X, Y = xi[:, 0], xi[:, 1]
    a, b, a2, b2 = dxi[:, 0], dxi[:, 1], d2xi[:, 0], d2xi[:, 1]
    x, dx, d2x = sphere_from_plane(X, Y, a, b, a2, b2)
    h = _h(ptr)
    A = dense_system(ptr, x, dx, d2x, c)
    C = evaluation_matrix(ptr, x, dx, c, t)
    lu = sla.lu_factor(A)
    z = sla.lu_solve(lu, np.concatenate([2 * np.asarray(g), np.zeros(M)]))
    u = C @ z
    ub = loss_grad(u)
    lam = sla.lu_solve(lu, C.T @ ub, trans=1)
    sig, zs = z[:N], z
    grad_xi = np.zeros((N, 2))
    others = np.ones(N, dtype=bool)
    for j in range(N):
        others[j] = False
        for d in (0, 1):
            Xj = X[j] + (1j * _STEP if d == 0 else 0.0)
            Yj = Y[j] + (1j * _STEP if d == 1 else 0.0)
            xj, dxj, d2xj = sphere_from_plane(Xj, Yj, a[j], b[j], a2[j], b2[j])
            # row j: node j as the target of the others, its diagonal, its row of 2 G
            row = 2 * h[others] * _kernel(xj[None, :], x[others], dx[others])
            dia = 1 + 2 * h[j] * _diag(xj, dxj, d2xj)
            erow = 2 * _green(xj[None, :], c)
            # column j: node j as the source seen from the others and from the targets
            col = 2 * h[j] * _kernel(x[others], xj[None, :], dxj[None, :])
            ccol = h[j] * _kernel(t, xj[None, :], dxj[None, :])
            drow, ddia, derow = row.imag / _STEP, dia.imag / _STEP, erow.imag / _STEP
            dcol, dccol = col.imag / _STEP, ccol.imag / _STEP
            lam_dA_z = (lam[j] * (drow @ sig[others] + ddia * sig[j] + derow @ zs[N:])
                        + (lam[:N][others] @ dcol) * sig[j])
            grad_xi[j, d] = (ub @ dccol) * sig[j] - lam_dA_z
        others[j] = True
    return 2 * lam[:N], grad_xi, u
