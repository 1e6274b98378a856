"""Discrete Helmholtz operator and its direct solve (CPU, float64).

TEST INFRASTRUCTURE: see the package header for who may import this.

Definitions (Sec. 3.1, Eq. 3.1 and Eq. 3.2; Sec. 3.4, Eq. 3.12):

    H(m, w) u = -Lap_h u - w^2 m (1 - i gamma) u
    P(m, w) u = -Lap_h u - w^2 m (alpha - i beta) u          (alpha = 1)

with m = kappa^2 the squared slowness, Lap_h the standard second-order
central-difference Laplacian on a node grid of spacings (hx, hz), and zero
values on the ghost nodes one cell outside every edge of the grid.  The top
edge is therefore a pressure-release (reflecting) surface, as the paper wants
for the sea surface (Sec. 4.1); the other edges are made non-reflecting by
the absorbing layer gamma.  H is complex symmetric (H^T = H), the property
Sec. 4.3 relies on.

Arrays are ``[nz][nx]`` (x fastest); a batch of fields is ``[B][nz][nx]``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl


def squared_slowness(kappa) -> np.ndarray:
    """m = kappa^2 (Eq. 3.1: m(x) = 1/c(x)^2, kappa = 1/c)."""
    k = np.asarray(kappa, dtype=np.float64)
    return k * k


def neg_laplacian(u, hx: float, hz: float) -> np.ndarray:
    """-Lap_h u with zero ghost nodes: (2u_c - u_W - u_E)/hx^2 + (2u_c - u_N - u_S)/hz^2
    (the standard central-difference scheme of Sec. 3.1)."""
    u = np.asarray(u)
    p = np.zeros(u.shape[:-2] + (u.shape[-2] + 2, u.shape[-1] + 2), dtype=np.result_type(u, np.float64))
    p[..., 1:-1, 1:-1] = u
    c = p[..., 1:-1, 1:-1]
    west, east = p[..., 1:-1, :-2], p[..., 1:-1, 2:]
    north, south = p[..., :-2, 1:-1], p[..., 2:, 1:-1]
    return (2.0 * c - west - east) / hx ** 2 + (2.0 * c - north - south) / hz ** 2


def helmholtz_coefficient(kappa, gamma, omega: float) -> np.ndarray:
    """The zeroth-order term w^2 m (1 - i gamma) of Eq. 3.1 (complex128)."""
    m = squared_slowness(kappa)
    g = np.asarray(gamma, dtype=np.float64)
    return omega ** 2 * m * (1.0 - 1j * g)


def shifted_coefficient(kappa, gamma, omega: float, beta: float = 0.5,
                        alpha: float = 1.0, include_gamma: bool = False) -> np.ndarray:
    """The zeroth-order term of the shifted Laplacian, Eq. 3.12:
    w^2 m (alpha - i beta); with ``include_gamma`` the absorbing layer is kept
    as well, w^2 m (alpha - i (beta + gamma))."""
    m = squared_slowness(kappa)
    shift = beta + (np.asarray(gamma, dtype=np.float64) if include_gamma else 0.0)
    return omega ** 2 * m * (alpha - 1j * shift)


def helmholtz_apply(u, kappa, gamma, omega: float, hx: float, hz: float) -> np.ndarray:
    """H(m, w) u for one field or a batch (Eq. 3.1-3.2)."""
    u = np.asarray(u, dtype=np.complex128)
    return neg_laplacian(u, hx, hz) - helmholtz_coefficient(kappa, gamma, omega) * u


def operator_apply(u, coef, hx: float, hz: float) -> np.ndarray:
    """(-Lap_h - diag(coef)) u for a precomputed zeroth-order coefficient."""
    u = np.asarray(u, dtype=np.complex128)
    return neg_laplacian(u, hx, hz) - coef * u


def operator_matrix(coef, hx: float, hz: float) -> sp.csc_matrix:
    """Sparse matrix of -Lap_h - diag(coef) in row-major (x fastest) order:
    (1/hx^2) I_z (x) T_x + (1/hz^2) T_z (x) I_x - diag(coef), T = tridiag(-1, 2, -1)."""
    nz, nx = np.shape(coef)

    def tri(n):
        return sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])

    lap = sp.kron(sp.identity(nz), tri(nx)) / hx ** 2 + sp.kron(tri(nz), sp.identity(nx)) / hz ** 2
    return (lap - sp.diags(np.asarray(coef, dtype=np.complex128).ravel())).tocsc()


def helmholtz_matrix(kappa, gamma, omega: float, hx: float, hz: float) -> sp.csc_matrix:
    return operator_matrix(helmholtz_coefficient(kappa, gamma, omega), hx, hz)


class DirectSolver:
    """Sparse LU factorisation of H(m, w) (one factorisation, many right-hand
    sides).  The factorisation is a library primitive (SuperLU); its answer
    is *the* discrete solution that every iterative result is judged by."""

    def __init__(self, kappa, gamma, omega: float, hx: float, hz: float):
        self.shape = np.shape(kappa)
        self.matrix = helmholtz_matrix(kappa, gamma, omega, hx, hz)
        self.lu = spl.splu(self.matrix)

    def solve(self, rhs) -> np.ndarray:
        """Solve H u = rhs for ``[nz][nx]`` or ``[B][nz][nx]`` right-hand sides."""
        b = np.asarray(rhs, dtype=np.complex128)
        flat = b.reshape(-1, self.shape[0] * self.shape[1])
        out = np.stack([self.lu.solve(col) for col in flat])
        return out.reshape(b.shape)

    def solve_adjoint(self, rhs) -> np.ndarray:
        """Solve H^* x = rhs directly with the conjugate-transposed factors
        (independent of the conjugation identity of Sec. 4.3)."""
        b = np.asarray(rhs, dtype=np.complex128)
        flat = b.reshape(-1, self.shape[0] * self.shape[1])
        out = np.stack([self.lu.solve(col, trans="H") for col in flat])
        return out.reshape(b.shape)


def solve_adjoint_by_conjugation(solver: DirectSolver, rhs) -> np.ndarray:
    """H^* x = b solved as x = conj(H^{-1} conj(b)) (Sec. 4.3, Eq. 4.8)."""
    return np.conj(solver.solve(np.conj(np.asarray(rhs, dtype=np.complex128))))


def relative_residual(x, rhs, kappa, gamma, omega: float, hx: float, hz: float) -> np.ndarray:
    """||b - H x||_2 / ||b||_2 per right-hand side, evaluated in float64."""
    x = np.asarray(x, dtype=np.complex128)
    b = np.asarray(rhs, dtype=np.complex128)
    r = b - helmholtz_apply(x, kappa, gamma, omega, hx, hz)
    axes = (-2, -1)
    return np.sqrt(np.sum(np.abs(r) ** 2, axis=axes)) / np.sqrt(np.sum(np.abs(b) ** 2, axis=axes))


def relative_error(x, x_ref) -> np.ndarray:
    """||x - x_ref||_2 / ||x_ref||_2 per field."""
    x = np.asarray(x, dtype=np.complex128)
    y = np.asarray(x_ref, dtype=np.complex128)
    axes = (-2, -1)
    return np.sqrt(np.sum(np.abs(x - y) ** 2, axis=axes)) / np.sqrt(np.sum(np.abs(y) ** 2, axis=axes))
