"""Shifted-Laplacian multigrid V-cycle (CPU, complex128).

TEST INFRASTRUCTURE: see the package header for who may import this.

Sec. 3.4 preconditions the Krylov method with a multigrid cycle on the
shifted Laplacian P = -Lap_h - w^2 m (alpha - i beta) (Eq. 3.12, alpha = 1,
beta = 0.5); the network preconditioner M_VU of Eq. 3.14 runs one such cycle
(levels = 3) on r starting from the network's output e_0.  The paper does not
give the cycle's parts; this oracle fixes them as follows (the same reading
the CUDA path implements):

* level 0 is P itself (5-point stencil, zero ghost nodes).  By default the
  absorbing layer is kept inside the shift, w^2 m (1 - i (beta + gamma));
  ``include_gamma=False`` gives the literal Eq. 3.12;
* coarse node (J, I) of level l+1 sits on node (2J+1, 2I+1) of level l;
* residual restriction R_l: full weighting (1/16)[1 2 1; 2 4 2; 1 2 1]
  centred on that node, zero outside the grid;
* prolongation: bilinear interpolation 4 R_l^T (zero ghost values);
* coarse operators are Galerkin products P_{l+1} = R_l P_l (4 R_l^T) (9-point
  stencils).  With an even number of nodes per side a rediscretised coarse
  grid cannot keep both Dirichlet edges in place; the Galerkin product
  inherits the fine grid's boundary exactly;
* smoother: damped Jacobi u <- u + w D_l^-1 (f - P_l u), D_l = diag(P_l);
* coarsest level: a fixed number of plain GMRES steps on P_L from the given
  initial guess (or a fixed number of Jacobi sweeps).

The products are formed with sparse matrices (a library primitive).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import helmholtz as hz_
from .krylov import gmres_fixed

_W1 = np.array([1.0, 2.0, 1.0])


@dataclass
class VCycleParams:
    levels: int = 3
    pre: int = 2
    post: int = 2
    jacobi_w: float = 0.8
    beta: float = 0.5
    include_gamma: bool = True
    coarse_kind: str = "gmres"      # "gmres" or "jacobi"
    coarse_iters: int = 10


def _pad1(a):
    p = np.zeros(a.shape[:-2] + (a.shape[-2] + 2, a.shape[-1] + 2), dtype=a.dtype)
    p[..., 1:-1, 1:-1] = a
    return p


def restrict_full_weighting(r) -> np.ndarray:
    """r_c(J, I) = sum_{a,b in {-1,0,1}} w_a w_b / 16 r(2J+1+a, 2I+1+b), w = (1,2,1),
    with zero values outside the fine grid."""
    r = np.asarray(r)
    nz, nx = r.shape[-2:]
    p = _pad1(r)  # p[zz+1, xx+1] = r[zz, xx]
    out = np.zeros(r.shape[:-2] + (nz // 2, nx // 2), dtype=np.result_type(r, np.float64))
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            wt = _W1[a + 1] * _W1[b + 1] / 16.0
            out += wt * p[..., 2 + a: 2 + a + nz: 2, 2 + b: 2 + b + nx: 2]
    return out


def prolong_bilinear(e_c, fine_shape) -> np.ndarray:
    """Bilinear interpolation from the coarse grid (node (J, I) on fine node
    (2J+1, 2I+1)) to the fine grid with zero coarse ghost values."""
    e_c = np.asarray(e_c)
    nz, nx = fine_shape

    def along_x(c):
        n = c.shape[-1]
        f = np.zeros(c.shape[:-1] + (2 * n,), dtype=c.dtype)
        f[..., 1::2] = c
        left = np.concatenate([np.zeros(c.shape[:-1] + (1,), dtype=c.dtype), c[..., :-1]], axis=-1)
        f[..., 0::2] = 0.5 * (left + c)
        return f

    t = along_x(e_c)
    t = np.swapaxes(along_x(np.swapaxes(t, -1, -2)), -1, -2)
    assert t.shape[-2:] == (nz, nx)
    return t


def restriction_matrix(nz: int, nx: int) -> sp.csr_matrix:
    """R as a sparse (nz/2 nx/2) x (nz nx) matrix, row-major ordering."""
    def r1(n):
        rows, cols, vals = [], [], []
        for i_c in range(n // 2):
            for a in (-1, 0, 1):
                i = 2 * i_c + 1 + a
                if 0 <= i < n:
                    rows.append(i_c)
                    cols.append(i)
                    vals.append(_W1[a + 1] / 4.0)
        return sp.csr_matrix((vals, (rows, cols)), shape=(n // 2, n))
    return sp.kron(r1(nz), r1(nx)).tocsr()


def fine_sl_matrix(kappa, gamma, omega: float, hx: float, hz: float,
                   p: "VCycleParams") -> sp.csr_matrix:
    coef = hz_.shifted_coefficient(kappa, gamma, omega, beta=p.beta, include_gamma=p.include_gamma)
    return hz_.operator_matrix(coef, hx, hz).tocsr()


@dataclass
class Level:
    nz: int
    nx: int
    op: sp.csr_matrix      # P_l
    diag: np.ndarray       # diag(P_l)


def build_hierarchy(kappa, gamma, omega: float, hx: float, hz: float, p: VCycleParams):
    nz, nx = np.shape(kappa)
    op = fine_sl_matrix(kappa, gamma, omega, hx, hz, p)
    out = [Level(nz, nx, op, op.diagonal())]
    for _ in range(1, p.levels):
        L = out[-1]
        if L.nx % 2 or L.nz % 2:
            raise ValueError("grid not divisible by 2^(levels-1)")
        R = restriction_matrix(L.nz, L.nx)
        op = (R @ L.op @ (4.0 * R.T)).tocsr()
        out.append(Level(L.nz // 2, L.nx // 2, op, op.diagonal()))
    return out


def apply_level(u, level: Level) -> np.ndarray:
    u = np.asarray(u, dtype=np.complex128)
    return (level.op @ u.ravel()).reshape(u.shape)


def jacobi_sweep(u, f, level: Level, w: float) -> np.ndarray:
    """u + w D^-1 (f - P u)."""
    d = level.diag.reshape(level.nz, level.nx)
    return u + w * (f - apply_level(u, level)) / d


def coarsest_solve(f, u0, level: Level, p: VCycleParams) -> np.ndarray:
    if p.coarse_kind == "gmres":
        return gmres_fixed(lambda v: apply_level(v, level), f, u0, p.coarse_iters)
    u = u0
    for _ in range(p.coarse_iters):
        u = jacobi_sweep(u, f, level, p.jacobi_w)
    return u


def vcycle(f, u0, hierarchy, p: VCycleParams, lev: int = 0) -> np.ndarray:
    """One V-cycle for P_lev u = f from the initial guess u0 (one field)."""
    f = np.asarray(f, dtype=np.complex128)
    u = np.asarray(u0, dtype=np.complex128).copy()
    L = hierarchy[lev]
    if lev == len(hierarchy) - 1:
        return coarsest_solve(f, u, L, p)
    for _ in range(p.pre):
        u = jacobi_sweep(u, f, L, p.jacobi_w)
    r_c = restrict_full_weighting(f - apply_level(u, L))
    e_c = vcycle(r_c, np.zeros_like(r_c), hierarchy, p, lev + 1)
    u = u + prolong_bilinear(e_c, (L.nz, L.nx))
    for _ in range(p.post):
        u = jacobi_sweep(u, f, L, p.jacobi_w)
    return u


class VCyclePreconditioner:
    """M(r) = V-cycle(P, r, u0): the plain preconditioner of Sec. 3.4 (u0 = 0)
    and the multigrid part of M_VU, Eq. 3.14 (u0 = the network's output)."""

    def __init__(self, kappa, gamma, omega: float, hx: float, hz: float, params: VCycleParams):
        self.params = params
        self.omega = omega
        self.hier = build_hierarchy(kappa, gamma, omega, hx, hz, params)

    def __call__(self, r, u0=None) -> np.ndarray:
        r = np.asarray(r, dtype=np.complex128)
        u0 = np.zeros_like(r) if u0 is None else u0
        return vcycle(r, u0, self.hier, self.params)
