"""Pins of the oracle's shifted-Laplacian V-cycle parts (Sec. 3.4, Eq. 3.12)
against textbook multigrid facts (no GPU).

* one damped-Jacobi sweep multiplies a discrete sine mode of a constant
  shifted Laplacian by its Fourier symbol 1 - w mu / d;
* full weighting and bilinear interpolation reproduce bilinear functions away
  from the edges, and interpolation is 4 x the transpose of full weighting;
* the Galerkin coarse operator of a constant shifted Laplacian has the
  closed-form 9-point interior stencil;
* the V-cycle, used as a stationary solver on the Poisson case (w = 0), contracts
  the error by a grid-independent factor well below one;
* the coarsest GMRES solve equals the least-squares minimiser over the
  explicit Krylov basis.
"""
import math

import numpy as np
import pytest

from oracle import helmholtz as H, krylov as K, multigrid as MG
from paper_2405_17696_gb300 import media


def test_jacobi_fourier_symbol():
    nx, nz, hx, hz = 16, 8, 20.0, 30.0
    c, om, w = 1500.0, 2 * math.pi * 4.0, 0.8
    kappa = np.full((nz, nx), 1 / c)
    p = MG.VCycleParams(levels=1, jacobi_w=w, beta=0.5, include_gamma=False)
    lev = MG.build_hierarchy(kappa, np.full((nz, nx), 0.7), om, hx, hz, p)[0]
    for (pp, qq) in [(1, 1), (5, 3), (15, 7)]:
        ix = np.arange(nx)[None, :]
        iz = np.arange(nz)[:, None]
        e = np.sin(math.pi * pp * (ix + 1) / (nx + 1)) * np.sin(math.pi * qq * (iz + 1) / (nz + 1))
        lam = 4 / hx ** 2 * math.sin(math.pi * pp / (2 * (nx + 1))) ** 2 \
            + 4 / hz ** 2 * math.sin(math.pi * qq / (2 * (nz + 1))) ** 2
        shift = om ** 2 / c ** 2 * (1 - 0.5j)
        mu, d = lam - shift, 2 / hx ** 2 + 2 / hz ** 2 - shift
        out = MG.jacobi_sweep(e.astype(complex), np.zeros_like(e, dtype=complex), lev, w)
        assert np.allclose(out, (1 - w * mu / d) * e, atol=1e-13)


def test_galerkin_coarse_stencil_closed_form():
    # Interior Galerkin stencil of -Lap_h - s I under full weighting and
    # bilinear interpolation (H = 2h): the textbook 9-point Laplacian
    # (1/H^2)[-1/4 -1/2 -1/4; -1/2 3 -1/2; -1/4 -1/2 -1/4] minus s times
    # the tensor-product mass stencil [1/8 3/4 1/8] (x) [1/8 3/4 1/8].
    n, h, c, om = 32, 10.0, 1500.0, 2 * math.pi * 3.0
    kappa = np.full((n, n), 1 / c)
    p = MG.VCycleParams(levels=2, beta=0.5, include_gamma=False)
    hier = MG.build_hierarchy(kappa, np.zeros((n, n)), om, h, h, p)
    s = om ** 2 / c ** 2 * (1 - 0.5j)
    H2 = (2 * h) ** 2
    lap = np.array([[-0.25, -0.5, -0.25], [-0.5, 3.0, -0.5], [-0.25, -0.5, -0.25]]) / H2
    m1 = np.array([0.125, 0.75, 0.125])
    expect = lap - s * np.outer(m1, m1)
    nc = n // 2
    A = hier[1].op.toarray()
    row = 7 * nc + 6
    got = np.array([[A[row, (7 + a) * nc + 6 + b] for b in (-1, 0, 1)] for a in (-1, 0, 1)])
    assert np.allclose(got, expect, rtol=1e-12, atol=1e-18)
    # and every coarse operator stays a 9-point stencil
    for lev in hier[1:]:
        assert lev.op.getnnz(axis=1).max() <= 9


def _bilinear(X, Z):
    return 0.7 + 0.3 * X - 0.2 * Z + 0.05 * X * Z


def test_transfers_exact_on_bilinear_data():
    nx, nz = 16, 12
    Xf, Zf = np.meshgrid(np.arange(nx, dtype=float), np.arange(nz, dtype=float))
    f = _bilinear(Xf, Zf)
    rc = MG.restrict_full_weighting(f)
    Xc, Zc = np.meshgrid(2 * np.arange(nx // 2) + 1.0, 2 * np.arange(nz // 2) + 1.0)
    exact = _bilinear(Xc, Zc)
    # interior coarse nodes (their 3x3 stencil stays inside the fine grid)
    assert np.allclose(rc[:-1, :-1], exact[:-1, :-1], atol=1e-13)
    # interpolation of coarse samples of a bilinear function
    fine = MG.prolong_bilinear(exact, (nz, nx))
    assert np.allclose(fine[1:, 1:], f[1:, 1:], atol=1e-13)


def test_prolongation_is_four_times_restriction_transpose():
    g = np.random.default_rng(5)
    nx, nz = 12, 10
    fine = g.normal(size=(nz, nx)) + 1j * g.normal(size=(nz, nx))
    coarse = g.normal(size=(nz // 2, nx // 2)) + 1j * g.normal(size=(nz // 2, nx // 2))
    lhs = 4 * np.vdot(coarse, MG.restrict_full_weighting(fine))
    rhs = np.vdot(MG.prolong_bilinear(coarse, (nz, nx)), fine)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


@pytest.mark.parametrize("n", [32, 64])
def test_vcycle_contracts_on_poisson(n):
    # w = 0: P is the Dirichlet Laplacian; V(2,2) with damped Jacobi, full
    # weighting, bilinear interpolation and Galerkin coarse grids contracts
    # the error by a grid-independent factor near the textbook 0.1.
    kappa = np.full((n, n), 1 / 1500.0)
    p = MG.VCycleParams(levels=4, pre=2, post=2, jacobi_w=0.8, coarse_kind="gmres", coarse_iters=16)
    pc = MG.VCyclePreconditioner(kappa, np.zeros((n, n)), 0.0, 10.0, 10.0, p)
    f = np.zeros((n, n), dtype=complex)
    u = np.random.default_rng(1).normal(size=(n, n)).astype(complex)
    norms = []
    for _ in range(6):
        u = pc(f, u)
        norms.append(np.linalg.norm(u))
    rate = (norms[-1] / norms[1]) ** (1 / 4)
    assert rate < 0.2


def test_coarsest_gmres_is_krylov_minimiser():
    w = media.crop_workload(16, 8)
    p = MG.VCycleParams(levels=1, coarse_iters=5)
    lev = MG.build_hierarchy(w.kappa, w.gamma, w.omegas[0], w.h, w.h, p)[0]
    f = media.complex_normal((w.nz, w.nx), seed=3).astype(complex)
    x = MG.coarsest_solve(f, np.zeros_like(f), lev, p)
    A = lambda v: MG.apply_level(v, lev)
    basis = [f]
    for _ in range(4):
        basis.append(A(basis[-1]))
    Kmat = np.stack([A(b).ravel() for b in basis], axis=1)
    y, *_ = np.linalg.lstsq(Kmat, f.ravel(), rcond=None)
    x_ref = sum(y[i] * basis[i] for i in range(5))
    assert np.linalg.norm(x - x_ref) < 1e-8 * np.linalg.norm(x_ref)
