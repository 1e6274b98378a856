"""Pins of the oracle's discrete Helmholtz operator and direct solve against
facts fixed by the mathematics (no GPU).

* discrete sine modes are eigenvectors of the zero-ghost 5-point Laplacian
  with eigenvalues in closed form (anisotropic hx != hz, nx != nz);
* a manufactured smooth solution is recovered at second order;
* the free-space Green's function (the outgoing branch for the paper's sign
  of the damping term, Eq. 3.1) is matched at second order;
* reciprocity u_s(x_r) = u_r(x_s) from complex symmetry (Sec. 4.3);
* the conjugation identity for the adjoint system (Eq. 4.8).
"""
import math

import numpy as np
import pytest

from oracle import green, helmholtz as H
from paper_2405_17696_gb300 import media


def _sine_mode(nx, nz, p, q):
    ix = np.arange(nx)[None, :]
    iz = np.arange(nz)[:, None]
    return np.sin(math.pi * p * (ix + 1) / (nx + 1)) * np.sin(math.pi * q * (iz + 1) / (nz + 1))


@pytest.mark.parametrize("p,q", [(1, 1), (3, 2), (12, 7), (17, 9)])
def test_sine_modes_are_eigenvectors(p, q):
    nx, nz, hx, hz = 19, 11, 7.0, 3.0
    u = _sine_mode(nx, nz, p, q)
    lam = (4 / hx ** 2) * math.sin(math.pi * p / (2 * (nx + 1))) ** 2 \
        + (4 / hz ** 2) * math.sin(math.pi * q / (2 * (nz + 1))) ** 2
    c, gam, om = 1800.0, 0.3, 2 * math.pi * 5.0
    kappa = np.full((nz, nx), 1.0 / c)
    gamma = np.full((nz, nx), gam)
    mu = lam - om ** 2 / c ** 2 * (1 - 1j * gam)
    out = H.helmholtz_apply(u, kappa, gamma, om, hx, hz)
    assert np.allclose(out, mu * u, rtol=0, atol=1e-12 * abs(mu))
    # the sparse-matrix form gives the same product
    A = H.helmholtz_matrix(kappa, gamma, om, hx, hz)
    assert np.allclose((A @ u.ravel().astype(complex)).reshape(nz, nx), mu * u, atol=1e-12 * abs(mu))


def test_matrix_is_complex_symmetric():
    w = media.crop_workload(24, 16)
    A = H.helmholtz_matrix(w.kappa, w.gamma, w.omegas[0], 11.0, 7.0)
    assert abs(A - A.T).max() == 0.0
    assert abs(A - A.conj().T).max() > 0.0   # symmetric, not Hermitian


def _mms_error(nx, nz, Lx, Lz, om):
    hx, hz = Lx / (nx + 1), Lz / (nz + 1)
    x = (np.arange(nx) + 1) * hx
    z = (np.arange(nz) + 1) * hz
    X = (x / Lx)[None, :]
    Z = (z / Lz)[:, None]
    p, q, th = 2, 1, 3.0
    s, sp_, spp = np.sin(p * math.pi * X), p * math.pi * np.cos(p * math.pi * X), -(p * math.pi) ** 2 * np.sin(p * math.pi * X)
    S, Spp = np.sin(q * math.pi * Z), -(q * math.pi) ** 2 * np.sin(q * math.pi * Z)
    E = np.exp(1j * th * X)
    u = s * S * E
    d2X = S * E * (spp + 2j * th * sp_ - th ** 2 * s)
    d2Z = s * E * Spp
    lap = d2X / Lx ** 2 + d2Z / Lz ** 2
    m = (1.0 / 2000.0 ** 2) * (1 + 0.3 * X * Z)
    gam = 0.2 * X ** 2 + 0.0 * Z
    g = -lap - om ** 2 * m * (1 - 1j * gam) * u
    uh = H.DirectSolver(np.sqrt(m), gam, om, hx, hz).solve(g)
    return float(np.linalg.norm(uh - u) / np.linalg.norm(u))


def test_manufactured_solution_second_order():
    Lx, Lz, om = 1600.0, 1200.0, 2 * math.pi * 1.5
    e1 = _mms_error(15, 11, Lx, Lz, om)
    e2 = _mms_error(31, 23, Lx, Lz, om)
    e3 = _mms_error(63, 47, Lx, Lz, om)
    assert e1 < 0.2
    assert 3.5 < e1 / e2 < 4.5
    assert 3.7 < e2 / e3 < 4.3


def _green_error(ppw, conj=True):
    c, f = 1500.0, 7.5
    lam = c / f
    h = lam / ppw
    L, n = 4 * ppw, 6 * ppw + 8 * ppw
    kappa = np.full((n, n), 1.0 / c)
    gamma = media.abl_gamma(n, n, L, 1.0, top=True)
    om = 2 * math.pi * f
    b = media.point_source_rhs(n, n, [(n // 2, n // 2)], h, h)[0]
    u = H.DirectSolver(kappa, gamma, om, h, h).solve(b)
    iz, ix = np.mgrid[0:n, 0:n]
    r = h * np.hypot(iz - n // 2, ix - n // 2)
    mask = (r >= lam) & (r <= 2 * lam)
    g = green.green_h1(om / c, r[mask])
    v = np.conj(u[mask]) if conj else u[mask]
    return float(np.linalg.norm(v - g) / np.linalg.norm(g))


def test_green_function_outgoing_branch():
    e10 = _green_error(10)
    e20 = _green_error(20)
    assert e20 < 0.05
    assert e10 / e20 > 3.5
    # the other branch (no conjugation) is far off: the sign of Eq. 3.1 matters
    assert _green_error(10, conj=False) > 0.5


def test_reciprocity():
    w = media.crop_workload(48, 32, freqs=(6.0,))
    s = H.DirectSolver(w.kappa, w.gamma, w.omegas[0], w.h, w.h)
    a, b = (2, 5), (20, 37)
    ga = media.point_source_rhs(w.nx, w.nz, [a], w.h, w.h)[0]
    gb = media.point_source_rhs(w.nx, w.nz, [b], w.h, w.h)[0]
    ua, ub = s.solve(ga), s.solve(gb)
    assert abs(ua[b] - ub[a]) <= 1e-12 * abs(ua[b])


def test_direct_solve_residual():
    w = media.crop_workload(64, 32, freqs=(3.0, 6.0))
    rhs = w.rhs()
    for j, om in enumerate(w.omegas):
        s = H.DirectSolver(w.kappa, w.gamma, om, w.h, w.h)
        b = rhs[j * len(w.positions):(j + 1) * len(w.positions)]
        x = s.solve(b)
        assert np.all(H.relative_residual(x, b, w.kappa, w.gamma, om, w.h, w.h) < 1e-12)


def test_adjoint_by_conjugation_matches_direct_adjoint():
    w = media.crop_workload(40, 24)
    s = H.DirectSolver(w.kappa, w.gamma, w.omegas[0], w.h, w.h)
    b = media.complex_normal((2, w.nz, w.nx), seed=11)
    x1 = H.solve_adjoint_by_conjugation(s, b)
    x2 = s.solve_adjoint(b)
    assert np.max(H.relative_error(x1, x2)) < 1e-12
    # and the adjoint really differs from the forward solve (gamma != 0)
    assert np.max(H.relative_error(s.solve(b), x2)) > 1e-3
