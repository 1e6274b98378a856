"""Pins of the oracle's Krylov solver and FWI gradient (no GPU).

* fixed-step GMRES returns the residual minimiser over the explicit Krylov
  basis (brute force);
* V-cycle-preconditioned FGMRES reaches the direct solution;
* the adjoint-state gradient of Eq. 3.5 agrees with central finite
  differences of the misfit in a random direction (this pins the sign and the
  (1 - i gamma) factor that Eq. 3.10 prints differently);
* the misfit vanishes at the model that generated noise-free data.
"""
import math

import numpy as np

from oracle import fwi, helmholtz as H, krylov as K, multigrid as MG
from paper_2405_17696_gb300 import media


def test_gmres_fixed_is_least_squares_minimiser():
    g = np.random.default_rng(0)
    n = 30
    A = np.eye(n) * 3 + 0.4 * (g.normal(size=(n, n)) + 1j * g.normal(size=(n, n))) / math.sqrt(n)
    b = g.normal(size=n) + 1j * g.normal(size=n)
    x0 = 0.1 * (g.normal(size=n) + 1j * g.normal(size=n))
    for k in (1, 3, 6):
        x = K.gmres_fixed(lambda v: A @ v, b, x0, k)
        r0 = b - A @ x0
        basis = [r0]
        for _ in range(k - 1):
            basis.append(A @ basis[-1])
        B = np.stack(basis, axis=1)
        y, *_ = np.linalg.lstsq(A @ B, r0, rcond=None)
        assert np.linalg.norm(x - (x0 + B @ y)) < 1e-10 * np.linalg.norm(x)


def test_fgmres_vcycle_reaches_direct_solution():
    w = media.crop_workload(64, 32, freqs=(4.0,))
    om = w.omegas[0]
    b = w.rhs()[1].astype(complex)
    pc = MG.VCyclePreconditioner(w.kappa, w.gamma, om, w.h, w.h, MG.VCycleParams(levels=3))
    A = lambda u: H.helmholtz_apply(u, w.kappa, w.gamma, om, w.h, w.h)
    x, it, rel = K.fgmres(A, pc, b, restart=10, tol=1e-10, max_iter=300)
    assert rel <= 1e-10
    xd = H.DirectSolver(w.kappa, w.gamma, om, w.h, w.h).solve(b)
    assert H.relative_error(x, xd) < 1e-8


def _fwi_problem():
    nx, nz, h = 16, 12, 25.0
    c = media.layered_velocity(nx, nz, seed=4, n_layers=4)
    kappa = 1.0 / c
    gamma = media.abl_gamma(nx, nz, 4)
    sources = media.point_source_rhs(nx, nz, [(1, 3), (1, 11)], h, h)
    receivers = np.array([1 * nx + i for i in range(0, nx, 2)])
    omegas = [2 * math.pi * 3.0, 2 * math.pi * 5.0]
    c_true = c * (1 + 0.05 * np.sin(np.arange(nz)[:, None] / 3.0))
    d_obs, _ = fwi.forward_data(1.0 / c_true, gamma, omegas, h, h, sources, receivers)
    return kappa, gamma, omegas, h, sources, receivers, d_obs


def test_gradient_matches_finite_differences():
    kappa, gamma, omegas, h, sources, receivers, d_obs = _fwi_problem()
    phi, grad = fwi.misfit_and_gradient(kappa, gamma, omegas, h, h, sources, receivers, d_obs)
    m = kappa.astype(np.float64) ** 2
    dm = np.random.default_rng(9).normal(size=m.shape) * m * 1e-3
    eps = 1e-2
    fp = fwi.misfit_at_m(m + eps * dm, gamma, omegas, h, h, sources, receivers, d_obs)
    fm = fwi.misfit_at_m(m - eps * dm, gamma, omegas, h, h, sources, receivers, d_obs)
    fd = (fp - fm) / (2 * eps)
    an = float(np.sum(grad * dm))
    assert phi > 0
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_misfit_zero_at_true_model():
    kappa, gamma, omegas, h, sources, receivers, _ = _fwi_problem()
    d, _ = fwi.forward_data(kappa, gamma, omegas, h, h, sources, receivers)
    assert fwi.misfit(kappa, gamma, omegas, h, h, sources, receivers, d) < 1e-20


def test_jacobian_matches_finite_differences_of_the_data():
    """J v (sensitivity, Eq. 3.10 from the operator of Eq. 3.1) against central differences
    of the forward data d(m) in m = kappa^2."""
    kappa, gamma, omegas, h, sources, receivers, _ = _fwi_problem()
    m = kappa.astype(np.float64) ** 2
    v = np.random.default_rng(4).normal(size=m.shape) * m * 1e-3
    jv = fwi.jacobian_apply(kappa.astype(np.float64), gamma, omegas, h, h, sources, receivers, v)
    eps = 1e-2
    dp, _ = fwi.forward_data(np.sqrt(m + eps * v), gamma, omegas, h, h, sources, receivers)
    dm_, _ = fwi.forward_data(np.sqrt(m - eps * v), gamma, omegas, h, h, sources, receivers)
    fd = (dp - dm_) / (2 * eps)
    assert np.linalg.norm(jv - fd) <= 1e-6 * np.linalg.norm(fd)


def test_jacobian_adjoint_identity_and_gradient():
    """<J v, w> = v . J^T w in the real inner product Re(sum conj(w) J v), and the misfit
    gradient is 2 J^T r with r = d(m) - d_obs."""
    kappa, gamma, omegas, h, sources, receivers, d_obs = _fwi_problem()
    k64 = kappa.astype(np.float64)
    g = np.random.default_rng(6)
    v = g.normal(size=k64.shape)
    wdat = g.normal(size=np.shape(d_obs)) + 1j * g.normal(size=np.shape(d_obs))
    jv = fwi.jacobian_apply(k64, gamma, omegas, h, h, sources, receivers, v)
    jtw = fwi.jacobian_adjoint(k64, gamma, omegas, h, h, sources, receivers, wdat)
    lhs = float(np.real(np.vdot(wdat, jv)))
    rhs = float(np.sum(v * jtw))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    d, _ = fwi.forward_data(k64, gamma, omegas, h, h, sources, receivers)
    _, grad = fwi.misfit_and_gradient(k64, gamma, omegas, h, h, sources, receivers, d_obs)
    jtr = fwi.jacobian_adjoint(k64, gamma, omegas, h, h, sources, receivers, d - d_obs)
    assert np.linalg.norm(grad - 2 * jtr) <= 1e-10 * np.linalg.norm(grad)


def test_gauss_newton_cg_reaches_the_normal_equations_solution():
    """With as many CG iterations as unknowns, the Gauss-Newton direction equals the
    solution of the (regularised) normal equations built from the explicit Jacobian."""
    w = media.crop_workload(6, 4, h=50.0, freqs=(2.0,), width=1)
    k64 = w.kappa.astype(np.float64)
    gam = w.gamma.astype(np.float64)
    omegas = [2 * math.pi * 2.0, 2 * math.pi * 3.0]
    sources = media.point_source_rhs(w.nx, w.nz, [(0, 1), (0, 4)], w.h, w.h)
    receivers = np.arange(0, w.nx)
    d_obs, _ = fwi.forward_data(1.0 / (1.0 / k64 * 1.03), gam, omegas, w.h, w.h, sources, receivers)
    n = k64.size
    J = np.stack([fwi.jacobian_apply(k64, gam, omegas, w.h, w.h, sources, receivers,
                                     np.eye(n)[i].reshape(k64.shape)).ravel() for i in range(n)], axis=1)
    JtJ = np.real(J.conj().T @ J)
    reg = 1e-3 * np.trace(JtJ) / n
    dm, phi, grad = fwi.gauss_newton_direction(k64, gam, omegas, w.h, w.h, sources, receivers, d_obs, n, reg)
    ref = np.linalg.solve(JtJ + reg * np.eye(n), -0.5 * grad.ravel())
    assert np.linalg.norm(dm.ravel() - ref) <= 1e-6 * np.linalg.norm(ref)


def test_regularizers_by_their_definitions():
    """Sec. 5.1's R_diff and R_high, pinned without the oracle's sparse operators:
    an affine field v = a x + b z has R_diff = a^2 (nx - 1) nz + b^2 nx (nz - 1) (every
    edge difference is a or b); constants cost nothing; R_high equals the squared norm of
    a nodal Laplacian assembled here by loops over the neighbours (natural boundary:
    only the neighbours inside the grid); both gradients match central finite
    differences."""
    nz, nx, hx, hz = 5, 7, 2.0, 3.0
    xs, zs = np.meshgrid(np.arange(nx) * hx, np.arange(nz) * hz)
    a, b = 0.7, -1.3
    v = a * xs + b * zs
    r_diff, _, _ = fwi.regularizer(v, None, hx, hz, 1)
    assert abs(r_diff - (a * a * (nx - 1) * nz + b * b * nx * (nz - 1))) <= 1e-12 * r_diff
    c = np.full((nz, nx), 3.5)
    assert abs(fwi.regularizer(c, None, hx, hz, 1)[0]) <= 1e-12
    assert abs(fwi.regularizer(c, None, hx, hz, 2)[0]) <= 1e-12
    g = np.random.default_rng(11)
    m = g.normal(size=(nz, nx))
    m_ref = g.normal(size=(nz, nx))
    u = m - m_ref
    lap = np.zeros_like(u)
    for j in range(nz):
        for i in range(nx):
            for dj, di, h in ((0, -1, hx), (0, 1, hx), (-1, 0, hz), (1, 0, hz)):
                jj, ii = j + dj, i + di
                if 0 <= jj < nz and 0 <= ii < nx:
                    lap[j, i] += (u[jj, ii] - u[j, i]) / (h * h)
    r_high, _, _ = fwi.regularizer(m, m_ref, hx, hz, 2)
    assert abs(r_high - float(np.sum(lap * lap))) <= 1e-12 * r_high
    for kind in (1, 2):
        _, grad, _ = fwi.regularizer(m, m_ref, hx, hz, kind)
        eps = 1e-6
        for (j, i) in ((0, 0), (2, 3), (4, 6)):
            mp, mm = m.copy(), m.copy()
            mp[j, i] += eps
            mm[j, i] -= eps
            fd = (fwi.regularizer(mp, m_ref, hx, hz, kind)[0] - fwi.regularizer(mm, m_ref, hx, hz, kind)[0]) / (2 * eps)
            assert abs(fd - grad[j, i]) <= 1e-6 * max(1.0, abs(fd))


def test_regularised_gauss_newton_reaches_its_normal_equations():
    """With a regulariser of Sec. 5.1 and three times as many CG steps as unknowns, the Gauss-Newton
    direction solves (J^T J + alpha K) dm = -(grad Phi + alpha grad R) / 2 built from the
    explicit Jacobian, for R_diff and R_high."""
    w = media.crop_workload(6, 4, h=50.0, freqs=(2.0,), width=1)
    k64 = w.kappa.astype(np.float64)
    gam = w.gamma.astype(np.float64)
    omegas = [2 * math.pi * 2.0, 2 * math.pi * 3.0]
    sources = media.point_source_rhs(w.nx, w.nz, [(0, 1), (0, 4)], w.h, w.h)
    receivers = np.arange(0, w.nx)
    d_obs, _ = fwi.forward_data(1.0 / (1.0 / k64 * 1.03), gam, omegas, w.h, w.h, sources, receivers)
    n = k64.size
    J = np.stack([fwi.jacobian_apply(k64, gam, omegas, w.h, w.h, sources, receivers,
                                     np.eye(n)[i].reshape(k64.shape)).ravel() for i in range(n)], axis=1)
    JtJ = np.real(J.conj().T @ J)
    m_ref = (k64 ** 2) * 1.1
    for kind in (1, 2):
        _, grad_r, K = fwi.regularizer(k64 ** 2, m_ref, w.h, w.h, kind)
        K = K.toarray()
        alpha = 1e-2 * np.trace(JtJ) / np.trace(K)
        # (more CG steps than unknowns: the regularised system's condition number is ~1e4)
        dm, phi, grad = fwi.gauss_newton_direction(k64, gam, omegas, w.h, w.h, sources, receivers, d_obs, 3 * n,
                                                   reg_kind=kind, alpha=alpha, m_ref=m_ref)
        ref = np.linalg.solve(JtJ + alpha * K, -0.5 * (grad + alpha * grad_r).ravel())
        assert np.linalg.norm(dm.ravel() - ref) <= 1e-6 * np.linalg.norm(ref)
