"""FWI data misfit and adjoint-state gradient (CPU, float64).

TEST INFRASTRUCTURE: see the package header for who may import this.

Misfit, Eq. 3.5 with Sigma = I and no regulariser (alpha = 0):

    Phi(m) = sum_j sum_s || P_s^T H(m, w_j)^{-1} g_s - d_sj ||_2^2 .

Gradient (the Jacobian of Eq. 3.10, written out from the operator of Eq. 3.1;
the paper prints J with a minus sign and without the (1 - i gamma) factor,
this oracle follows the derivative of the stated operator):

    dH/dm_k = -w^2 (1 - i gamma_k) e_k e_k^T
    => du = w^2 H^{-1} diag((1 - i gamma) u) dm
    dPhi = 2 Re( r^H P_s^T du ),  r = P_s^T u - d
    => grad_k = 2 w^2 Re( conj(lambda_k) (1 - i gamma_k) u_k ),  H^* lambda = P_s r.

Because H is complex symmetric, H^* = conj(H) and mu = conj(lambda) solves
H mu = P_s conj(r): the conjugation identity of Sec. 4.3 (Eq. 4.8), so

    grad_k = 2 w^2 sum_{s,j} Re( (1 - i gamma_k) u_k mu_k ).

Receivers are flat grid indices (iz * nx + ix); P_s^T samples u at them and
P_s scatters a receiver vector back onto the grid.

Regularisers of the reconstruction (Sec. 5.1), on v = m - m_ref:
    R_diff(m) = || grad_h v ||_2^2            (diffusion)
    R_high(m) = || Lap_h v ||_2^2             (spline smoothing)
with grad_h the forward differences on the grid's interior edges and Lap_h =
-grad_h^T grad_h, the nodal Laplacian with the grid's natural boundary (the paper
does not state a boundary for these operators).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .helmholtz import DirectSolver


def sample(u, receivers) -> np.ndarray:
    """P_s^T u: the wavefield at the receiver nodes (Eq. 3.3)."""
    u = np.asarray(u)
    return u.reshape(u.shape[:-2] + (-1,))[..., np.asarray(receivers)]


def scatter(r, receivers, shape) -> np.ndarray:
    """P_s r: a receiver vector placed on the grid (zero elsewhere)."""
    r = np.asarray(r)
    rec = np.asarray(receivers)
    out = np.zeros(r.shape[:-1] + (shape[0] * shape[1],), dtype=np.result_type(r, np.complex128))
    for idx in np.ndindex(r.shape[:-1]):
        for q, k in enumerate(rec):
            out[idx + (k,)] += r[idx + (q,)]
    return out.reshape(r.shape[:-1] + tuple(shape))


def forward_data(kappa, gamma, omegas, hx, hz, sources, receivers):
    """d_sj = P^T H(m, w_j)^{-1} g_s for every frequency j and source s.

    ``sources`` are complex right-hand sides ``[ns][nz][nx]``.
    Returns complex128 ``[nf][ns][nr]`` and the wavefields ``[nf][ns][nz][nx]``."""
    d, us = [], []
    for w in omegas:
        u = DirectSolver(kappa, gamma, w, hx, hz).solve(sources)
        us.append(u)
        d.append(sample(u, receivers))
    return np.stack(d), np.stack(us)


def misfit(kappa, gamma, omegas, hx, hz, sources, receivers, d_obs) -> float:
    """Phi(m) of Eq. 3.5 (Sigma = I, alpha = 0)."""
    d, _ = forward_data(kappa, gamma, omegas, hx, hz, sources, receivers)
    return float(np.sum(np.abs(d - np.asarray(d_obs)) ** 2))


def misfit_and_gradient(kappa, gamma, omegas, hx, hz, sources, receivers, d_obs):
    """(Phi, dPhi/dm) with m = kappa^2; gradient float64 ``[nz][nx]``."""
    gamma64 = np.asarray(gamma, dtype=np.float64)
    shape = np.shape(kappa)
    phi = 0.0
    grad = np.zeros(shape)
    for j, w in enumerate(omegas):
        solver = DirectSolver(kappa, gamma, w, hx, hz)
        u = solver.solve(sources)                          # [ns][nz][nx]
        r = sample(u, receivers) - np.asarray(d_obs)[j]    # [ns][nr]
        phi += float(np.sum(np.abs(r) ** 2))
        mu = solver.solve(scatter(np.conj(r), receivers, shape))
        grad += 2.0 * w ** 2 * np.sum(np.real((1.0 - 1j * gamma64) * u * mu), axis=0)
    return phi, grad


def misfit_at_m(m, gamma, omegas, hx, hz, sources, receivers, d_obs) -> float:
    """Phi as a function of m itself (kappa = sqrt(m)), for finite differences."""
    return misfit(np.sqrt(np.asarray(m, dtype=np.float64)), gamma, omegas, hx, hz, sources,
                  receivers, d_obs)


def jacobian_apply(kappa, gamma, omegas, hx, hz, sources, receivers, dm):
    """J dm: the first-order change of the data of every frequency j and source s for a
    real change dm of m = kappa^2 (the sensitivity of Eq. 3.10, written out from the
    operator of Eq. 3.1):  du = w^2 H^{-1} ((1 - i gamma) u dm),  dd = P_s^T du.
    Returns complex128 ``[nf][ns][nr]``."""
    g64 = np.asarray(gamma, dtype=np.float64)
    dm = np.asarray(dm, dtype=np.float64)
    out = []
    for w in omegas:
        solver = DirectSolver(kappa, gamma, w, hx, hz)
        u = solver.solve(sources)
        du = solver.solve(w ** 2 * (1.0 - 1j * g64) * u * dm)
        out.append(sample(du, receivers))
    return np.stack(out)


def jacobian_adjoint(kappa, gamma, omegas, hx, hz, sources, receivers, dd):
    """J^T dd for real model perturbations: the m-vector with <J v, dd> = v . J^T dd in the
    real inner product Re(sum conj(dd) J v), i.e. Re(J^H dd).  Written out:
    Re(J^H dd)_k = sum_{j,s} w^2 Re((1 - i gamma_k) u_k mu_k),  H mu = P_s conj(dd_sj)
    (the conjugation identity of Sec. 4.3).  Returns float64 ``[nz][nx]``."""
    g64 = np.asarray(gamma, dtype=np.float64)
    shape = np.shape(kappa)
    out = np.zeros(shape)
    for j, w in enumerate(omegas):
        solver = DirectSolver(kappa, gamma, w, hx, hz)
        u = solver.solve(sources)
        mu = solver.solve(scatter(np.conj(np.asarray(dd)[j]), receivers, shape))
        out += w ** 2 * np.sum(np.real((1.0 - 1j * g64) * u * mu), axis=0)
    return out


def nodal_gradient(nx: int, nz: int, hx: float, hz: float):
    """grad_h of Sec. 5.1's R_diff as a sparse matrix on fields raveled row-major ([nz][nx]):
    the forward differences (v[i + 1] - v[i]) / hx on the (nx - 1) x nz interior x-edges,
    then (v[j + 1] - v[j]) / hz on the nx x (nz - 1) interior z-edges."""
    def diff1(n, h):
        return sp.diags([-np.ones(n - 1), np.ones(n - 1)], [0, 1], shape=(n - 1, n)) / h
    gx = sp.kron(sp.identity(nz), diff1(nx, hx))
    gz = sp.kron(diff1(nz, hz), sp.identity(nx))
    return sp.vstack([gx, gz]).tocsr()


def regularizer(m, m_ref, hx: float, hz: float, kind: int):
    """R(m) of Sec. 5.1 on v = m - m_ref (m_ref None: zero): kind 1 R_diff = ||grad_h v||^2,
    kind 2 R_high = ||Lap_h v||^2 with Lap_h = -grad_h^T grad_h, kind 0 none.  Returns
    (R, grad R, K) with K the symmetric matrix for which R = v^T K v and grad R = 2 K v
    (G^T G or (G^T G)^2, G = grad_h)."""
    m = np.asarray(m, dtype=np.float64)
    nz, nx = m.shape
    v = (m - (0.0 if m_ref is None else np.asarray(m_ref, dtype=np.float64))).ravel()
    if kind == 0:
        return 0.0, np.zeros_like(m), sp.csr_matrix((v.size, v.size))
    G = nodal_gradient(nx, nz, hx, hz)
    L = (G.T @ G).tocsr()
    K = L if kind == 1 else (L @ L).tocsr()
    Kv = K @ v
    return float(v @ Kv), (2.0 * Kv).reshape(m.shape), K


def gauss_newton_direction(kappa, gamma, omegas, hx, hz, sources, receivers, d_obs, cg_iters: int,
                           reg: float = 0.0, reg_kind: int = 0, alpha: float = 0.0, m_ref=None):
    """The Gauss-Newton step of Sec. 3.3 (Alg. 1) for the objective Phi(m) + alpha R(m)
    (R of Sec. 5.1, `regularizer`): dm approximately solving
    (J^T J + alpha K + reg I) dm = -(J^T r + alpha K (m - m_ref)),  r = d(m) - d_obs
    (J^T r = grad Phi / 2 for Eq. 3.5), by cg_iters iterations of conjugate gradients from
    dm = 0 (Hestenes and Stiefel).  Returns (dm, Phi, grad Phi)."""
    phi, grad = misfit_and_gradient(kappa, gamma, omegas, hx, hz, sources, receivers, d_obs)
    m = np.asarray(kappa, dtype=np.float64) ** 2
    _, grad_r, K = regularizer(m, m_ref, hx, hz, reg_kind)
    b = -0.5 * (grad + alpha * grad_r)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    for _ in range(cg_iters):
        Ap = jacobian_adjoint(kappa, gamma, omegas, hx, hz, sources, receivers,
                              jacobian_apply(kappa, gamma, omegas, hx, hz, sources, receivers, p)) + reg * p
        if reg_kind:
            Ap = Ap + alpha * (K @ p.ravel()).reshape(p.shape)
        step = rr / float(np.sum(p * Ap))
        x = x + step * p
        r = r - step * Ap
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, phi, grad
