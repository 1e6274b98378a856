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
"""
from __future__ import annotations

import numpy as np

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


def gauss_newton_direction(kappa, gamma, omegas, hx, hz, sources, receivers, d_obs, cg_iters: int,
                           reg: float = 0.0):
    """The Gauss-Newton step of Sec. 3.3 (Alg. 1): dm approximately solving
    (J^T J + reg I) dm = -J^T r,  r = d(m) - d_obs  (J^T r = grad Phi / 2 for Eq. 3.5),
    by cg_iters iterations of conjugate gradients from dm = 0 (Hestenes and Stiefel).
    Returns (dm, Phi, grad Phi)."""
    phi, grad = misfit_and_gradient(kappa, gamma, omegas, hx, hz, sources, receivers, d_obs)
    b = -0.5 * grad
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    for _ in range(cg_iters):
        Ap = jacobian_adjoint(kappa, gamma, omegas, hx, hz, sources, receivers,
                              jacobian_apply(kappa, gamma, omegas, hx, hz, sources, receivers, p)) + reg * p
        alpha = rr / float(np.sum(p * Ap))
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, phi, grad
