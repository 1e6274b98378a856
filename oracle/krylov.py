"""Krylov solvers (CPU, complex128).

TEST INFRASTRUCTURE: see the package header for who may import this.

The paper preconditions "GMRES" with a shifted-Laplacian V-cycle or with the
encoder-solver network (Sec. 3.4, Eq. 3.14) and uses a fixed number of
V-cycle-preconditioned GMRES steps to make training data (Eq. 4.3, Alg. 2).
Because the network preconditioner is nonlinear, the outer method is the
flexible variant (right preconditioning, the preconditioned directions z_j
are kept): Saad, "A flexible inner-outer preconditioned GMRES algorithm",
SIAM J. Sci. Comput. 14 (1993).  Orthogonalisation here is modified
Gram-Schmidt; in exact arithmetic it spans the same spaces as any other
Gram-Schmidt variant, so the minimiser returned is the same.
"""
from __future__ import annotations

import numpy as np


def _vdot(a, b) -> complex:
    """<a, b> = sum conj(a) b."""
    return complex(np.vdot(a.ravel(), b.ravel()))


def _norm(a) -> float:
    return float(np.sqrt(np.sum(np.abs(a) ** 2)))


def fgmres_cycle(apply_a, precond, b, x0, k: int, tol_abs: float = 0.0):
    """One cycle of at most ``k`` flexible GMRES steps from ``x0``.

    Returns (x, steps, residual_estimates) where x = x0 + Z y and y solves
    min_y || beta e_1 - Hbar y ||_2 over the steps taken.  The cycle stops
    early once the least-squares residual drops to ``tol_abs`` or on an exact
    (happy) breakdown h_{j+1,j} = 0.
    """
    b = np.asarray(b, dtype=np.complex128)
    x0 = np.asarray(x0, dtype=np.complex128)
    r = b - apply_a(x0)
    beta = _norm(r)
    if beta == 0.0:
        return x0.copy(), 0, [0.0]
    V = [r / beta]
    Z = []
    Hbar = np.zeros((k + 1, k), dtype=np.complex128)
    estimates = [beta]
    steps = 0
    for j in range(k):
        z = np.asarray(precond(V[j]), dtype=np.complex128)
        Z.append(z)
        w = np.asarray(apply_a(z), dtype=np.complex128)
        for i in range(j + 1):
            Hbar[i, j] = _vdot(V[i], w)
            w = w - Hbar[i, j] * V[i]
        Hbar[j + 1, j] = _norm(w)
        steps = j + 1
        e1 = np.zeros(j + 2, dtype=np.complex128)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(Hbar[: j + 2, : j + 1], e1, rcond=None)
        est = _norm(e1 - Hbar[: j + 2, : j + 1] @ y)
        estimates.append(est)
        if Hbar[j + 1, j] == 0.0 or est <= tol_abs:
            break
        V.append(w / Hbar[j + 1, j])
    e1 = np.zeros(steps + 1, dtype=np.complex128)
    e1[0] = beta
    y, *_ = np.linalg.lstsq(Hbar[: steps + 1, :steps], e1, rcond=None)
    x = x0 + sum(y[i] * Z[i] for i in range(steps))
    return x, steps, estimates


def fgmres(apply_a, precond, b, x0=None, restart: int = 10, tol: float = 1e-6,
           max_iter: int = 300):
    """Restarted flexible GMRES until ||b - A x|| <= tol ||b|| (true residual,
    recomputed at every restart) or ``max_iter`` total steps.

    Returns (x, total_steps, relative_true_residual)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.complex128).copy()
    bnorm = _norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    total = 0
    rel = _norm(b - apply_a(x)) / bnorm
    while rel > tol and total < max_iter:
        k = min(restart, max_iter - total)
        x, steps, _ = fgmres_cycle(apply_a, precond, b, x, k, tol_abs=tol * bnorm)
        total += steps
        rel = _norm(b - apply_a(x)) / bnorm
        if steps == 0:
            break
    return x, total, rel


def gmres_fixed(apply_a, b, x0, k: int, precond=None):
    """Exactly ``k`` (flexibly) preconditioned GMRES steps from ``x0`` without
    restart (the 'iter' steps of Eq. 4.3 and Alg. 2); fewer only on an exact
    breakdown.  With ``precond`` None this is plain GMRES."""
    pc = precond if precond is not None else (lambda v: v)
    x, _, _ = fgmres_cycle(apply_a, pc, b, x0, k, tol_abs=0.0)
    return x
