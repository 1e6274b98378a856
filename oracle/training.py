"""Training data and loss of the encoder-solver network (CPU, float64).

TEST INFRASTRUCTURE: see the package header for who may import this.

* Eq. 4.3: for a draw x, b = H x, x~ = GMRES(H, M = V-cycle, b, x0 = 0) after
  `iters` steps, r = b - H x~, e = x - x~ (the flexible variant, since the
  V-cycle with a GMRES coarsest solve is not a linear operator).
* Alg. 2 data step: e_net = network(r); e~ = GMRES(H, V-cycle, r, x0 = e_net)
  after one step; new pair (r - H e~, e - e~) in the residual-correction
  reading, or (H e~, e~) as printed.
* Eq. 4.2: loss = (1/m) sum_i ||e_net(r_i) - e_i||^2, e_net = h^2 rms(r) out.
* Eq. 3.14: M_VU(r) = a e_0 + V(r - a H e_0) (the V-cycle corrects the residual the
  network leaves; a = 1 unless the network's step raises it, then a minimises it),
  without a, or a V-cycle on P started from u_0 = e_0.
"""
from __future__ import annotations

import numpy as np

from . import cnn
from . import helmholtz as H
from . import multigrid as MG
from .krylov import fgmres_cycle


def make_samples(kappa, gamma, omega, h, x, iters, params=None, hz=None):
    """Eq. 4.3 pairs; h is hx, and hz (default h) the vertical spacing."""
    hz = h if hz is None else hz
    p = params if params is not None else MG.VCycleParams()
    pc = MG.VCyclePreconditioner(kappa, gamma, omega, h, hz, p)
    A = lambda u: H.helmholtz_apply(u, kappa, gamma, omega, h, hz)
    rs, es = [], []
    for xi, k in zip(np.asarray(x, dtype=np.complex128), iters):
        b = A(xi)
        xt, _, _ = fgmres_cycle(A, pc, b, np.zeros_like(b), int(k), tol_abs=0.0)
        rs.append(b - A(xt))
        es.append(xi - xt)
    return np.stack(rs), np.stack(es)


def mvu_compose(e0, r, A, pc, composition: str = "residual"):
    """M_VU of Eq. 3.14 for one residual, given the network's estimate e0.

    ``guarded``: a e0 + V(r - a H e0, 0) with a = 1 while ||r - H e0|| <= ||r||, else
    the complex a = <H e0, r> / <H e0, H e0> that minimises ||r - a H e0||.  ``residual``: e0 + V(r - H e0, 0):
    exact when e0 = H^-1 r, the plain V-cycle when e0 = 0.  ``initial_guess``: V(r, u_0 = e0)
    on the shifted operator."""
    if composition == "guarded":
        t = A(e0)
        tt = np.vdot(t, t).real
        tr = np.vdot(t, r)
        if tt <= 2.0 * tr.real:          # the network's step does not raise the residual
            a = 1.0
        else:
            a = tr / tt
        return a * e0 + pc(r - a * t)
    if composition == "residual":
        return e0 + pc(r - A(e0))
    if composition == "initial_guess":
        return pc(r, e0)
    raise ValueError(composition)


def network_error(P, specs, kappa, gamma, omega, h, r, quantize=None, hz=None):
    """e_net = hx hz rms(r) (out_re + i out_im) for residuals r [B][nz][nx]; on an
    anisotropic grid (hz given) the network sees the geometric-mean spacing sqrt(hx hz)
    in its input w h kappa, and the output scale is hx hz."""
    hz = h if hz is None else hz
    hg = float(np.sqrt(h * hz))
    enc = cnn.encoder_input(kappa, gamma, omega, hg)
    x, rms = cnn.solver_input(r, gamma)
    if quantize is not None:
        enc, x = quantize(enc), quantize(x)
    out, tape = cnn.network_forward(P, specs, enc, x, quantize=quantize)
    return cnn.solver_output_to_error(out, rms, hg), out, tape, rms


def refine_from_estimate(kappa, gamma, omega, h, r, e, e_net, literal=False, params=None, hz=None):
    """The data step of Alg. 2 (Sec. 4.2) given the network's error estimates.

    For each pair (r, e) with H e = r: e~ = x after one V-cycle-preconditioned
    (F)GMRES step on H x = r started from x0 = e_net, and the new pair is
    (r - H e~, e - e~) in the residual-correction reading (the error that is still
    left after the step, with its residual), or (H e~, e~) as Alg. 2 prints it."""
    hz = h if hz is None else hz
    p = params if params is not None else MG.VCycleParams()
    pc = MG.VCyclePreconditioner(kappa, gamma, omega, h, hz, p)
    A = lambda u: H.helmholtz_apply(u, kappa, gamma, omega, h, hz)
    r2, e2 = [], []
    for ri, ei, x0 in zip(np.asarray(r, dtype=np.complex128), np.asarray(e, dtype=np.complex128),
                          np.asarray(e_net, dtype=np.complex128)):
        et, _, _ = fgmres_cycle(A, pc, ri, x0, 1, tol_abs=0.0)
        if literal:
            r2.append(A(et))
            e2.append(et)
        else:
            r2.append(ri - A(et))
            e2.append(ei - et)
    return np.stack(r2), np.stack(e2)


def refine_samples(P, specs, kappa, gamma, omega, h, r, e, literal=False, params=None, quantize=None, hz=None):
    """Alg. 2 data step with the network of parameters P as the estimator
    (network output alone, no V-cycle)."""
    e_net, _, _, _ = network_error(P, specs, kappa, gamma, omega, h, r, quantize, hz=hz)
    return refine_from_estimate(kappa, gamma, omega, h, r, e, e_net, literal, params, hz=hz)


def loss_and_grad(P, specs, kappa, gamma, omega, h, r, e, quantize=None, relative=False, grad_quantize=None,
                  hz=None):
    """(loss, {name: (dw, db)}) of Eq. 4.2 for one batch of one medium/frequency;
    relative=True weighs sample i by 1 / ||e_i||^2.  quantize rounds the inputs and
    stored activations, grad_quantize the gradient operand of every convolution
    (both bf16_round for a BF16 network)."""
    e_net, out, tape, rms = network_error(P, specs, kappa, gamma, omega, h, r, quantize, hz=hz)
    hz = h if hz is None else hz
    m = r.shape[0]
    e = np.asarray(e, dtype=np.complex128)
    d = e_net - e
    wt = 1.0 / np.sum(np.abs(e) ** 2, axis=(1, 2)) if relative else np.ones(m)
    loss = float(np.sum(wt * np.sum(np.abs(d) ** 2, axis=(1, 2))) / m)
    s = (h * hz) * rms[:, None, None] * wt[:, None, None]
    g_out = np.stack([2.0 * d.real * s / m, 2.0 * d.imag * s / m], axis=-1)
    grads, _ = cnn.backward(P, specs, tape, g_out, grad_quantize=grad_quantize)
    return loss, grads
