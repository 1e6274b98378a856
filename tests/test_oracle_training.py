"""Pins of the oracle's Alg. 2 data step (Sec. 4.2): the refined training pair
built from a network estimate by one preconditioned GMRES step.

* With the exact error as the estimate, the step has nothing left to do: the
  residual-correction reading returns the pair (0, 0), the printed reading
  returns (r, e) itself.
* One flexible-GMRES step from x0 is the one-dimensional minimal-residual step
  along z = V(r0 / ||r0||), whose coefficient has the closed form
  <H z, r0> / <H z, H z>; the oracle's e~ must equal x0 + that multiple of z.
* Both readings keep H e' = r' for pairs with H e = r, and the step never raises
  the residual of its starting point.
"""
import numpy as np

from oracle import helmholtz as H, multigrid as MG, training as T
from paper_2405_17696_gb300 import media


def _problem(seed=0):
    w = media.crop_workload(32, 16, freqs=(5.0,), width=4)
    kap, gam = w.kappa.astype(np.float64), w.gamma.astype(np.float64)
    om = float(np.float32(w.omegas[0]))
    x = media.complex_normal((2, w.nz, w.nx), seed=seed).astype(np.complex128)
    A = lambda u: H.helmholtz_apply(u, kap, gam, om, w.h, w.h)
    r = np.stack([A(xi) for xi in x])      # pairs (r, e) = (H x, x) satisfy H e = r exactly
    return w, kap, gam, om, A, r, x


def test_exact_estimate_leaves_nothing_to_refine():
    w, kap, gam, om, A, r, e = _problem(1)
    r2, e2 = T.refine_from_estimate(kap, gam, om, w.h, r, e, e_net=e, literal=False)
    assert np.max(np.abs(r2)) == 0.0 and np.max(np.abs(e2)) == 0.0
    r3, e3 = T.refine_from_estimate(kap, gam, om, w.h, r, e, e_net=e, literal=True)
    for i in range(2):
        assert np.linalg.norm(r3[i] - r[i]) <= 1e-12 * np.linalg.norm(r[i])
        assert np.linalg.norm(e3[i] - e[i]) <= 1e-12 * np.linalg.norm(e[i])


def test_one_step_is_the_closed_form_minimal_residual_step():
    w, kap, gam, om, A, r, e = _problem(2)
    pc = MG.VCyclePreconditioner(kap, gam, om, w.h, w.h, MG.VCycleParams())
    g = np.random.default_rng(3)
    e_net = e + 0.3 * (g.normal(size=e.shape) + 1j * g.normal(size=e.shape)) * np.abs(e).mean()
    r2, e2 = T.refine_from_estimate(kap, gam, om, w.h, r, e, e_net=e_net, literal=False)
    r3, e3 = T.refine_from_estimate(kap, gam, om, w.h, r, e, e_net=e_net, literal=True)
    for i in range(2):
        r0 = r[i] - A(e_net[i])
        z = pc(r0 / np.linalg.norm(r0))
        hz = A(z)
        alpha = np.vdot(hz, r0) / np.vdot(hz, hz)
        et = e_net[i] + alpha * z
        scale = np.linalg.norm(et)
        assert np.linalg.norm(e3[i] - et) <= 1e-10 * scale
        assert np.linalg.norm(e2[i] - (e[i] - et)) <= 1e-10 * scale
        assert np.linalg.norm(r2[i] - (r[i] - A(et))) <= 1e-10 * np.linalg.norm(r[i])
        assert np.linalg.norm(r3[i] - A(et)) <= 1e-10 * np.linalg.norm(r[i])
        # the step lowers the residual of its start and the pairs stay consistent
        assert np.linalg.norm(r2[i]) < np.linalg.norm(r0)
        assert np.linalg.norm(A(e2[i]) - r2[i]) <= 1e-10 * np.linalg.norm(r[i])
        assert np.linalg.norm(A(e3[i]) - r3[i]) <= 1e-10 * np.linalg.norm(r[i])


def test_anisotropic_network_scaling_reduces_to_the_isotropic_one():
    """On a grid with hx hz = h^2 the network sees the same input (w sqrt(hx hz) kappa) and
    its output gets the same scale (hx hz) as on the isotropic grid of spacing h."""
    from oracle import cnn
    w = media.crop_workload(16, 16, freqs=(5.0,), width=4)
    kap, gam = w.kappa.astype(np.float64), w.gamma.astype(np.float64)
    specs = cnn.layer_specs(widths=(16, 32))
    P = cnn.unflatten(0.5 * cnn.he_init(specs, seed=1), specs)
    r = media.complex_normal((1, 16, 16), seed=2).astype(np.complex128)
    h = 20.0
    e_iso, _, _, _ = T.network_error(P, specs, kap, gam, 30.0, h, r)
    e_ani, _, _, _ = T.network_error(P, specs, kap, gam, 30.0, 2.0 * h, r, hz=h / 2.0)
    assert np.allclose(e_iso, e_ani, rtol=1e-13, atol=0)
    e_other, _, _, _ = T.network_error(P, specs, kap, gam, 30.0, 2.0 * h, r, hz=h)
    assert not np.allclose(e_iso, e_other)
