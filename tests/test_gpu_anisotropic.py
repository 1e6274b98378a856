"""Anisotropic grids, hx != hz (the paper's SEG/EAGE and Marmousi grids have unequal
spacings, Sec. 5.2 and 5.5), on the GPU against the oracle: the operator, the
V-cycle, MG-FGMRES solves, the network preconditioner (which sees the geometric-mean
spacing sqrt(hx hz)), the Eq. 4.3 training pairs and the FWI gradient."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import cnn, fwi, helmholtz as H, multigrid as MG, training as T  # noqa: E402
from paper_2405_17696_gb300 import media  # noqa: E402

HX, HZ = 22.0, 14.0          # the SEG/EAGE grid's spacings (13.5 km / 608, 4.2 km / 304), rounded


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_17696_gb300 import build
    build.build()
    from paper_2405_17696_gb300 import native as n
    return n


def _medium(nx=96, nz=48):
    c = media.layered_velocity(nx, nz, seed=5, n_layers=6)
    return nx, nz, media.kappa_of(c), media.abl_gamma(nx, nz, 8), [4.0, 6.0]


def _ctx(native, nx, nz, kappa, gamma, freqs, net=None, **opts):
    om = torch.from_numpy(np.asarray([2 * math.pi * f for f in freqs], np.float32)).cuda()
    return native.helm_setup(torch.from_numpy(kappa).cuda(), torch.from_numpy(gamma).cuda(), nx, nz, HX, HZ, om,
                             net=net, opts=native.helm_default_opts(**opts))


def _f64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def test_operator_vcycle_and_solve(native):
    nx, nz, kap, gam, freqs = _medium()
    ctx = _ctx(native, nx, nz, kap, gam, freqs, mg_levels=3, max_iter=800)
    try:
        nb = 2
        fi = np.array([0, 1], np.int32)
        x = media.complex_normal((nb, nz, nx), seed=3)
        y = np.zeros_like(x)
        native.helm_apply(ctx, x, y, nb, fi, native.HELM_OP_H)
        f = media.complex_normal((nb, nz, nx), seed=4)
        u = np.zeros_like(f)
        native.helm_vcycle(ctx, f, None, u, nb, fi)
        rhs = media.point_source_rhs(nx, nz, [(2, 20), (2, 70)], HX, HZ)
        xs = np.zeros(rhs.shape, np.complex128)
        st, it, rel, _ = native.helm_solve(ctx, rhs, xs, nb, fi, 1e-8, native.HELM_SOLVE_ZERO_X0)
    finally:
        native.helm_destroy(ctx)
    assert st == native.HELM_OK
    for b in range(nb):
        om = float(np.float32(2 * math.pi * freqs[fi[b]]))
        ref = H.helmholtz_apply(x[b].astype(np.complex128), _f64(kap), _f64(gam), om, HX, HZ)
        coef = np.abs(H.helmholtz_coefficient(_f64(kap), _f64(gam), om))
        scale = (4.0 / HX ** 2 + 4.0 / HZ ** 2 + coef) * np.abs(x[b])
        assert np.all(np.abs(y[b] - ref) <= 2e-6 * scale.max())
        pc = MG.VCyclePreconditioner(_f64(kap), _f64(gam), om, HX, HZ, MG.VCycleParams(levels=3))
        vref = pc(f[b].astype(np.complex128))
        assert np.linalg.norm(u[b] - vref) <= 2e-4 * np.linalg.norm(vref)
        xd = H.DirectSolver(_f64(kap), _f64(gam), om, HX, HZ).solve(rhs[b])
        assert H.relative_residual(xs[b], rhs[b], _f64(kap), _f64(gam), om, HX, HZ) <= 1e-6
        assert H.relative_error(xs[b], xd) <= 1e-4


def test_network_preconditioner_and_training_pairs(native):
    nx, nz, kap, gam, freqs = _medium(64, 32)
    widths = (16, 32, 64)
    specs = cnn.layer_specs(widths=widths)
    theta = 0.5 * cnn.he_init(specs, seed=4)
    net = native.cnn_create(len(widths), widths)
    native.cnn_set_params(net, theta.astype(np.float32))
    ctx = _ctx(native, nx, nz, kap, gam, freqs, net=net, mg_levels=3, precond=native.HELM_PC_CNN)
    try:
        nb = 2
        fi = np.array([1, 0], np.int32)
        r = media.complex_normal((nb, nz, nx), seed=12) * 1e-3
        e0 = np.zeros_like(r)
        native.cnn_precond_apply(ctx, r, e0, nb, fi, 0)
        x = media.complex_normal((nb, nz, nx), seed=13)
        rs = np.zeros_like(x)
        es = np.zeros_like(x)
        native.cnn_make_samples(ctx, x, [2, 4], rs, es, nb, fi)
    finally:
        native.helm_destroy(ctx)
        native.cnn_destroy(net)
    P = cnn.unflatten(cnn.bf16_round(theta), specs)
    for b in range(nb):
        om = float(np.float32(2 * math.pi * freqs[fi[b]]))
        ref0, _, _, _ = T.network_error(P, specs, _f64(kap), _f64(gam), om, HX, r[b:b + 1], quantize=cnn.bf16_round,
                                        hz=HZ)
        assert np.linalg.norm(e0[b] - ref0[0]) <= 2e-2 * np.linalg.norm(ref0[0])
        r_ref, e_ref = T.make_samples(_f64(kap), _f64(gam), om, HX, x[b:b + 1], [2, 4][b:b + 1],
                                      params=MG.VCycleParams(levels=3), hz=HZ)
        xt = x[b] - e_ref[0]
        assert np.linalg.norm(es[b] - e_ref[0]) <= 1e-5 * np.linalg.norm(xt)


def test_fwi_gradient(native):
    nx, nz, kap, gam, freqs = _medium(64, 32)
    c0 = media.gaussian_smooth(1.0 / kap, 4.0)
    k0 = media.kappa_of(c0)
    src = [(2, 4 + 8 * s) for s in range(8)]
    rcv = [2 * nx + ix for ix in range(1, nx, 2)]
    om = [float(np.float32(2 * math.pi * f)) for f in freqs]
    g = media.point_source_rhs(nx, nz, src, HX, HZ)
    d_obs, _ = fwi.forward_data(_f64(kap), _f64(gam), om, HX, HZ, g, np.array(rcv))
    phi_ref, grad_ref = fwi.misfit_and_gradient(_f64(k0), _f64(gam), om, HX, HZ, g, np.array(rcv), d_obs)
    ctx = _ctx(native, nx, nz, k0, gam, freqs, mg_levels=3)
    try:
        grad = np.zeros((nz, nx), np.float32)
        phi = native.fwi_misfit_grad(ctx, [iz * nx + ix for iz, ix in src], rcv,
                                     np.ascontiguousarray(d_obs, np.complex64), grad, tol=1e-8)
    finally:
        native.helm_destroy(ctx)
    assert abs(phi - phi_ref) <= 1e-5 * phi_ref
    assert np.linalg.norm(grad - grad_ref) <= 1e-3 * np.linalg.norm(grad_ref)
