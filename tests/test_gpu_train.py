"""GPU parity of the training path (Sec. 4.1-4.2, Eq. 4.2-4.3, Alg. 2) against
the oracle, through the C ABI.

* Eq. 4.3 data: r and e from fixed-step V-cycle-preconditioned FGMRES equal the
  oracle's, and H e = r holds for every generated pair;
* Alg. 2 data step in both readings keeps H e = r;
* the loss of Eq. 4.2 and its gradient (hand-written BF16 backward on the
  tensor cores, FP32 weight gradients) agree with the oracle's float64
  backward through the same BF16-rounded forward;
* Adam steps on the GPU lower the loss.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import cnn, helmholtz as H, multigrid as MG, training as T  # noqa: E402
from paper_2405_17696_gb300 import media  # noqa: E402


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_17696_gb300 import build
    build.build()
    from paper_2405_17696_gb300 import native as n
    return n


def _setup(native, w, widths=None, theta=None, **opts):
    net = None
    if widths is not None:
        net = native.cnn_create(len(widths), widths)
        native.cnn_set_params(net, theta.astype(np.float32))
        opts.setdefault("precond", native.HELM_PC_CNN)
    o = native.helm_default_opts(**opts)
    om = torch.from_numpy(np.asarray(w.omegas, dtype=np.float32)).cuda()
    ctx = native.helm_setup(torch.from_numpy(w.kappa).cuda(), torch.from_numpy(w.gamma).cuda(), w.nx, w.nz, w.h,
                            w.h, om, net=net, opts=o)
    return net, ctx


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def _pair_defect_ok(e, r, kap, gam, om, h):
    """H e = r up to the complex64 storage of e: |H e - r| <= 1e-6 || (|H| |e|) ||
    (unit roundoff 6e-8 with a margin; e is O(1) while r may be 1e-4 of H e's terms)."""
    e64 = e.astype(np.complex128)
    he = H.helmholtz_apply(e64, kap, gam, om, h, h)
    coef = np.abs(H.helmholtz_coefficient(kap, gam, om))
    scale = np.linalg.norm((8.0 / h ** 2 + coef) * np.abs(e64))
    return np.linalg.norm(he - r) <= 1e-6 * scale


def test_make_samples_parity(native):
    w = media.crop_workload(64, 32, freqs=(5.0,), width=8)
    x = media.complex_normal((4, w.nz, w.nx), seed=media.SEED_DATAGEN)
    iters = [1, 3, 5, 10]
    _, ctx = _setup(native, w, mg_levels=3)
    try:
        r = np.zeros_like(x)
        e = np.zeros_like(x)
        native.cnn_make_samples(ctx, x, iters, r, e, 4)
    finally:
        native.helm_destroy(ctx)
    om = float(np.float32(w.omegas[0]))
    kap, gam = _f64(w.kappa), _f64(w.gamma)
    r_ref, e_ref = T.make_samples(kap, gam, om, w.h, x, iters)
    for i in range(4):
        # e is the small remainder x - x~: compare the iterate x~ (relative 1e-5)
        assert np.linalg.norm(e[i] - e_ref[i]) <= 1e-5 * np.linalg.norm(x[i] - e_ref[i]), i
        # r = b - H x~ cancels two O(||b||) terms once GMRES has converged, so the
        # complex64 rounding of x~ (unit roundoff 6e-8) enters r as |H| |x~| u
        xt = (x[i] - e_ref[i]).astype(np.complex128)
        coef = np.abs(H.helmholtz_coefficient(kap, gam, om))
        r_floor = 2.5e-7 * np.linalg.norm((8.0 / w.h ** 2 + coef) * np.abs(xt))
        assert np.linalg.norm(r[i] - r_ref[i]) <= 2e-3 * np.linalg.norm(r_ref[i]) + r_floor, i
        assert _pair_defect_ok(e[i], r[i], kap, gam, om, w.h), i


@pytest.mark.parametrize("literal", [0, 1])
def test_refine_samples_keep_pairs_consistent(native, literal):
    w = media.crop_workload(64, 32, freqs=(5.0,), width=8)
    specs = cnn.layer_specs(widths=(16, 32))
    theta = 0.5 * cnn.he_init(specs, seed=1)
    net, ctx = _setup(native, w, widths=(16, 32), theta=theta, mg_levels=3)
    try:
        x = media.complex_normal((3, w.nz, w.nx), seed=7)
        r = np.zeros_like(x)
        e = np.zeros_like(x)
        native.cnn_make_samples(ctx, x, [2, 2, 2], r, e, 3)
        r2 = np.zeros_like(x)
        e2 = np.zeros_like(x)
        native.cnn_refine_samples(ctx, r, e, r2, e2, 3, literal=literal)
    finally:
        native.helm_destroy(ctx)
        native.cnn_destroy(net)
    om = float(np.float32(w.omegas[0]))
    kap, gam = _f64(w.kappa), _f64(w.gamma)
    for i in range(3):
        assert _pair_defect_ok(e2[i], r2[i], kap, gam, om, w.h), i
        assert np.linalg.norm(r2[i]) > 0


@pytest.mark.parametrize("literal", [0, 1])
def test_refine_samples_parity(native, literal):
    """Alg. 2 data step against the oracle, element by element: the GPU network's own
    estimate e_net (cnn_precond_apply without V-cycle) is handed to the oracle's step,
    so that both sides take one preconditioned GMRES step from the same x0."""
    w = media.crop_workload(64, 32, freqs=(5.0,), width=8)
    specs = cnn.layer_specs(widths=(16, 32))
    theta = 0.5 * cnn.he_init(specs, seed=1)
    net, ctx = _setup(native, w, widths=(16, 32), theta=theta, mg_levels=3)
    try:
        x = media.complex_normal((3, w.nz, w.nx), seed=17)
        r = np.zeros_like(x)
        e = np.zeros_like(x)
        native.cnn_make_samples(ctx, x, [1, 2, 4], r, e, 3)
        e_net = np.zeros_like(x)
        native.cnn_precond_apply(ctx, r, e_net, 3, None, 0)
        r2 = np.zeros_like(x)
        e2 = np.zeros_like(x)
        native.cnn_refine_samples(ctx, r, e, r2, e2, 3, literal=literal)
    finally:
        native.helm_destroy(ctx)
        native.cnn_destroy(net)
    om = float(np.float32(w.omegas[0]))
    kap, gam = _f64(w.kappa), _f64(w.gamma)
    r_ref, e_ref = T.refine_from_estimate(kap, gam, om, w.h, r, e, e_net, literal=bool(literal))
    coef = np.abs(H.helmholtz_coefficient(kap, gam, om))
    for i in range(3):
        # the step's iterate e~ (e - e' in the residual-correction reading): relative 1e-5
        et = e_ref[i] if literal else e[i] - e_ref[i]
        et_gpu = e2[i] if literal else e[i] - e2[i]
        assert np.linalg.norm(et_gpu - et) <= 1e-5 * np.linalg.norm(et), i
        # the residual: relative 2e-3 plus the complex64 rounding of e~ through |H|
        r_floor = 2.5e-7 * np.linalg.norm((8.0 / w.h ** 2 + coef) * np.abs(et))
        assert np.linalg.norm(r2[i] - r_ref[i]) <= 2e-3 * np.linalg.norm(r_ref[i]) + r_floor, i


@pytest.mark.parametrize("widths", [(16, 32), (16, 32, 64, 128)])
@pytest.mark.parametrize("relative", [0, 1])
def test_loss_and_gradient_parity(native, relative, widths):
    """Loss of Eq. 4.2 and its gradient against the oracle's float64 backward through
    the same BF16 decisions: inputs, weights and stored activations rounded to BF16
    (as the GPU stores them) and the gradient operand of every convolution rounded to
    BF16 (as the GPU's backward pass forms it).

    The single-layer backward agrees element by element to FP32 accumulation error
    (tests/test_gpu_conv_backward.py).  Through the whole network the remaining
    difference is which side of a BF16 rounding an activation falls when its FP32 and
    float64 sums straddle the boundary; these flips compound with depth.  The bound per
    layer (and for the whole gradient) is therefore 1e-2 relative, or three times the
    oracle's own spread when every value it rounds is first moved by a random relative
    step of the size of the GPU's FP32 accumulation error (sums of K ~ 10^3 products
    with unit roundoff 2^-24: about sqrt(K) 2^-24 = 2^-19), whichever is larger."""
    w = media.crop_workload(32, 32, freqs=(5.0,), width=6)
    specs = cnn.layer_specs(widths=widths)
    g = np.random.default_rng(5)
    theta = 0.5 * cnn.he_init(specs, seed=3) + 0.01 * g.normal(size=cnn.n_params(specs))
    r = media.complex_normal((2, w.nz, w.nx), seed=8)
    e = media.complex_normal((2, w.nz, w.nx), seed=9) * 20.0
    net, ctx = _setup(native, w, widths=widths, theta=theta, mg_levels=2)
    try:
        grad = np.zeros(theta.size, np.float32)
        native.cnn_set_loss(net, relative)
        loss = native.cnn_loss_grad(net, ctx, r, e, 2, grad_out=grad)
        grad2 = np.zeros(theta.size, np.float32)
        native.cnn_loss_grad(net, ctx, r, e, 2, grad_out=grad2)
    finally:
        native.helm_destroy(ctx)
        native.cnn_destroy(net)
    assert np.array_equal(grad, grad2)          # deterministic: no floating-point atomics
    om = float(np.float32(w.omegas[0]))
    P = cnn.unflatten(cnn.bf16_round(theta), specs)
    kap, gam = _f64(w.kappa), _f64(w.gamma)
    loss_ref, grads = T.loss_and_grad(P, specs, kap, gam, om, w.h, r, e, quantize=cnn.bf16_round,
                                      relative=bool(relative), grad_quantize=cnn.bf16_round)
    jitter = np.random.default_rng(17)
    nudged = lambda a: cnn.bf16_round(np.asarray(a, dtype=np.float64) *
                                      (1 + 2.0 ** -19 * jitter.standard_normal(np.shape(a))))
    _, grads_alt = T.loss_and_grad(P, specs, kap, gam, om, w.h, r, e, quantize=nudged, relative=bool(relative),
                                   grad_quantize=nudged)
    gref = cnn.flatten_grads(grads, specs)
    galt = cnn.flatten_grads(grads_alt, specs)
    assert abs(loss - loss_ref) <= 1e-2 * loss_ref, (loss, loss_ref)
    rel = np.linalg.norm(grad - gref) / np.linalg.norm(gref)
    spread = np.linalg.norm(galt - gref) / np.linalg.norm(gref)
    assert rel <= max(1e-2, 3 * spread), (rel, spread)
    # every layer separately (weights and bias), encoder included, and every layer receives gradient
    o = 0
    for name, ci, co, _ in specs:
        n = co * 9 * ci + co
        gl, rl, al = grad[o:o + n], gref[o:o + n], galt[o:o + n]
        assert np.any(gl[:co * 9 * ci] != 0), name
        err = np.linalg.norm(gl - rl) / np.linalg.norm(rl)
        sp = np.linalg.norm(al - rl) / np.linalg.norm(rl)
        assert err <= max(1e-2, 3 * sp), (name, err, sp)
        o += n


def test_adam_steps_lower_the_loss(native):
    w = media.crop_workload(64, 32, freqs=(5.0,), width=8)
    widths = (16, 32, 64)
    specs = cnn.layer_specs(widths=widths)
    theta = 0.5 * cnn.he_init(specs, seed=media.SEED_CNN)
    net, ctx = _setup(native, w, widths=widths, theta=theta, mg_levels=3)
    try:
        x = media.complex_normal((8, w.nz, w.nx), seed=media.SEED_DATAGEN)
        r = torch.zeros((8, w.nz, w.nx), dtype=torch.complex64, device="cuda")
        e = torch.zeros_like(r)
        native.cnn_make_samples(ctx, torch.from_numpy(x).cuda(), [3] * 8, r, e, 8)
        losses = [native.cnn_train_step(net, ctx, r, e, 8, 1e-3) for _ in range(30)]
    finally:
        native.helm_destroy(ctx)
        native.cnn_destroy(net)
    assert np.mean(losses[-5:]) < 0.9 * losses[0], losses


def test_trained_network_reduces_iterations(native):
    """What the trained network gains (Sec. 4.1-4.2): on a 128x64 layered medium at
    6 Hz, Alg. 2 training from seeded He weights (1500 Adam steps through
    cnn_retrain_step, batch 16, Eq. 4.3 data, each pair's error weighted by
    1 / ||e||^2) makes CNN-FGMRES reach 1e-6 in well under the iterations of
    MG-FGMRES.  Training is deterministic (no floating-point atomics in the backward
    pass), so one seeded run is the whole claim."""
    from paper_2405_17696_gb300 import retrain as RT
    nx, nz, h = 128, 64, 20.0
    c = media.layered_velocity(nx, nz, seed=0)
    w = media.Workload("gain", nx, nz, h, [6.0], media.kappa_of(c), media.abl_gamma(nx, nz, 16),
                       media.top_row_positions(nx, 8))
    kap = torch.from_numpy(w.kappa).cuda()
    gam = torch.from_numpy(w.gamma).cuda()
    om = torch.from_numpy(np.asarray(w.omegas, np.float32)).cuda()
    rhs = torch.from_numpy(w.rhs()).cuda()
    nb = rhs.shape[0]

    def solve(ctx):
        x = torch.zeros(rhs.shape, dtype=torch.complex128, device="cuda")
        st, it, rel, _ = native.helm_solve(ctx, rhs, x, nb, None, 1e-6, native.HELM_SOLVE_ZERO_X0)
        assert st == native.HELM_OK and rel.max() <= 1e-6
        return float(it.mean())

    ctx = native.helm_setup(kap, gam, nx, nz, h, h, om, opts=native.helm_default_opts(mg_levels=3, max_iter=600))
    try:
        mg = solve(ctx)
    finally:
        native.helm_destroy(ctx)
    widths = (16, 32, 64, 128)
    net = native.cnn_create(len(widths), widths, seed=media.SEED_CNN)
    ctx = None
    try:
        ctx = native.helm_setup(kap, gam, nx, nz, h, h, om, net=net, opts=native.helm_default_opts(
            mg_levels=3, max_iter=600, precond=native.HELM_PC_CNN, max_rhs=32))
        untrained = solve(ctx)
        steps = 1500
        cfg = RT.RetrainConfig(initial_size=128, data_epochs=3, epochs=3 + -(-(steps - 56) // 64), batch=16,
                               lr=1e-3, lr_final=1e-4, max_steps=steps, relative_loss=True)
        hist = RT.retrain(native, net, ctx, cfg=cfg)
        trained = solve(ctx)
    finally:
        if ctx is not None:
            native.helm_destroy(ctx)
        native.cnn_destroy(net)
    assert hist.epoch_loss[-1] < 0.5 * hist.epoch_loss[0], hist.epoch_loss
    assert trained <= 0.6 * mg, (trained, mg, untrained)
