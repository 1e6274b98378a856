"""Pins of the oracle's encoder-solver network pieces (no GPU).

* the 'same' 3x3 convolution equals scipy's 2-D cross-correlation with zero
  padding, channel by channel (a library routine, called);
* 'down' equals 'same' sampled at the odd nodes (2Y+1, 2X+1); 'up' equals
  'same' applied to the nearest-neighbour upsampled input;
* gather/scatter are adjoint (<conv(x), y> = <x, conv^T(y)> without bias);
* the backward pass of the whole encoder-solver network matches central finite
  differences of a scalar loss, for the parameters and for the input;
* one Adam step from zero moments moves every parameter by lr in the
  direction opposite to its gradient sign (Kingma & Ba's bias correction).
"""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def _rng(s):
    return np.random.default_rng(s)


def test_same_conv_is_cross_correlation():
    g = _rng(0)
    x = g.normal(size=(2, 7, 9, 3))
    w = g.normal(size=(4, 9, 3))
    b = g.normal(size=4)
    y = cnn.conv_forward(x, w, b, "same")
    for n in range(2):
        for co in range(4):
            ref = b[co] + sum(correlate2d(x[n, :, :, ci], w[co, :, ci].reshape(3, 3), mode="same", boundary="fill")
                              for ci in range(3))
            assert np.allclose(y[n, :, :, co], ref, atol=1e-12)


def test_down_and_up_modes():
    g = _rng(1)
    x = g.normal(size=(1, 8, 10, 2))
    w = g.normal(size=(3, 9, 2))
    b = g.normal(size=3)
    same = cnn.conv_forward(x, w, b, "same")
    down = cnn.conv_forward(x, w, b, "down")
    assert np.allclose(down, same[:, 1::2, 1::2], atol=1e-12)
    up = cnn.conv_forward(x, w, b, "up")
    xu = np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)
    assert np.allclose(up, cnn.conv_forward(xu, w, b, "same"), atol=1e-12)


@pytest.mark.parametrize("mode", ["same", "down", "up"])
def test_conv_adjoint_identity(mode):
    g = _rng(2)
    x = g.normal(size=(2, 6, 8, 3))
    w = g.normal(size=(5, 9, 3))
    y0 = cnn.conv_forward(x, w, np.zeros(5), mode)
    gy = g.normal(size=y0.shape)
    dx, dw, db = cnn.conv_backward(x, w, gy, mode)
    assert abs(np.sum(y0 * gy) - np.sum(x * dx)) < 1e-10 * abs(np.sum(y0 * gy))
    assert abs(np.sum(y0 * gy) - np.sum(w * dw)) < 1e-10 * abs(np.sum(y0 * gy))


def _tiny():
    specs = cnn.layer_specs(widths=(2, 4), in_enc=3, in_sol=3, out_ch=2)
    theta = cnn.he_init(specs, seed=5) + 0.05 * _rng(6).normal(size=cnn.n_params(specs))
    g = _rng(7)
    enc_in = g.normal(size=(1, 8, 8, 3))
    sol_in = g.normal(size=(2, 8, 8, 3))
    target = g.normal(size=(2, 8, 8, 2))
    return specs, theta, enc_in, sol_in, target


def _loss(specs, theta, enc_in, sol_in, target):
    out, tape = cnn.network_forward(cnn.unflatten(theta, specs), specs, enc_in, sol_in)
    val, gout = cnn.mse(out, target)
    return val, gout, tape


def test_network_backward_matches_finite_differences():
    specs, theta, enc_in, sol_in, target = _tiny()
    P = cnn.unflatten(theta, specs)
    val, gout, tape = _loss(specs, theta, enc_in, sol_in, target)
    grads, _ = cnn.backward(P, specs, tape, gout)
    gflat = cnn.flatten_grads(grads, specs)
    # the loss is piecewise smooth (ReLU kinks lie close to the evaluation
    # point in such a narrow net), so the step must be small
    d = _rng(8).normal(size=theta.size)
    eps = 1e-8
    fp = _loss(specs, theta + eps * d, enc_in, sol_in, target)[0]
    fm = _loss(specs, theta - eps * d, enc_in, sol_in, target)[0]
    fd = (fp - fm) / (2 * eps)
    assert abs(fd - gflat @ d) <= 1e-5 * abs(fd)
    # every layer receives gradient (encoder included, through the context features)
    assert all(np.any(grads[name][0] != 0) for name, *_ in specs)


def test_network_input_gradient():
    specs, theta, enc_in, sol_in, target = _tiny()
    P = cnn.unflatten(theta, specs)
    out, tape = cnn.network_forward(P, specs, enc_in, sol_in)
    val, gout = cnn.mse(out, target)
    _, gx = cnn.backward(P, specs, tape, gout, wrt=sol_in)
    d = _rng(9).normal(size=sol_in.shape)
    eps = 1e-8
    fp = cnn.mse(cnn.network_forward(P, specs, enc_in, sol_in + eps * d)[0], target)[0]
    fm = cnn.mse(cnn.network_forward(P, specs, enc_in, sol_in - eps * d)[0], target)[0]
    assert abs((fp - fm) / (2 * eps) - np.sum(gx * d)) <= 1e-5 * abs((fp - fm) / (2 * eps))


def test_adam_first_step():
    g = _rng(10)
    theta = g.normal(size=20)
    grad = g.normal(size=20)
    t1, m, v = cnn.adam_step(theta, grad, np.zeros(20), np.zeros(20), 1, lr=1e-3, eps=0.0)
    assert np.allclose(t1 - theta, -1e-3 * np.sign(grad), atol=1e-15)
    assert np.allclose(m, 0.1 * grad) and np.allclose(v, 0.001 * grad * grad)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    g = _rng(11)
    x = np.concatenate([g.normal(size=1000) * 10.0 ** g.integers(-20, 20, size=1000),
                        [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0, -0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16_round(x), ref)


def test_training_data_and_loss_gradient():
    # Eq. 4.3 pairs satisfy H e = r exactly; the Eq. 4.2 loss gradient (through
    # the rms scaling of the network input and output) matches finite differences
    from oracle import helmholtz as H, training as T
    from paper_2405_17696_gb300 import media
    w = media.crop_workload(16, 16, freqs=(5.0,), width=4)
    kap, gam, om = w.kappa.astype(float), w.gamma.astype(float), w.omegas[0]
    x = media.complex_normal((2, w.nz, w.nx), seed=3)
    r, e = T.make_samples(kap, gam, om, w.h, x, [1, 3], params=None)
    for i in range(2):
        assert np.linalg.norm(H.helmholtz_apply(e[i], kap, gam, om, w.h, w.h) - r[i]) <= 1e-10 * np.linalg.norm(r[i])
    specs = cnn.layer_specs(widths=(2, 4))
    theta = 0.5 * cnn.he_init(specs, seed=4) + 0.02 * _rng(5).normal(size=cnn.n_params(specs))
    loss, grads = T.loss_and_grad(cnn.unflatten(theta, specs), specs, kap, gam, om, w.h, r, e)
    gflat = cnn.flatten_grads(grads, specs)
    d = _rng(6).normal(size=theta.size)
    eps = 1e-8
    lp = T.loss_and_grad(cnn.unflatten(theta + eps * d, specs), specs, kap, gam, om, w.h, r, e)[0]
    lm = T.loss_and_grad(cnn.unflatten(theta - eps * d, specs), specs, kap, gam, om, w.h, r, e)[0]
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - gflat @ d) <= 1e-5 * abs(fd)


def test_mvu_composition_special_cases():
    """Eq. 3.14 composition: an exact network estimate is returned unchanged
    (V(0) = 0), a zero estimate gives the plain V-cycle, and the V-cycle
    started from e0 is the other reading."""
    from oracle import helmholtz as H, multigrid as MG, training as T
    from paper_2405_17696_gb300 import media
    w = media.crop_workload(32, 32, freqs=(5.0,), width=6)
    kap, gam = np.float64(w.kappa), np.float64(w.gamma)
    om = float(w.omegas[0])
    A = lambda u: H.helmholtz_apply(u, kap, gam, om, w.h, w.h)
    pc = MG.VCyclePreconditioner(kap, gam, om, w.h, w.h, MG.VCycleParams(levels=2))
    r = media.complex_normal((w.nz, w.nx), seed=11).astype(np.complex128)
    exact = H.DirectSolver(kap, gam, om, w.h, w.h).solve(r)
    for comp in ("residual", "guarded"):
        out = T.mvu_compose(exact, r, A, pc, comp)
        assert np.linalg.norm(out - exact) <= 1e-10 * np.linalg.norm(exact), comp
    zero = np.zeros_like(r)
    assert np.allclose(T.mvu_compose(zero, r, A, pc, "residual"), pc(r), rtol=0, atol=1e-14)
    assert np.allclose(T.mvu_compose(zero, r, A, pc, "guarded"), pc(r), rtol=0, atol=1e-14)
    # a good estimate (its step lowers the residual) is used as it is: the guarded
    # composition equals the plain one
    good = exact + 1e-3 * np.linalg.norm(exact) / np.sqrt(exact.size) * media.complex_normal(
        (w.nz, w.nx), seed=14).astype(np.complex128)
    assert np.linalg.norm(r - A(good)) < np.linalg.norm(r)
    assert np.allclose(T.mvu_compose(good, r, A, pc, "guarded"), T.mvu_compose(good, r, A, pc, "residual"),
                       rtol=0, atol=1e-12 * np.linalg.norm(exact))
    # a harmful estimate (its step raises the residual) is scaled: the result does not
    # depend on the estimate's complex scale, and the residual handed on is at most ||r||
    e_bad = media.complex_normal((w.nz, w.nx), seed=13).astype(np.complex128)
    assert np.linalg.norm(r - A(e_bad)) > np.linalg.norm(r)
    m1 = T.mvu_compose(e_bad, r, A, pc, "guarded")
    m2 = T.mvu_compose((2.5 - 1.5j) * e_bad, r, A, pc, "guarded")
    assert np.linalg.norm(m1 - m2) <= 1e-10 * np.linalg.norm(m1)
    t = A(e_bad)
    a = np.vdot(t, r) / np.vdot(t, t)
    assert np.linalg.norm(r - a * t) <= np.linalg.norm(r)
    assert np.linalg.norm(r - a * t) <= np.linalg.norm(r - 1.01 * a * t)
    # with a linear V-cycle (Jacobi coarsest solve) the correction is affine in
    # e0: M(e0) - M(0) = e0 - V(H e0); a sign slip in r - H e0 breaks it
    lin = MG.VCyclePreconditioner(kap, gam, om, w.h, w.h, MG.VCycleParams(levels=2, coarse_kind="jacobi"))
    e0 = media.complex_normal((w.nz, w.nx), seed=12).astype(np.complex128) * 1e-3
    m0 = T.mvu_compose(zero, r, A, lin, "residual")
    d = T.mvu_compose(e0, r, A, lin, "residual") - m0
    assert np.linalg.norm(d - (e0 - lin(A(e0)))) <= 1e-12 * np.linalg.norm(m0)
    assert np.linalg.norm(d) > 1e-3 * np.linalg.norm(e0)
    assert np.allclose(T.mvu_compose(e0, r, A, pc, "initial_guess"), pc(r, e0), rtol=0, atol=1e-14)


def test_relative_loss_gradient_matches_finite_differences():
    """The relative-error weighting of the training loss (each pair divided by
    ||e_i||^2): the oracle's gradient against central differences."""
    from oracle import training as T
    from paper_2405_17696_gb300 import media
    w = media.crop_workload(16, 16, freqs=(5.0,), width=4)
    specs = cnn.layer_specs(widths=(16,))
    theta = 0.5 * cnn.he_init(specs, seed=3)
    r = media.complex_normal((2, 16, 16), seed=4)
    e = media.complex_normal((2, 16, 16), seed=5) * np.array([1.0, 10.0])[:, None, None]
    kap, gam = np.float64(w.kappa), np.float64(w.gamma)
    om = float(w.omegas[0])
    loss, grads = T.loss_and_grad(cnn.unflatten(theta, specs), specs, kap, gam, om, w.h, r, e, relative=True)
    g = cnn.flatten_grads(grads, specs)
    k = np.argsort(-np.abs(g))[:6]
    for i in k:
        t1, t2 = theta.copy(), theta.copy()
        t1[i] += 1e-6
        t2[i] -= 1e-6
        l1, _ = T.loss_and_grad(cnn.unflatten(t1, specs), specs, kap, gam, om, w.h, r, e, relative=True)
        l2, _ = T.loss_and_grad(cnn.unflatten(t2, specs), specs, kap, gam, om, w.h, r, e, relative=True)
        fd = (l1 - l2) / 2e-6
        assert abs(fd - g[i]) <= 1e-4 * abs(g[i]) + 1e-9, (i, fd, g[i])
    # equal weights reduce to Eq. 4.2 scaled by 1 / ||e||^2
    e1 = e[:1]
    l_rel, _ = T.loss_and_grad(cnn.unflatten(theta, specs), specs, kap, gam, om, w.h, r[:1], e1, relative=True)
    l_mse, _ = T.loss_and_grad(cnn.unflatten(theta, specs), specs, kap, gam, om, w.h, r[:1], e1)
    assert abs(l_rel - l_mse / np.sum(np.abs(e1) ** 2)) <= 1e-12 * l_rel


@pytest.mark.parametrize("mode", ["same", "down", "up"])
def test_pointwise_and_tap_by_tap_forms_match_the_layer(mode):
    """The point-by-point forward and input gradient and the tap-by-tap weight gradient
    (used where the full im2col would not fit) equal conv_forward / conv_backward."""
    g = _rng(21)
    x = g.normal(size=(2, 6, 10, 5))
    w = g.normal(size=(4, 9, 5))
    b = g.normal(size=4)
    y = cnn.conv_forward(x, w, b, mode)
    gy = g.normal(size=y.shape)
    dx, dw, db = cnn.conv_backward(x, w, gy, mode)
    pts_out = [(n, Y, X) for n in range(2) for Y in range(y.shape[1]) for X in range(y.shape[2])]
    yp = cnn.conv_forward_points(x, w, b, mode, pts_out)
    assert np.allclose(yp, np.array([y[p] for p in pts_out]), rtol=0, atol=1e-12)
    pts_in = [(n, yy, xx) for n in range(2) for yy in range(6) for xx in range(10)]
    dxp = cnn.conv_input_grad_points(gy, w, x.shape, mode, pts_in)
    assert np.allclose(dxp, np.array([dx[p] for p in pts_in]), rtol=0, atol=1e-12)
    dw2, db2 = cnn.conv_weight_grad(x, gy, mode)
    assert np.allclose(dw2, dw, rtol=0, atol=1e-12) and np.allclose(db2, db, rtol=0, atol=1e-12)


def test_up_layer_is_four_phase_convolutions_on_the_coarse_grid():
    """The identity the tensor-core up layer is built on: nearest x2 upsampling followed by
    a 3x3 convolution (zero padding on the fine grid) equals, for each output parity
    (py, px), a 2x2 convolution on the coarse grid (zero padding there) whose weights are
    the sums of the 3x3 taps that read the same coarse node, fine node 2Y + p with tap d
    reading coarse node floor((2Y + p + d) / 2).  Exact up to FP64 rounding."""
    g = _rng(29)
    B, ny, nx, cin, cout = 2, 5, 7, 3, 4
    x = g.normal(size=(B, ny, nx, cin))
    w = g.normal(size=(cout, 9, cin))
    ref = cnn.conv_forward(x, w, np.zeros(cout), "up")
    xp = np.zeros((B, ny + 2, nx + 2, cin))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((B, 2 * ny, 2 * nx, cout))
    for py in (0, 1):
        for px in (0, 1):
            wm = np.zeros((2, 2, cout, cin))
            for t in range(9):
                dy, dx = t // 3 - 1, t % 3 - 1
                ey, ex = (py + dy) // 2 - py + 1, (px + dx) // 2 - px + 1
                wm[ey, ex] += w[:, t, :]
            for ey in (0, 1):
                for ex in (0, 1):
                    # coarse node (Y + py - 1 + ey, X + px - 1 + ex), + 1 for the padding
                    blk = xp[:, py + ey:py + ey + ny, px + ex:px + ex + nx]
                    y[:, py::2, px::2] += np.einsum("byxc,oc->byxo", blk, wm[ey, ex])
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
