"""GPU parity of the tensor-core network layers and of the whole
encoder-solver forward pass against the oracle (Fig. 1 caption, Eq. 3.13,
4.1), through the C ABI.

Both sides take the same decisions in the same precision: inputs and weights
are rounded to bfloat16, every stored activation is rounded to bfloat16, and
the sums are exact-ish on the oracle side (float64) and FP32 on the tensor
cores; the output layer stays FP32.  Single layers therefore agree to about
one bfloat16 unit; the whole network, whose activations may round to the
other side of a tie after ~60 layers, agrees to 1e-2 relative L2.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import cnn  # noqa: E402


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_17696_gb300 import build
    build.build()
    from paper_2405_17696_gb300 import native as n
    return n


MODES = {"same": 0, "down": 1, "up": 2}


@pytest.mark.parametrize("c0,c1,bcast,cout,mode,hin,win,nb,res,relu", [
    (16, 0, 0, 16, "same", 20, 12, 2, False, True),      # 480 pixels: ragged last tile
    (3, 0, 0, 16, "same", 16, 16, 1, False, True),       # network input layer (3 -> padded 16)
    (32, 0, 0, 32, "same", 16, 24, 2, True, True),       # ResNet second conv: residual + ReLU
    (64, 64, 1, 64, "same", 8, 16, 3, False, True),      # concat with a batch-shared context
    (16, 16, 0, 16, "same", 12, 20, 2, False, True),     # concat of two 16-channel tensors
    (16, 0, 0, 32, "down", 24, 16, 2, False, True),
    (128, 0, 0, 64, "up", 6, 10, 2, False, True),
    (32, 0, 0, 16, "up", 40, 70, 2, False, True),        # the last decoder layer's shape: many tiles, ragged
    (64, 0, 0, 32, "up", 17, 30, 2, True, True),         # residual on the fine grid
    (32, 16, 0, 16, "up", 9, 14, 2, False, False),       # concat input, no activation
    (16, 0, 0, 64, "up", 5, 130, 1, False, True),        # 130 coarse columns: two column tiles
    (128, 128, 0, 128, "same", 8, 8, 2, False, True),
    (16, 0, 0, 2, "same", 16, 20, 2, False, False),      # output layer, 2 channels
    (32, 16, 0, 16, "same", 6, 200, 2, True, True),      # 3 channel groups, wide rows: 2 column tiles
    (16, 0, 0, 128, "same", 5, 127, 1, False, True),     # 127 wide: one M block per row
    (64, 0, 0, 64, "same", 37, 40, 1, True, True),       # narrow rows packed into M blocks, ragged rows
    (32, 32, 1, 32, "down", 18, 22, 2, False, True),     # concat in the stride-2 gather path
])
@pytest.mark.parametrize("path", [0, 1, 2, 3, "single", "upsplit"])
def test_conv_layer_parity(native, c0, c1, bcast, cout, mode, hin, win, nb, res, relu, path):
    """path 0: the TMA halo-tile kernel (up layers on phase-merged weights); path 1: the
    gather kernel; path 2: the TMA
    kernel with the column taps in N for 16-channel same-grid layers; path 3: the TMA
    kernel with the three tap rows in N for 16- and 32-channel same-grid layers; "single":
    the TMA kernel with one accumulator buffer; "upsplit": up layers with a tile per output
    row parity."""
    g = np.random.default_rng(c0 * 7 + cout + MODES[mode])
    x0 = cnn.bf16_round(g.normal(size=(nb, hin, win, c0)))
    x1 = cnn.bf16_round(g.normal(size=((1 if bcast else nb), hin, win, c1))) if c1 else None
    w = cnn.bf16_round(g.normal(size=(cout, 9, c0 + c1)) / np.sqrt(9 * (c0 + c1)))
    b = g.normal(size=cout) * 0.1
    ho, wo = cnn.out_shape(hin, win, mode)
    r = cnn.bf16_round(g.normal(size=(nb, ho, wo, cout))) if res else None
    xin = x0 if x1 is None else np.concatenate([x0, np.broadcast_to(x1, (nb,) + x1.shape[1:])], axis=-1)
    ref = cnn.conv_forward(xin, w, b, mode)
    if r is not None:
        ref = ref + r
    if relu:
        ref = np.maximum(ref, 0)
    ref = cnn.bf16_round(ref)
    y = np.zeros((nb, ho, wo, cout), np.float32)
    f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
    t0, g0 = native.cnn_conv_launch_counts()
    n0 = native.cnn_conv_narrow_launches()
    n6 = native.cnn_conv_rowtaps_launches()
    single, upsplit = path == "single", path == "upsplit"
    path = 0 if single or upsplit else path
    native.cnn_set_conv_path(path)
    native.cnn_set_conv_buffers(1 if single else 0)
    native.cnn_set_conv_upsplit(1 if upsplit else 0)
    try:
        native.cnn_conv3x3(f32(x0), c0, f32(x1), c1, bcast, nb, hin, win, f32(w), f32(b), cout, f32(r),
                           MODES[mode], 1 if relu else 0, y)
    finally:
        native.cnn_set_conv_path(0)
        native.cnn_set_conv_buffers(0)
        native.cnn_set_conv_upsplit(0)
    t1, g1 = native.cnn_conv_launch_counts()
    used_tma = path != 1
    assert (t1 - t0, g1 - g0) == ((1, 0) if used_tma else (0, 1))
    narrow = path == 2 and mode == "same" and cout <= 16
    assert native.cnn_conv_narrow_launches() - n0 == (1 if narrow else 0)
    rowtaps = path == 3 and mode == "same" and cout <= 32
    assert native.cnn_conv_rowtaps_launches() - n6 == (1 if rowtaps else 0)
    err = np.abs(y - ref)
    tol = 2.0 ** -7 * np.abs(ref) + 1e-3 * np.abs(ref).max()
    if mode == "up" and used_tma:
        # the tensor-map kernel runs an up layer on its phase-merged weights: per output parity
        # the taps that read the same coarse node are added in FP32 and rounded to BF16 once,
        # an error of at most 2^-8 |w_a + w_b + ...| <= 2^-8 (|w_a| + |w_b| + ...) per merged
        # weight, so at most 2^-8 sum |w| |x| over the nine taps per output
        tol = tol + 2.0 ** -8 * cnn.conv_forward(np.abs(xin), np.abs(w), np.zeros(cout), mode)
    assert np.all(err <= tol), (err.max(), np.abs(ref).max())


@pytest.mark.parametrize("widths,ny,nx,nsol,path", [((16, 32), 32, 32, 2, 0), ((16, 32, 64, 128), 64, 32, 2, 0),
                                                    ((16, 32, 64, 128), 64, 160, 2, 3)])
def test_network_forward_parity(native, widths, ny, nx, nsol, path):
    # Half-scale He weights keep the random network contractive: with full-scale
    # weights a one-unit change of a single rounding decision already moves the
    # output of this 60-layer BF16 network by a few percent (measured on the
    # oracle), which would hide real errors.  The tolerance is three times the
    # oracle's own spread under perturbed rounding, at least 1e-2.
    specs = cnn.layer_specs(widths=widths)
    g = np.random.default_rng(3)
    theta = 0.5 * cnn.he_init(specs, seed=2) + 0.02 * g.normal(size=cnn.n_params(specs))
    theta_bf = cnn.bf16_round(theta)                        # the weights the GPU uses
    enc_in = cnn.bf16_round(g.normal(size=(1, ny, nx, 3)))
    sol_in = cnn.bf16_round(g.normal(size=(nsol, ny, nx, 3)))
    P = cnn.unflatten(theta_bf, specs)
    ref, _ = cnn.network_forward(P, specs, enc_in, sol_in, quantize=cnn.bf16_round)
    nudged = lambda a: cnn.bf16_round(np.asarray(a, dtype=np.float32).astype(np.float64) * (1 + 2.0 ** -22))
    alt, _ = cnn.network_forward(P, specs, enc_in, sol_in, quantize=nudged)
    spread = np.linalg.norm(alt - ref) / np.linalg.norm(ref)
    net = native.cnn_create(len(widths), widths)
    try:
        assert native.cnn_num_params(net) == theta.size
        native.cnn_set_params(net, theta.astype(np.float32))
        out = np.zeros((nsol, ny, nx, 2), np.float32)
        native.cnn_set_conv_path(path)
        try:
            native.cnn_forward(net, enc_in.astype(np.float32), 1, sol_in.astype(np.float32), nsol, ny, nx, out)
        finally:
            native.cnn_set_conv_path(0)
        back = np.zeros(theta.size, np.float32)
        native.cnn_get_params(net, back)
    finally:
        native.cnn_destroy(net)
    assert np.array_equal(back, theta.astype(np.float32))
    rel = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert rel <= max(1e-2, 3 * spread), (rel, spread)


# --------------------------------------------------------------------------
# the network as a preconditioner inside the solver (Eq. 3.14)
# --------------------------------------------------------------------------

def _net_ctx(native, w, widths=(16, 32, 64), seed=4, **opts):
    from paper_2405_17696_gb300 import media  # noqa: F401
    specs = cnn.layer_specs(widths=widths)
    theta = cnn.he_init(specs, seed=seed) * 0.5
    net = native.cnn_create(len(widths), widths)
    native.cnn_set_params(net, theta.astype(np.float32))
    o = native.helm_default_opts(precond=native.HELM_PC_CNN, **opts)
    om = torch.from_numpy(np.asarray(w.omegas, dtype=np.float32)).cuda()
    ctx = native.helm_setup(torch.from_numpy(w.kappa).cuda(), torch.from_numpy(w.gamma).cuda(), w.nx, w.nz, w.h,
                            w.h, om, net=net, opts=o)
    return net, ctx, specs, theta


@pytest.mark.parametrize("comp", [3, 2, 0])
def test_network_preconditioner_parity(native, comp):
    from paper_2405_17696_gb300 import media
    from oracle import helmholtz as H, multigrid as MG, training as T
    w = media.crop_workload(64, 32, freqs=(4.0, 7.0), width=8)
    net, ctx, specs, theta = _net_ctx(native, w, mg_levels=3, cnn_vcycle=comp)
    try:
        nb = 3
        fi = np.array([1, 0, 1], np.int32)
        r = media.complex_normal((nb, w.nz, w.nx), seed=12) * 1e-3
        e0 = np.zeros_like(r)
        native.cnn_precond_apply(ctx, r, e0, nb, fi, 0)
        e = np.zeros_like(r)
        native.cnn_precond_apply(ctx, r, e, nb, fi, 1)
    finally:
        native.helm_destroy(ctx)
        native.cnn_destroy(net)
    P = cnn.unflatten(cnn.bf16_round(theta), specs)
    kap, gam = w.kappa.astype(np.float64), w.gamma.astype(np.float64)
    for b in range(nb):
        om = float(np.float32(w.omegas[fi[b]]))
        enc = cnn.bf16_round(cnn.encoder_input(kap, gam, om, w.h))
        x, rms = cnn.solver_input(r[b], gam)
        out, _ = cnn.network_forward(P, specs, enc, cnn.bf16_round(x), quantize=cnn.bf16_round)
        ref0 = cnn.solver_output_to_error(out, rms, w.h)[0]
        assert np.linalg.norm(e0[b] - ref0) <= 2e-2 * np.linalg.norm(ref0)
        # the multigrid part, from the GPU's own e_0: (a) e_0 + V(r - (a) H e_0)
        pc = MG.VCyclePreconditioner(kap, gam, om, w.h, w.h, MG.VCycleParams(levels=3))
        A = lambda u: H.helmholtz_apply(u, kap, gam, om, w.h, w.h)
        ref = T.mvu_compose(e0[b].astype(np.complex128), r[b].astype(np.complex128), A, pc,
                            "guarded" if comp == 3 else "residual")
        assert np.linalg.norm(e[b] - ref) <= 2e-4 * np.linalg.norm(ref)


def test_cnn_fgmres_solve(native):
    from oracle import helmholtz as H
    from paper_2405_17696_gb300 import media
    w = media.crop_workload(128, 64, freqs=(4.0, 6.0), width=16)
    net, ctx, specs, theta = _net_ctx(native, w, mg_levels=3)
    try:
        rhs = w.rhs()
        fi = w.freq_index()
        x = torch.zeros(rhs.shape, dtype=torch.complex128, device="cuda")
        st, iters, rel, stat = native.helm_solve(ctx, torch.from_numpy(rhs).cuda(), x, rhs.shape[0], fi, 1e-6,
                                                 native.HELM_SOLVE_ZERO_X0)
        xs = x.cpu().numpy()
    finally:
        native.helm_destroy(ctx)
        native.cnn_destroy(net)
    assert st == native.HELM_OK, (stat, iters)
    kap, gam = w.kappa.astype(np.float64), w.gamma.astype(np.float64)
    for b in range(rhs.shape[0]):
        om = float(np.float32(w.omegas[fi[b]]))
        assert H.relative_residual(xs[b], rhs[b], kap, gam, om, w.h, w.h) <= 1e-6


def test_init_params_he_normal(native):
    """cnn_init_params: zero biases, per-layer He-normal spread, reproducible by seed."""
    widths = (16, 32, 64, 128)
    specs = cnn.layer_specs(widths=widths)
    net = native.cnn_create(len(widths), widths)
    try:
        native.cnn_init_params(net, 7, 0.5)
        a = np.zeros(cnn.n_params(specs), np.float32)
        native.cnn_get_params(net, a)
        native.cnn_init_params(net, 7, 0.5)
        b = np.zeros_like(a)
        native.cnn_get_params(net, b)
        native.cnn_init_params(net, 8, 0.5)
        c = np.zeros_like(a)
        native.cnn_get_params(net, c)
    finally:
        native.cnn_destroy(net)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    o = 0
    for name, ci, co, _ in specs:
        nw = co * 9 * ci
        wts, bias = a[o:o + nw], a[o + nw:o + nw + co]
        o += nw + co
        assert np.all(bias == 0), name
        sd = 0.5 * np.sqrt(2.0 / (9 * ci))
        # sample std within 5 standard errors of the target
        assert abs(wts.std() / sd - 1) < 5 / np.sqrt(2 * nw) + 1e-3, (name, wts.std(), sd)
        assert abs(wts.mean()) < 5 * sd / np.sqrt(nw), name


def test_autotune_keeps_the_network_output(native):
    """cnn_autotune times the candidate tilings of each layer shape and keeps the
    fastest; the network's output stays the oracle's (same tolerance as the
    forward parity test) and agrees with the untuned pass."""
    from paper_2405_17696_gb300 import media
    w = media.crop_workload(128, 64, freqs=(5.0,), width=12)
    net, ctx, specs, theta = _net_ctx(native, w, mg_levels=3)
    native.cnn_autotune_reset()
    try:
        nb = 4
        fi = np.zeros(nb, np.int32)
        r = media.complex_normal((nb, w.nz, w.nx), seed=21) * 1e-3
        e0 = np.zeros_like(r)
        native.cnn_precond_apply(ctx, r, e0, nb, fi, 0)
        n = native.cnn_autotune(ctx, nb)
        e1 = np.zeros_like(r)
        native.cnn_precond_apply(ctx, r, e1, nb, fi, 0)
    finally:
        native.cnn_autotune_reset()
        native.helm_destroy(ctx)
        native.cnn_destroy(net)
    assert n >= 8   # distinct layer shapes of the solver pass
    assert np.linalg.norm(e1 - e0) <= 2e-2 * np.linalg.norm(e0)
    P = cnn.unflatten(cnn.bf16_round(theta), specs)
    kap, gam = w.kappa.astype(np.float64), w.gamma.astype(np.float64)
    om = float(np.float32(w.omegas[0]))
    enc = cnn.bf16_round(cnn.encoder_input(kap, gam, om, w.h))
    for b in range(nb):
        x, rms = cnn.solver_input(r[b], gam)
        out, _ = cnn.network_forward(P, specs, enc, cnn.bf16_round(x), quantize=cnn.bf16_round)
        ref = cnn.solver_output_to_error(out, rms, w.h)[0]
        assert np.linalg.norm(e1[b] - ref) <= 2e-2 * np.linalg.norm(ref)
