"""GPU parity of one convolution layer's backward pass (training by Adam, Sec. 4.1;
the layers of the Fig. 1 caption) against the oracle, element by element, through
the C ABI (cnn_conv3x3_backward), and of the forward convolution at sizes where
every CTA of the persistent kernels loops over several tiles.

Both sides use the same BF16-rounded inputs, weights and upstream gradient; the
oracle sums in float64, the GPU in FP32 on the tensor cores.  So the weight and
bias gradients (sums over every output pixel) agree to FP32 accumulation error,
and the input gradients (the forward kernel with transposed weights, FP32
output) likewise: the bound below is 1e-3 relative to each element plus 1e-4 of
the largest, far inside the 1e-2 the gradients are held to, and a wrong tap,
transposition or sign moves elements by O(1).
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


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _close(got, ref, rel=1e-3, floor=1e-4):
    err = np.abs(got - ref)
    tol = rel * np.abs(ref) + floor * max(np.abs(ref).max(), 1e-30)
    return bool(np.all(err <= tol)), float(err.max()), float(np.abs(ref).max())


def _inputs(seed, c0, c1, bcast, cout, mode, hin, win, nb):
    g = np.random.default_rng(seed)
    x0 = cnn.bf16_round(g.normal(size=(nb, hin, win, c0)))
    x1 = cnn.bf16_round(g.normal(size=((1 if bcast else nb), hin, win, c1))) if c1 else None
    w = cnn.bf16_round(g.normal(size=(cout, 9, c0 + c1)) / np.sqrt(9 * (c0 + c1)))
    ho, wo = cnn.out_shape(hin, win, mode)
    gy = cnn.bf16_round(g.normal(size=(nb, ho, wo, cout)))
    return x0, x1, w, gy


def _run(native, x0, c0, x1, c1, bcast, nb, hin, win, w, cout, mode, gy, want_dx=True):
    gx0 = np.zeros(x0.shape, np.float32) if want_dx else None
    gx1 = np.zeros(x1.shape, np.float32) if (want_dx and x1 is not None) else None
    dw = np.zeros(w.shape, np.float32)
    db = np.zeros(cout, np.float32)
    native.cnn_conv3x3_backward(_f32(x0), c0, _f32(x1), c1, bcast, nb, hin, win, _f32(w), cout, MODES[mode],
                                _f32(gy), gx0, gx1, dw, db)
    return gx0, gx1, dw, db


@pytest.mark.parametrize("c0,c1,bcast,cout,mode,hin,win,nb", [
    (16, 0, 0, 16, "same", 20, 12, 2),
    (3, 0, 0, 16, "same", 16, 16, 1),       # network input layer (3 channels padded to 16)
    (16, 16, 0, 16, "same", 12, 20, 2),     # concatenation
    (64, 64, 1, 64, "same", 8, 16, 3),      # concatenation with a batch-shared context
    (16, 0, 0, 2, "same", 16, 20, 2),       # output layer
    (16, 0, 0, 32, "down", 24, 16, 2),
    (32, 0, 0, 64, "down", 18, 22, 1),
    (32, 0, 0, 16, "up", 10, 6, 2),
    (128, 0, 0, 64, "up", 6, 10, 2),
    (64, 0, 0, 64, "same", 37, 40, 1),      # ragged tiles
])
@pytest.mark.parametrize("wpath", [0, 1])
def test_conv_layer_backward_parity(native, c0, c1, bcast, cout, mode, hin, win, nb, wpath):
    """wpath 0: the tensor-core weight gradient; 1: the FP32 CUDA-core kernel."""
    x0, x1, w, gy = _inputs(c0 * 7 + cout + MODES[mode], c0, c1, bcast, cout, mode, hin, win, nb)
    xin = x0 if x1 is None else np.concatenate([x0, np.broadcast_to(x1, (nb,) + x1.shape[1:])], axis=-1)
    dx_ref, dw_ref, db_ref = cnn.conv_backward(xin, w, gy, mode)
    native.cnn_set_wgrad_path(wpath)
    try:
        gx0, gx1, dw, db = _run(native, x0, c0, x1, c1, bcast, nb, hin, win, w, cout, mode, gy)
    finally:
        native.cnn_set_wgrad_path(0)
    ok, e, m = _close(dw, dw_ref)
    assert ok, ("dw", e, m)
    ok, e, m = _close(db, db_ref)
    assert ok, ("db", e, m)
    ok, e, m = _close(gx0, dx_ref[..., :c0])
    assert ok, ("dx0", e, m)
    if c1:
        ref1 = dx_ref[..., c0:]
        if bcast:
            ref1 = ref1.sum(axis=0, keepdims=True)
        ok, e, m = _close(gx1, ref1)
        assert ok, ("dx1", e, m)


@pytest.mark.parametrize("c0,c1,cout,mode,hin,win,nb", [
    (16, 16, 16, "same", 128, 128, 4),      # 512 K tiles: >= 3 per CTA
    (32, 0, 64, "down", 256, 256, 4),       # 512 K tiles on the 128 x 128 output grid
    (128, 0, 64, "up", 64, 128, 8),         # 2048 K tiles (4 parities); tap groups of the M split
    (128, 128, 128, "same", 32, 64, 8),     # the coarsest concatenation: 5 tap groups
])
def test_weight_gradient_multi_tile_parity(native, c0, c1, cout, mode, hin, win, nb):
    """Sizes where every CTA of the tensor-core weight gradient accumulates three or more
    K tiles in TMEM: weight and bias gradients element by element against the oracle's
    tap-by-tap form, and the input gradient at sampled nodes against its pointwise form."""
    x0, x1, w, gy = _inputs(11 + c0 + cout, c0, c1, 0, cout, mode, hin, win, nb)
    xin = x0 if x1 is None else np.concatenate([x0, x1], axis=-1)
    plan = native.cnn_wgrad_plan(MODES[mode], c0, c1, 16 * -(-cout // 16), hin, win, nb,
                                 torch.cuda.get_device_properties(0).multi_processor_count)
    assert plan["ktiles"] >= 3 * plan["splits"]
    gx0, gx1, dw, db = _run(native, x0, c0, x1, c1, 0, nb, hin, win, w, cout, mode, gy)
    dw_ref, db_ref = cnn.conv_weight_grad(xin, gy, mode)
    ok, e, m = _close(dw, dw_ref)
    assert ok, ("dw", e, m)
    ok, e, m = _close(db, db_ref)
    assert ok, ("db", e, m)
    g = np.random.default_rng(5)
    pts = [(int(g.integers(nb)), int(g.integers(hin)), int(g.integers(win))) for _ in range(300)]
    pts += [(nb - 1, hin - 1, x) for x in range(win)] + [(0, y, 0) for y in range(hin)]   # edges
    dx_ref = cnn.conv_input_grad_points(gy, w, xin.shape, mode, pts)
    got = np.concatenate([gx0, gx1], axis=-1) if c1 else gx0
    ok, e, m = _close(np.array([got[p] for p in pts]), dx_ref)
    assert ok, ("dx", e, m)


def test_weight_gradient_is_deterministic(native):
    """Two runs of the tensor-core weight gradient give bit-identical results."""
    x0, x1, w, gy = _inputs(3, 16, 16, 0, 16, "same", 96, 128, 3)
    a = _run(native, x0, 16, x1, 16, 0, 3, 96, 128, w, 16, "same", gy, want_dx=False)
    b = _run(native, x0, 16, x1, 16, 0, 3, 96, 128, w, 16, "same", gy, want_dx=False)
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


@pytest.mark.parametrize("c0,c1,bcast,cout,mode,hin,win,nb,path", [
    (16, 16, 0, 16, "same", 256, 256, 16, 0),  # >= 3 tiles per CTA of the persistent forward kernel
    (32, 0, 0, 64, "down", 256, 256, 16, 0),
    (128, 0, 0, 64, "up", 64, 128, 8, 0),
    (64, 64, 1, 64, "same", 128, 128, 16, 0),  # batch-shared context
    (16, 16, 0, 16, "same", 256, 256, 16, 3),  # tap rows in N: slot ring across tiles, two groups
    (32, 0, 0, 32, "same", 200, 300, 16, 3),   # 32 channels, three column tiles of 100
    (16, 16, 0, 16, "same", 256, 256, 16, "single"),   # one accumulator buffer: per-tile phases
    (128, 0, 0, 64, "up", 64, 128, 16, "single"),
    (64, 0, 0, 32, "up", 64, 200, 16, "upsplit"),    # a tile per output row parity, alternating
    (32, 0, 0, 16, "up", 96, 160, 16, "upsplit"),
])
def test_conv_forward_multi_tile_sampled_parity(native, c0, c1, bcast, cout, mode, hin, win, nb, path):
    """The persistent TMA convolution at sizes where every CTA loops over three or more
    tiles (accumulator-buffer alternation, barrier phases and ring reuse across tiles),
    checked at sampled output nodes (all of a few full rows and columns, and random ones)
    against the oracle's point-by-point forward, to one BF16 unit (up layers: plus the
    rounding of their phase-merged weights).  Path 3: the same-grid layers with the three
    tap rows in N."""
    g = np.random.default_rng(c0 + cout)
    x0 = cnn.bf16_round(g.normal(size=(nb, hin, win, c0))).astype(np.float32)
    x1 = cnn.bf16_round(g.normal(size=((1 if bcast else nb), hin, win, c1))).astype(np.float32) if c1 else None
    w = cnn.bf16_round(g.normal(size=(cout, 9, c0 + c1)) / np.sqrt(9 * (c0 + c1)))
    b = g.normal(size=cout) * 0.1
    ho, wo = cnn.out_shape(hin, win, mode)
    y = torch.zeros((nb, ho, wo, cout), dtype=torch.float32, device="cuda")
    n6 = native.cnn_conv_rowtaps_launches()
    single, upsplit = path == "single", path == "upsplit"
    path = 0 if single or upsplit else path
    native.cnn_set_conv_path(path)
    native.cnn_set_conv_buffers(1 if single else 0)
    native.cnn_set_conv_upsplit(1 if upsplit else 0)
    try:
        native.cnn_conv3x3(torch.from_numpy(x0).cuda(), c0, None if x1 is None else torch.from_numpy(x1).cuda(),
                           c1, bcast, nb, hin, win, _f32(w), _f32(b), cout, None, MODES[mode], 1, y)
    finally:
        native.cnn_set_conv_path(0)
        native.cnn_set_conv_buffers(0)
        native.cnn_set_conv_upsplit(0)
    launch = native.cnn_conv_last_launch()
    npad = 16 if cout <= 16 else 32 * -(-cout // 32)
    plan = native.cnn_conv_plan(MODES[mode], 16 * -(-c0 // 16), 16 * -(-c1 // 16) if c1 else 0, npad, hin, win, nb,
                                narrow=2 if path == 3 else (3 if single else (4 if upsplit else 0)))
    assert plan["nbuf"] == (1 if single else (2 if path != 3 else plan["nbuf"]))
    assert plan["mode"] == (6 if path == 3 else MODES[mode])
    if upsplit:
        assert plan["nph"] == 2
    assert native.cnn_conv_rowtaps_launches() - n6 == (1 if path == 3 else 0)
    assert plan["tiles"] >= 3 * launch[0], (plan["tiles"], launch)
    y = y.cpu().numpy()
    pts = [(int(g.integers(nb)), int(g.integers(ho)), int(g.integers(wo))) for _ in range(400)]
    pts += [(nb - 1, ho - 1, X) for X in range(wo)] + [(0, Y, wo - 1) for Y in range(ho)]
    pts += [(nb // 2, ho // 2, X) for X in range(wo)]
    xin = x0 if x1 is None else np.concatenate([x0, np.broadcast_to(x1, (nb,) + x1.shape[1:])], axis=-1)
    ref = cnn.bf16_round(np.maximum(cnn.conv_forward_points(xin.astype(np.float64), w, b, mode, pts), 0.0))
    got = np.array([y[p] for p in pts])
    err = np.abs(got - ref)
    tol = 2.0 ** -7 * np.abs(ref) + 1e-3 * np.abs(ref).max()
    if mode == "up":
        # phase-merged BF16 weights: at most 2^-8 sum |w| |x| over the nine taps per output
        tol = tol + 2.0 ** -8 * cnn.conv_forward_points(np.abs(xin).astype(np.float64), np.abs(w),
                                                        np.zeros(cout), mode, pts)
    assert np.all(err <= tol), (err.max(), np.abs(ref).max())
