"""Encoder-solver U-Net reference (CPU, float64 numpy).

TEST INFRASTRUCTURE: see the package header for who may import this.

The architecture follows the caption of Fig. 1 and Sec. 3.4 (Eq. 3.13-3.14,
Eq. 4.1); the figure itself is not available, so the reading below fixes
what the caption leaves open.

Tensors are NHWC: ``[batch][ny][nx][channels]``.  A 3x3 convolution layer
has weights ``[cout][9][cin]`` (tap t = (dy+1)*3 + (dx+1)) and a bias
``[cout]``; outside the image the input is zero.  Three sampling modes:

* ``same``: output on the input grid, input node (y+dy, x+dx);
* ``down``: output on the half grid, output node (Y, X) reads input node
  (2Y+1+dy, 2X+1+dx) (coarse node centred on fine node (2Y+1, 2X+1), as in
  the multigrid transfers);
* ``up``: output on the double grid: nearest-neighbour upsampling
  u(y, x) = in(y // 2, x // 2) followed by a ``same`` convolution.

A ResNet layer is relu(x + conv2(relu(conv1(x)))).  Widths c_0..c_{L-1}
(16, 32, 64, 128), L levels.

Encoder (input: 3 channels [c_ref kappa, gamma, w h kappa]):
  level 0: in conv 3->c0 + relu, 2 ResNet layers              -> e_0
  level l: down conv c_{l-1}->c_l + relu, 2 ResNet layers      -> e_l
  up path: z_{L-1} = e_{L-1}; for l = L-2..0:
           up conv c_{l+1}->c_l + relu, concat [., e_l], conv 2c_l->c_l + relu,
           1 ResNet layer -> z_l
Solver (input: 3 channels [Re r^, Im r^, gamma], r^ = r / rms(r)):
  level 0: in conv 3->c0 + relu, concat [., z_0], conv 2c0->c0 + relu, ResNet -> s_0
  level l: down conv + relu, concat [., z_l], conv 2c_l->c_l + relu, ResNet -> s_l
  up path: t_{L-1} = s_{L-1}; for l = L-2..0:
           up conv + relu, concat [., s_l], conv 2c_l->c_l + relu, ResNet -> t_l
  out conv c0->2 (no activation): [Re, Im] of the error estimate
Preconditioner (Eq. 3.14 with the scaling that makes it 1-homogeneous):
  e_0 = h^2 rms(r) (out_re + i out_im)(r / rms(r)); the composition with the
  V-cycle is `training.mvu_compose`.
"""
from __future__ import annotations

import math

import numpy as np

C_REF = 1500.0   # m/s, reference velocity of the encoder's first input channel


# --------------------------------------------------------------------------
# layers
# --------------------------------------------------------------------------

def _src_index(n_in: int, n_out: int, mode: str, d: int):
    """For each output coordinate, the input coordinate of tap offset d and
    whether it lies inside the input."""
    o = np.arange(n_out)
    if mode == "same":
        i = o + d
        return np.clip(i, 0, n_in - 1), (i >= 0) & (i < n_in)
    if mode == "down":
        i = 2 * o + 1 + d
        return np.clip(i, 0, n_in - 1), (i >= 0) & (i < n_in)
    if mode == "up":
        u = o + d                      # coordinate on the upsampled grid (size 2 n_in)
        ok = (u >= 0) & (u < 2 * n_in)
        return np.where(ok, u // 2, 0), ok
    raise ValueError(mode)


def out_shape(ny: int, nx: int, mode: str):
    if mode == "same":
        return ny, nx
    if mode == "down":
        return ny // 2, nx // 2
    return 2 * ny, 2 * nx


def gather_taps(x, mode: str):
    """im2col: [B][ny'][nx'][9][cin] with the zero padding of the mode."""
    B, ny, nx, cin = x.shape
    my, mx = out_shape(ny, nx, mode)
    out = np.zeros((B, my, mx, 9, cin), dtype=x.dtype)
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        iy, oky = _src_index(ny, my, mode, dy)
        ix, okx = _src_index(nx, mx, mode, dx)
        blk = x[:, iy][:, :, ix]                       # [B][my][mx][cin]
        mask = (oky[:, None] & okx[None, :])[None, :, :, None]
        out[:, :, :, t, :] = np.where(mask, blk, 0.0)
    return out


def scatter_taps(g, in_shape, mode: str):
    """Adjoint of gather_taps: g [B][my][mx][9][cin] -> [B][ny][nx][cin]."""
    B, ny, nx, cin = in_shape
    my, mx = out_shape(ny, nx, mode)
    out = np.zeros(in_shape, dtype=g.dtype)
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        iy, oky = _src_index(ny, my, mode, dy)
        ix, okx = _src_index(nx, mx, mode, dx)
        mask = (oky[:, None] & okx[None, :])[None, :, :, None]
        contrib = np.where(mask, g[:, :, :, t, :], 0.0)
        for a in range(my):
            if not oky[a]:
                continue
            np.add.at(out[:, iy[a]], (slice(None), ix), contrib[:, a])
    return out


def conv_forward(x, w, b, mode: str):
    """y[n, Y, X, co] = b[co] + sum_{t, ci} w[co, t, ci] xt[n, Y, X, t, ci]."""
    cols = gather_taps(x, mode)
    return np.einsum("nyxtc,otc->nyxo", cols, w) + b


def conv_backward(x, w, gy, mode: str):
    """(dx, dw, db) of conv_forward for the upstream gradient gy."""
    cols = gather_taps(x, mode)
    dw = np.einsum("nyxtc,nyxo->otc", cols, gy)
    db = gy.sum(axis=(0, 1, 2))
    gcols = np.einsum("nyxo,otc->nyxtc", gy, w)
    dx = scatter_taps(gcols, x.shape, mode)
    return dx, dw, db


def _src_point(i: int, n_in: int, mode: str, d: int):
    """Input coordinate read by output coordinate i through tap offset d (None outside)."""
    if mode == "same":
        v = i + d
    elif mode == "down":
        v = 2 * i + 1 + d
    else:
        u = i + d
        return u // 2 if 0 <= u < 2 * n_in else None
    return v if 0 <= v < n_in else None


def conv_forward_points(x, w, b, mode: str, points):
    """y at the output nodes points = [(n, Y, X)], one by one from the definition
    y[n, Y, X, co] = b[co] + sum over taps t and input channels of w[co, t, ci] x[n, src_t(Y, X), ci]."""
    _, ny, nx, _ = x.shape
    out = np.zeros((len(points), w.shape[0]))
    for k, (n, Y, X) in enumerate(points):
        acc = np.array(b, dtype=np.float64)
        for t in range(9):
            iy, ix = _src_point(Y, ny, mode, t // 3 - 1), _src_point(X, nx, mode, t % 3 - 1)
            if iy is not None and ix is not None:
                acc = acc + w[:, t, :] @ x[n, iy, ix, :]
        out[k] = acc
    return out


def conv_input_grad_points(gy, w, in_shape, mode: str, points):
    """The input gradient of conv_forward at the input nodes points = [(n, y, x)]: the sum
    over every output node (Y, X) and tap t with src_t(Y, X) = (y, x) of w[:, t, :]^T gy[n, Y, X]."""
    _, ny, nx, _ = in_shape
    _, my, mx, _ = gy.shape
    out = np.zeros((len(points), w.shape[2]))
    for k, (n, y, x) in enumerate(points):
        acc = np.zeros(w.shape[2])
        for t in range(9):
            dy, dx = t // 3 - 1, t % 3 - 1
            Ys = [Y for Y in range(max(0, (y - 2) // 2 - 2), min(my, 2 * y + 4)) if _src_point(Y, ny, mode, dy) == y]
            Xs = [X for X in range(max(0, (x - 2) // 2 - 2), min(mx, 2 * x + 4)) if _src_point(X, nx, mode, dx) == x]
            for Y in Ys:
                for X in Xs:
                    acc = acc + w[:, t, :].T @ gy[n, Y, X, :]
        out[k] = acc
    return out


def conv_weight_grad(x, gy, mode: str):
    """(dw, db) of conv_forward, tap by tap: dw[co, t, ci] = sum over output nodes p of
    gy[p, co] x[src_t(p), ci] (zero outside the input), db = sum over p of gy[p]."""
    B, ny, nx, cin = x.shape
    _, my, mx, cout = gy.shape
    dw = np.zeros((cout, 9, cin))
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        iy, oky = _src_index(ny, my, mode, dy)
        ix, okx = _src_index(nx, mx, mode, dx)
        xt = x[:, iy][:, :, ix] * (oky[:, None] & okx[None, :])[None, :, :, None]
        dw[:, t, :] = np.tensordot(gy, xt, axes=([0, 1, 2], [0, 1, 2]))
    return dw, gy.sum(axis=(0, 1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64: the
    8-bit-exponent, 8-bit-significand format, i.e. float32 with the low 16 bits
    rounded away."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


# --------------------------------------------------------------------------
# network description (layer order = parameter order)
# --------------------------------------------------------------------------

def layer_specs(widths=(16, 32, 64, 128), in_enc: int = 3, in_sol: int = 3, out_ch: int = 2):
    """[(name, cin, cout, mode)] for the encoder then the solver."""
    L = len(widths)
    c = list(widths)
    specs = []

    def res(prefix, ch):
        specs.append((prefix + ".a", ch, ch, "same"))
        specs.append((prefix + ".b", ch, ch, "same"))

    # encoder
    specs.append(("enc.in", in_enc, c[0], "same"))
    res("enc.r0.0", c[0])
    res("enc.r0.1", c[0])
    for l in range(1, L):
        specs.append((f"enc.down{l}", c[l - 1], c[l], "down"))
        res(f"enc.r{l}.0", c[l])
        res(f"enc.r{l}.1", c[l])
    for l in range(L - 2, -1, -1):
        specs.append((f"enc.up{l}", c[l + 1], c[l], "up"))
        specs.append((f"enc.cat{l}", 2 * c[l], c[l], "same"))
        res(f"enc.ru{l}", c[l])
    # solver
    specs.append(("sol.in", in_sol, c[0], "same"))
    specs.append(("sol.cat0", 2 * c[0], c[0], "same"))
    res("sol.r0", c[0])
    for l in range(1, L):
        specs.append((f"sol.down{l}", c[l - 1], c[l], "down"))
        specs.append((f"sol.cat{l}", 2 * c[l], c[l], "same"))
        res(f"sol.r{l}", c[l])
    for l in range(L - 2, -1, -1):
        specs.append((f"sol.up{l}", c[l + 1], c[l], "up"))
        specs.append((f"sol.ucat{l}", 2 * c[l], c[l], "same"))
        res(f"sol.ru{l}", c[l])
    specs.append(("sol.out", c[0], out_ch, "same"))
    return specs


def n_params(specs) -> int:
    return sum(co * 9 * ci + co for _, ci, co, _ in specs)


def unflatten(flat, specs):
    """{name: (w [cout][9][cin], b [cout])} from the flat parameter vector
    (per layer: weights then bias, in layer order)."""
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, ci, co, _ in specs:
        nw = co * 9 * ci
        out[name] = (flat[o:o + nw].reshape(co, 9, ci), flat[o + nw:o + nw + co])
        o += nw + co
    assert o == flat.size
    return out


def flatten_grads(grads, specs):
    parts = []
    for name, _, _, _ in specs:
        dw, db = grads[name]
        parts += [dw.ravel(), db.ravel()]
    return np.concatenate(parts)


# --------------------------------------------------------------------------
# forward with a tape, backward
# --------------------------------------------------------------------------

class Tape:
    def __init__(self, quantize=None):
        self.ops = []
        self.q = quantize if quantize is not None else (lambda a: a)


def _conv(tape, P, specs_by_name, name, x, act: bool):
    w, b = P[name]
    mode = specs_by_name[name][3]
    y = conv_forward(x, w, b, mode)
    out = relu(y) if act else y
    if name != "sol.out":
        out = tape.q(out)
    tape.ops.append(("conv", name, x, out, act, mode))
    return out


def _res(tape, P, sbn, prefix, x):
    h = _conv(tape, P, sbn, prefix + ".a", x, True)
    y = conv_forward(h, *P[prefix + ".b"], "same")
    out = tape.q(relu(x + y))
    tape.ops.append(("res", prefix, x, h, out))
    return out


def _cat(tape, a, b):
    out = np.concatenate([a, b], axis=-1)
    tape.ops.append(("cat", a, b, out))
    return out


def encoder_forward(P, specs, x, tape=None):
    """Context features [z_0..z_{L-1}] (Eq. 3.13)."""
    tape = tape if tape is not None else Tape()
    sbn = {s[0]: s for s in specs}
    L = sum(1 for s in specs if s[0].startswith("enc.down")) + 1
    e = []
    h = _conv(tape, P, sbn, "enc.in", x, True)
    h = _res(tape, P, sbn, "enc.r0.0", h)
    h = _res(tape, P, sbn, "enc.r0.1", h)
    e.append(h)
    for l in range(1, L):
        h = _conv(tape, P, sbn, f"enc.down{l}", h, True)
        h = _res(tape, P, sbn, f"enc.r{l}.0", h)
        h = _res(tape, P, sbn, f"enc.r{l}.1", h)
        e.append(h)
    z = [None] * L
    z[L - 1] = e[L - 1]
    t = e[L - 1]
    for l in range(L - 2, -1, -1):
        u = _conv(tape, P, sbn, f"enc.up{l}", t, True)
        t = _conv(tape, P, sbn, f"enc.cat{l}", _cat(tape, u, e[l]), True)
        t = _res(tape, P, sbn, f"enc.ru{l}", t)
        z[l] = t
    return z, tape


def solver_forward(P, specs, x, z, tape=None):
    """Network output [B][ny][nx][2] for input x [B][ny][nx][3] and context z."""
    tape = tape if tape is not None else Tape()
    sbn = {s[0]: s for s in specs}
    L = len(z)
    s = []
    h = _conv(tape, P, sbn, "sol.in", x, True)
    h = _conv(tape, P, sbn, "sol.cat0", _cat(tape, h, z[0]), True)
    h = _res(tape, P, sbn, "sol.r0", h)
    s.append(h)
    for l in range(1, L):
        h = _conv(tape, P, sbn, f"sol.down{l}", h, True)
        h = _conv(tape, P, sbn, f"sol.cat{l}", _cat(tape, h, z[l]), True)
        h = _res(tape, P, sbn, f"sol.r{l}", h)
        s.append(h)
    t = s[L - 1]
    for l in range(L - 2, -1, -1):
        u = _conv(tape, P, sbn, f"sol.up{l}", t, True)
        t = _conv(tape, P, sbn, f"sol.ucat{l}", _cat(tape, u, s[l]), True)
        t = _res(tape, P, sbn, f"sol.ru{l}", t)
    out = _conv(tape, P, sbn, "sol.out", t, False)
    return out, tape


def network_forward(P, specs, enc_in, sol_in, quantize=None):
    """Encoder then solver on one tape; the batch of solver inputs shares the
    context features of one encoder input (Eq. 4.1).  ``quantize`` (e.g.
    bf16_round) is applied to every stored activation, as a BF16 network
    stores them; the output layer stays unrounded."""
    tape = Tape(quantize)
    z, _ = encoder_forward(P, specs, enc_in, tape)
    zb = []
    for zz in z:
        v = np.broadcast_to(zz, (sol_in.shape[0],) + zz.shape[1:])
        tape.ops.append(("bcast", zz, v))
        zb.append(v)
    out, _ = solver_forward(P, specs, sol_in, zb, tape)
    return out, tape


def backward(P, specs, tape, g_out, wrt=None, grad_quantize=None):
    """Reverse pass over the tape for the upstream gradient g_out of the last
    output.  Returns {name: (dw, db)} and, if ``wrt`` is given, the gradient
    with respect to that tape input.  An array used by several consumers
    (skip connections, context features) sums their gradients.
    ``grad_quantize`` (e.g. bf16_round) is applied to the (masked) output gradient
    of every convolution before its weight and input gradients are formed, as a
    BF16 network does with its gradient operand; the gradient handed on through a
    skip connection is not rounded."""
    qg = grad_quantize if grad_quantize is not None else (lambda a: a)
    grads = {name: (np.zeros_like(P[name][0]), np.zeros_like(P[name][1])) for name, *_ in specs}
    acc = {}

    def add(arr, g):
        k = id(arr)
        acc[k] = (arr, acc[k][1] + g) if k in acc else (arr, g)

    def take(arr):
        k = id(arr)
        return acc.pop(k)[1] if k in acc else None

    add(tape.ops[-1][3], g_out)
    for op in reversed(tape.ops):
        kind = op[0]
        if kind == "conv":
            _, name, x, out, act, mode = op
            g = take(out)
            if g is None:
                continue
            if act:
                g = g * (out > 0)
            dx, dw, db = conv_backward(x, P[name][0], qg(g), mode)
            gw, gb = grads[name]
            grads[name] = (gw + dw, gb + db)
            add(x, dx)
        elif kind == "res":
            _, prefix, x, h, out = op
            g = take(out)
            if g is None:
                continue
            g = g * (out > 0)
            dh, dw, db = conv_backward(h, P[prefix + ".b"][0], qg(g), "same")
            gw, gb = grads[prefix + ".b"]
            grads[prefix + ".b"] = (gw + dw, gb + db)
            add(x, g)
            add(h, dh)
        elif kind == "cat":
            _, a, b, out = op
            g = take(out)
            if g is None:
                continue
            ca = a.shape[-1]
            add(a, g[..., :ca])
            add(b, g[..., ca:])
        elif kind == "bcast":
            _, z, v = op
            g = take(v)
            if g is not None:
                add(z, g.sum(axis=0, keepdims=True))
    gx = take(wrt) if wrt is not None else None
    return grads, gx


def mse(e_net, e_true):
    """Eq. 4.2 for one batch: (1/m) sum_i ||e_net_i - e_true_i||^2 (m = batch size)."""
    d = np.asarray(e_net, dtype=np.float64) - np.asarray(e_true, dtype=np.float64)
    m = d.shape[0]
    return float(np.sum(d * d) / m), 2.0 * d / m


def adam_step(theta, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """Kingma & Ba (2015), Algorithm 1, one step (t >= 1)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


# --------------------------------------------------------------------------
# the network as a preconditioner (Eq. 3.14, 4.1)
# --------------------------------------------------------------------------

def encoder_input(kappa, gamma, omega: float, h: float):
    """[1][ny][nx][3]: c_ref kappa, gamma, w h kappa."""
    k = np.asarray(kappa, dtype=np.float64)
    g = np.asarray(gamma, dtype=np.float64)
    return np.stack([C_REF * k, g, omega * h * k], axis=-1)[None]


def solver_input(r, gamma):
    """([B][ny][nx][3], rms per RHS): [Re, Im] of r / rms(r) and gamma."""
    r = np.asarray(r, dtype=np.complex128)
    if r.ndim == 2:
        r = r[None]
    rms = np.sqrt(np.mean(np.abs(r) ** 2, axis=(1, 2)))
    safe = np.where(rms > 0, rms, 1.0)
    rn = r / safe[:, None, None]
    g = np.broadcast_to(np.asarray(gamma, dtype=np.float64), rn.shape[1:])
    x = np.stack([rn.real, rn.imag, np.broadcast_to(g, rn.shape)], axis=-1)
    return x, rms


def solver_output_to_error(out, rms, h: float):
    """e_0 = h^2 rms(r) (out_re + i out_im)."""
    return (h * h) * rms[:, None, None] * (out[..., 0] + 1j * out[..., 1])


def he_init(specs, seed: int):
    """Seeded He-normal weights, zero biases, flat (an input, not the method)."""
    g = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for _, ci, co, _ in specs:
        std = math.sqrt(2.0 / (9 * ci))
        parts += [g.normal(0.0, std, size=co * 9 * ci), np.zeros(co)]
    return np.concatenate(parts)
