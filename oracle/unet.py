"""CPU reference of the warm-start network (FP64 numpy) -- TEST INFRASTRUCTURE ONLY.

The learned warm start maps a control field (the 2-component body force on a periodic
lattice) to the 8 steady post-streaming populations, which the LBM then iterates to the
requested residual.  The network is a 4-level U-Net:

  level l (l = 0..3) has C_l = base * 2^l channels and two 3x3 convolutions;
  encoder: conv(2 or C_{l-1} -> C_l), conv(C_l -> C_l), then 2x2 average pooling;
  decoder: bilinear 2x upsampling (periodic; each coarse value sits at the centre of its
           2x2 fine block, so fine cells take 3/4 of their own coarse cell and 1/4 of
           the neighbour on their side, per axis), concatenation [up, skip_l],
           conv(C_{l+1} + C_l -> C_l),
           conv(C_l -> C_l);
  head: 1x1 convolution C_0 -> 8.

All convolutions use circular padding (the lattice is periodic) and carry a bias; there
is no nonlinearity: the steady populations are a linear function of the force
(Section 3.1: the collision is affine in the populations and the force, streaming is a
permutation), so a linear multi-scale convolution operator is the right model class.

Tensors are (B, H, W, C) float64.  Weights of a 3x3 convolution are (3, 3, Cin, Cout)
indexed [dy+1, dx+1, ci, co] with out[b, y, x, co] = bias[co] +
sum_{dy,dx,ci} in[b, (y+dy) mod H, (x+dx) mod W, ci] w[dy+1, dx+1, ci, co].
"""
from __future__ import annotations

import numpy as np


def layer_shapes(base: int = 32, cin: int = 2, cout: int = 8, levels: int = 4):
    """[(name, kernel, cin, cout)] in execution order."""
    ch = [base * 2 ** l for l in range(levels)]
    shapes = []
    c = cin
    for l in range(levels):
        shapes.append(("enc%d_a" % l, 3, c, ch[l]))
        shapes.append(("enc%d_b" % l, 3, ch[l], ch[l]))
        c = ch[l]
    for l in range(levels - 2, -1, -1):
        shapes.append(("dec%d_a" % l, 3, ch[l + 1] + ch[l], ch[l]))
        shapes.append(("dec%d_b" % l, 3, ch[l], ch[l]))
    shapes.append(("head", 1, ch[0], cout))
    return shapes


def init_params(shapes, seed: int = 0):
    """He-style scaled normal weights (fan-in), zero biases."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, k, ci, co in shapes:
        params[name + ".w"] = rng.standard_normal((k, k, ci, co)) * np.sqrt(1.0 / (k * k * ci))
        params[name + ".b"] = np.zeros(co)
    return params


def conv(x, w, b):
    k = w.shape[0]
    out = np.zeros(x.shape[:3] + (w.shape[3],)) + b
    r = k // 2
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            xs = np.roll(x, shift=(-dy, -dx), axis=(1, 2))  # xs[y, x] = x[y+dy, x+dx]
            out += xs @ w[dy + r, dx + r]
    return out


def conv_backward(x, w, gout):
    """(grad_x, grad_w, grad_b) of conv for upstream gradient gout."""
    k = w.shape[0]
    r = k // 2
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            xs = np.roll(x, shift=(-dy, -dx), axis=(1, 2))
            gw[dy + r, dx + r] = np.einsum("bhwc,bhwd->cd", xs, gout)
            gx += np.roll(gout @ w[dy + r, dx + r].T, shift=(dy, dx), axis=(1, 2))
    gb = gout.sum(axis=(0, 1, 2))
    return gx, gw, gb


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) * 0.25


def _up_axis(x, axis):
    # linear 2x interpolation with the coarse value at the centre of its two fine cells
    # (fine 2j at -1/4, fine 2j+1 at +1/4 coarse cells from coarse j), periodic
    even = 0.75 * x + 0.25 * np.roll(x, 1, axis=axis)   # 3/4 x[j] + 1/4 x[j-1]
    odd = 0.75 * x + 0.25 * np.roll(x, -1, axis=axis)   # 3/4 x[j] + 1/4 x[j+1]
    out = np.stack([even, odd], axis=axis + 1)
    shape = list(x.shape)
    shape[axis] *= 2
    return out.reshape(shape)


def _up_axis_backward(g, axis):
    shape = list(g.shape)
    shape[axis] //= 2
    shape.insert(axis + 1, 2)
    gr = g.reshape(shape)
    ge = np.take(gr, 0, axis=axis + 1)
    go = np.take(gr, 1, axis=axis + 1)
    # transpose of _up_axis: x[j] feeds even[j], odd[j] (3/4), even[j+1], odd[j-1] (1/4)
    return 0.75 * (ge + go) + 0.25 * (np.roll(ge, -1, axis=axis) + np.roll(go, 1, axis=axis))


def up(x):
    """Bilinear 2x upsampling of (B, H, W, C), periodic."""
    return _up_axis(_up_axis(x, 1), 2)


def up_backward(g):
    return _up_axis_backward(_up_axis_backward(g, 2), 1)


def forward(params, x, levels: int = 4, keep: bool = False):
    """Network output (B, H, W, 8); with keep, also the activations for backward."""
    acts = {}
    skips = []
    h = x
    for l in range(levels):
        acts["enc%d_a" % l] = h
        h = conv(h, params["enc%d_a.w" % l], params["enc%d_a.b" % l])
        acts["enc%d_b" % l] = h
        h = conv(h, params["enc%d_b.w" % l], params["enc%d_b.b" % l])
        if l < levels - 1:
            skips.append(h)
            h = pool(h)
    for l in range(levels - 2, -1, -1):
        h = np.concatenate([up(h), skips[l]], axis=3)
        acts["dec%d_a" % l] = h
        h = conv(h, params["dec%d_a.w" % l], params["dec%d_a.b" % l])
        acts["dec%d_b" % l] = h
        h = conv(h, params["dec%d_b.w" % l], params["dec%d_b.b" % l])
    acts["head"] = h
    y = conv(h, params["head.w"], params["head.b"])
    return (y, acts) if keep else y


def backward(params, acts, gy, levels: int = 4):
    """Gradients of a scalar loss with upstream gradient gy w.r.t. every parameter."""
    grads = {}
    g, grads["head.w"], grads["head.b"] = conv_backward(acts["head"], params["head.w"], gy)
    skip_grads = {}
    for l in range(0, levels - 1):  # decoder in reverse execution order: level 0 first
        g, grads["dec%d_b.w" % l], grads["dec%d_b.b" % l] = conv_backward(
            acts["dec%d_b" % l], params["dec%d_b.w" % l], g)
        g, grads["dec%d_a.w" % l], grads["dec%d_a.b" % l] = conv_backward(
            acts["dec%d_a" % l], params["dec%d_a.w" % l], g)
        cu = params["dec%d_a.w" % l].shape[2] - params["dec%d_b.w" % l].shape[2]
        skip_grads[l] = g[..., cu:]
        g = up_backward(g[..., :cu])
    for l in range(levels - 1, -1, -1):
        if l < levels - 1:
            g = pool_backward(g) + skip_grads[l]
        g, grads["enc%d_b.w" % l], grads["enc%d_b.b" % l] = conv_backward(
            acts["enc%d_b" % l], params["enc%d_b.w" % l], g)
        g, grads["enc%d_a.w" % l], grads["enc%d_a.b" % l] = conv_backward(
            acts["enc%d_a" % l], params["enc%d_a.w" % l], g)
    return grads


def mse_loss(y, t):
    """0.5 * mean((y - t)^2) and its gradient."""
    d = y - t
    return 0.5 * float(np.mean(d * d)), d / d.size


# ---- the GPU's storage formats ------------------------------------------------------
# The GPU network keeps weights, activations and gradients in BF16 and accumulates in
# FP32.  The functions below run the same network with BF16 rounding applied exactly
# where the GPU stores a tensor: the packed input, every convolution output (bias
# included), every pooled and upsampled tensor, the output gradient and every input
# gradient; the head output is FP32 and the weights are used in BF16.  Sums are taken in
# FP64, so the GPU differs from these only by the order and width of its FP32 sums and
# by the roundings that such a difference flips; an element-wise comparison can then use
# a tolerance of a few BF16 units (2^-8) of each tensor's scale.


def bf16(a):
    """Round to the nearest BF16 value (ties to even), as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def forward_formats(params, x, levels: int = 4, rnd=bf16):
    """(y, acts, weights used) of the forward pass in the GPU's storage formats; rnd is
    the rounding of stored tensors (identity gives forward() exactly)."""
    pw = {k: (rnd(v) if k.endswith(".w") else v) for k, v in params.items()}
    acts, skips = {}, []
    h = rnd(x)
    for l in range(levels):
        for part in ("a", "b"):
            name = "enc%d_%s" % (l, part)
            acts[name] = h
            h = rnd(conv(h, pw[name + ".w"], pw[name + ".b"]))
        if l < levels - 1:
            skips.append(h)
            h = rnd(pool(h))
    for l in range(levels - 2, -1, -1):
        h = np.concatenate([rnd(up(h)), skips[l]], axis=3)
        for part in ("a", "b"):
            name = "dec%d_%s" % (l, part)
            acts[name] = h
            h = rnd(conv(h, pw[name + ".w"], pw[name + ".b"]))
    acts["head"] = h
    y = conv(h, pw["head.w"], pw["head.b"])
    if rnd is bf16:
        y = y.astype(np.float32).astype(np.float64)
    return y, acts, pw


def backward_formats(pw, acts, gy, levels: int = 4, rnd=bf16):
    """Parameter gradients in the GPU's storage formats for the upstream gradient gy
    (weights pw and activations acts from forward_formats)."""
    grads = {}

    def back(name, g):
        gx, grads[name + ".w"], grads[name + ".b"] = conv_backward(acts[name], pw[name + ".w"], g)
        return rnd(gx)

    g = back("head", rnd(gy))
    skip = {}
    for l in range(levels - 1):
        g = back("dec%d_b" % l, g)
        g = back("dec%d_a" % l, g)
        cu = pw["dec%d_a.w" % l].shape[2] - pw["dec%d_b.w" % l].shape[2]
        skip[l] = g[..., cu:]
        g = rnd(up_backward(g[..., :cu]))
    for l in range(levels - 1, -1, -1):
        if l < levels - 1:
            g = rnd(pool_backward(g) + skip[l])
        g = back("enc%d_b" % l, g)
        g = back("enc%d_a" % l, g)
    return grads
