"""Pins of the warm-start network's CPU reference (oracle/unet.py), CPU only:
convolution of a delta is the (flipped) kernel, bilinear upsampling reproduces linear
functions, translation equivariance by multiples of the coarsest cell, linearity, and
backward = finite differences of forward."""
import numpy as np

from oracle import unet


def test_conv_of_a_delta_is_the_kernel():
    rng = np.random.default_rng(0)
    w = rng.standard_normal((3, 3, 2, 3))
    x = np.zeros((1, 8, 8, 2))
    x[0, 4, 5, 1] = 1.0
    y = unet.conv(x, w, np.zeros(3))
    # out[y0, x0] picks in[y0+dy, x0+dx]: the delta at (4,5) lands at (4-dy, 5-dx)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            assert np.allclose(y[0, 4 - dy, 5 - dx], w[dy + 1, dx + 1, 1])
    assert np.count_nonzero(np.abs(y) > 0) == 9 * 3


def test_upsampling_is_bilinear():
    # coarse cell j is the centre of fine cells 2j, 2j+1 (position 2j + 1/2): sampling a
    # linear function there, the upsampled values are that function at the fine cells
    # (away from the periodic seam), and constants stay constant
    H = W = 8
    jy, jx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    f = lambda y, x: 0.3 + 1.7 * y - 0.9 * x + 0.2 * x * y  # bilinear
    c = f(2 * jy + 0.5, 2 * jx + 0.5)[None, :, :, None]
    u = unet.up(c)[0, :, :, 0]
    iy, ix = np.meshgrid(np.arange(2 * H), np.arange(2 * W), indexing="ij")
    inner = (iy >= 1) & (iy <= 2 * H - 2) & (ix >= 1) & (ix <= 2 * W - 2)
    assert np.allclose(u[inner], f(iy, ix)[inner], atol=1e-12)
    assert np.allclose(unet.up(np.full((1, 4, 4, 3), 2.5)), 2.5)
    # the backward is the transpose
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 4, 6, 3))
    y = rng.standard_normal((2, 8, 12, 3))
    assert np.isclose(np.sum(unet.up(x) * y), np.sum(x * unet.up_backward(y)), rtol=1e-13)


def test_network_is_linear_plus_bias_and_translation_equivariant():
    shapes = unet.layer_shapes(base=4)
    p = unet.init_params(shapes, seed=1)
    for k in p:
        if k.endswith(".b"):
            p[k] = np.random.default_rng(2).standard_normal(p[k].shape)
    rng = np.random.default_rng(3)
    x1, x2 = rng.standard_normal((2, 1, 16, 16, 2))
    y0 = unet.forward(p, np.zeros_like(x1))
    y1, y2 = unet.forward(p, x1), unet.forward(p, x2)
    y12 = unet.forward(p, 2 * x1 - 3 * x2)
    assert np.allclose(y12 - y0, 2 * (y1 - y0) - 3 * (y2 - y0), atol=1e-12)
    ys = unet.forward(p, np.roll(x1, (8, -8), axis=(1, 2)))
    assert np.allclose(ys, np.roll(y1, (8, -8), axis=(1, 2)), atol=1e-12)


def test_backward_matches_finite_differences():
    shapes = unet.layer_shapes(base=4)
    p = unet.init_params(shapes, seed=5)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((2, 16, 16, 2))
    t = rng.standard_normal((2, 16, 16, 8))
    y, acts = unet.forward(p, x, keep=True)
    L, gy = unet.mse_loss(y, t)
    grads = unet.backward(p, acts, gy)
    h = 1e-6
    for name in ("enc0_a.w", "enc3_b.w", "dec1_a.w", "dec0_b.b", "head.w", "enc2_a.b"):
        idx = tuple(rng.integers(0, s) for s in p[name].shape)
        old = p[name][idx]
        p[name][idx] = old + h
        Lp = unet.mse_loss(unet.forward(p, x), t)[0]
        p[name][idx] = old - h
        Lm = unet.mse_loss(unet.forward(p, x), t)[0]
        p[name][idx] = old
        fd = (Lp - Lm) / (2 * h)
        # central differences of a quadratic: only cancellation, ~ eps L / h
        assert abs(fd - grads[name][idx]) <= 1e-6 * abs(fd) + 1e-9 * max(L, 1.0), \
            (name, fd, grads[name][idx])
