"""CPU pins of the format-faithful network reference (oracle/unet.py forward_formats,
backward_formats), used for the element-wise GPU comparison:
- its BF16 rounding equals torch's float32 -> bfloat16 conversion (round to nearest even);
- with the identity as rounding it is exactly the FP64 network and its gradients;
- with BF16 it stays within a few BF16 units of the exact network's scale, while a
  network with one weight tap moved to its neighbour is far outside that."""
import numpy as np
import pytest

from oracle import unet as U

torch = pytest.importorskip("torch")


def test_bf16_rounding_is_round_to_nearest_even():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(4096) * 10.0 ** rng.integers(-20, 20, 4096),
                        [0.0, -0.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 3.0e38]])
    ref = torch.as_tensor(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16(a), ref)


def _net(base=8, levels=3, B=2, H=16, W=16, seed=1):
    shapes = U.layer_shapes(base=base, levels=levels)
    rng = np.random.default_rng(seed)
    params = U.init_params(shapes, seed=seed + 1)
    for name, _, _, co in shapes:
        params[name + ".b"] = 0.1 * rng.standard_normal(co)
    x = rng.standard_normal((B, H, W, 2))
    t = rng.standard_normal((B, H, W, 8))
    return params, x, t, levels


def test_identity_rounding_is_the_exact_network():
    params, x, t, levels = _net()
    y, acts, pw = U.forward_formats(params, x, levels, rnd=lambda v: v)
    yref, aref = U.forward(params, x, levels=levels, keep=True)
    assert np.array_equal(y, yref)
    gy = U.mse_loss(yref, t)[1]
    g = U.backward_formats(pw, acts, gy, levels, rnd=lambda v: v)
    gref = U.backward(params, aref, gy, levels=levels)
    for k in gref:
        assert np.allclose(g[k], gref[k], rtol=1e-12, atol=1e-15), k


def test_bf16_formats_stay_near_the_exact_network_and_a_moved_tap_does_not():
    params, x, t, levels = _net()
    y, acts, pw = U.forward_formats(params, x, levels)
    yref = U.forward(params, x, levels=levels)
    scale = np.abs(yref).max()
    assert np.abs(y - yref).max() <= 2.0 ** -4 * scale
    bad = {k: v.copy() for k, v in params.items()}
    w = bad["enc1_a.w"]
    w[1, 2], w[1, 1] = w[1, 1].copy(), w[1, 2].copy()
    ybad = U.forward(bad, x, levels=levels)
    assert np.abs(ybad - yref).max() > 2.0 ** -3 * scale
    assert np.mean(np.abs(ybad - y) > 2.0 ** -5 * scale) > 0.1
