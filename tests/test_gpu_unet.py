"""GPU warm-start network (BF16 storage, FP32 accumulation on the tensor cores) against
the CPU references in oracle/unet.py: forward output, loss and every parameter gradient,
for the configured 4-level, 32-channel network and for smaller shapes; the
FP32-activation forward used for warm starts against the FP64 network with BF16-rounded
weights; and training by the library's own kernels lowers the loss.

Element-wise tolerances.  The BF16 path is compared with forward_formats /
backward_formats, which round to BF16 exactly where the GPU stores a tensor, so the two
differ only by the order and width of the FP32 sums and the BF16 roundings that this
flips: every element must lie within 2^-6 of the tensor's largest magnitude (a few BF16
units; a misplaced tap or a bad tile gives errors of order 1 at many elements).  The
exact-activation path is the linear map of the BF16 weights up to FP32 sums and the
split of each activation into two BF16 parts: every element within 1e-4 of the
output's largest magnitude.  The FP64 network without any rounding is also kept in
view: relative L2 distance below 2e-2 (outputs) and 5e-2 (gradients)."""
import numpy as np
import pytest

from oracle import unet as U

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_2609_31347_b300 import lbm as m
    assert torch.cuda.is_available()
    m.load_library()
    return m


def unflatten(p, shapes):
    out, o = {}, 0
    for name, k, ci, co in shapes:
        n = k * k * ci * co
        out[name + ".w"] = p[o:o + n].reshape(k, k, ci, co)
        o += n
        out[name + ".b"] = p[o:o + co]
        o += co
    assert o == p.size
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


ELEM_TOL = 2.0 ** -6  # of the tensor's largest magnitude, element by element


@pytest.mark.parametrize("base,levels,B,H,W", [(32, 4, 2, 128, 128), (16, 2, 3, 48, 32),
                                               (16, 1, 1, 16, 48), (16, 3, 2, 64, 64)])
def test_forward_and_gradients_match_cpu_reference(lbm, base, levels, B, H, W):
    net = lbm.UNet(B, H, W, base=base, levels=levels, seed=3)
    shapes = U.layer_shapes(base=base, levels=levels)
    assert net.nparams == sum(k * k * ci * co + co for _, k, ci, co in shapes)
    rng = np.random.default_rng(7)
    p = net.params(0).cpu().numpy().astype(np.float64)
    pr = unflatten(p.copy(), shapes)
    for name, _, _, co in shapes:  # nonzero biases so that the bias paths are exercised
        pr[name + ".b"][:] = 0.1 * rng.standard_normal(co)
    p = np.concatenate([np.concatenate([pr[n + ".w"].ravel(), pr[n + ".b"]]) for n, *_ in shapes])
    net.set_params(torch.as_tensor(p.astype(np.float32), device="cuda"))
    pr = unflatten(net.params(0).cpu().numpy().astype(np.float64), shapes)  # FP32-rounded
    x = rng.standard_normal((B, H, W, 2))
    t = rng.standard_normal((B, H, W, 8))
    xd = torch.as_tensor(x.astype(np.float32), device="cuda")
    td = torch.as_tensor(t.astype(np.float32), device="cuda")
    y = net.forward(xd).cpu().numpy().astype(np.float64)
    yref, acts = U.forward(pr, x, levels=levels, keep=True)
    yfmt, afmt, pw = U.forward_formats(pr, x.astype(np.float32).astype(np.float64),
                                       levels=levels)
    assert np.abs(y - yfmt).max() <= ELEM_TOL * np.abs(yfmt).max(), \
        np.abs(y - yfmt).max() / np.abs(yfmt).max()
    assert rel(y, yref) < 2e-2
    loss = float(net.train_step(xd, td, 0.0).item())
    Lref, gy = U.mse_loss(yref, t)
    assert abs(loss - Lref) <= 1e-2 * Lref
    Lfmt, gyf = U.mse_loss(yfmt, t)
    assert abs(loss - Lfmt) <= 1e-4 * Lfmt
    g = unflatten(net.params(1).cpu().numpy().astype(np.float64), shapes)
    gref = U.backward(pr, acts, gy, levels=levels)
    gfmt = U.backward_formats(pw, afmt, gyf, levels=levels)
    for name, *_ in shapes:
        for part in (".w", ".b"):
            k = name + part
            err = np.abs(g[k] - gfmt[k]).max() / np.abs(gfmt[k]).max()
            assert err <= ELEM_TOL, (k, err)
            e = rel(g[k], gref[k])
            assert e < 5e-2, (k, e)
    net.status()
    # lr = 0 leaves the parameters alone
    assert np.array_equal(net.params(0).cpu().numpy().astype(np.float64),
                          np.concatenate([np.concatenate([pr[n + ".w"].ravel(), pr[n + ".b"]])
                                          for n, *_ in shapes]))
    net.close()


@pytest.mark.parametrize("base,levels,B,H,W", [(32, 4, 1, 128, 128), (16, 2, 2, 32, 64)])
def test_exact_activation_forward_is_the_bf16_weight_network(lbm, base, levels, B, H, W):
    # FP32 activations with split-BF16 products: the map of the BF16-rounded weights up
    # to FP32 sums (relative error ~1e-5), against the FP64 reference with those weights
    net = lbm.UNet(B, H, W, base=base, levels=levels, seed=4)
    shapes = U.layer_shapes(base=base, levels=levels)
    rng = np.random.default_rng(9)
    p = net.params(0).cpu().numpy().astype(np.float64)
    pr = unflatten(p.copy(), shapes)
    for name, _, _, co in shapes:
        pr[name + ".b"][:] = 0.1 * rng.standard_normal(co)
    p = np.concatenate([np.concatenate([pr[n + ".w"].ravel(), pr[n + ".b"]]) for n, *_ in shapes])
    net.set_params(torch.as_tensor(p.astype(np.float32), device="cuda"))
    pr = unflatten(net.params(0).cpu().numpy().astype(np.float64), shapes)
    for n, *_ in shapes:
        pr[n + ".w"] = U.bf16(pr[n + ".w"])
    x = rng.standard_normal((B, H, W, 2)).astype(np.float32)
    y = net.forward(torch.as_tensor(x, device="cuda"), exact_acts=True).cpu().numpy()
    yref = U.forward(pr, x.astype(np.float64), levels=levels)
    net.status()
    err = np.abs(y - yref).max() / np.abs(yref).max()
    assert err <= 1e-4, err
    # BF16 activations are ~100x further off
    yb = net.forward(torch.as_tensor(x, device="cuda")).cpu().numpy()
    assert rel(yb, yref) > 10 * rel(y, yref)
    net.close()


def test_invalid_shapes_are_rejected(lbm):
    for kw in (dict(base=24), dict(levels=0), dict(levels=6), dict(base=128, levels=4)):
        with pytest.raises(lbm.LBMError) as e:
            lbm.UNet(1, 128, 128, **kw)
        assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LBMError):
        lbm.UNet(1, 128, 96, levels=4)  # W not a multiple of 16 * 2^3
    with pytest.raises(lbm.LBMError):
        lbm.UNet(1, 100, 128, levels=4)  # H not a multiple of 2^3


def test_training_lowers_the_loss(lbm):
    # a realisable target: another network of the same shape (the map is linear)
    B, H, W = 4, 64, 64
    teacher = lbm.UNet(B, H, W, base=16, levels=3, seed=11)
    student = lbm.UNet(B, H, W, base=16, levels=3, seed=12)
    rng = np.random.default_rng(0)
    X = torch.as_tensor(rng.standard_normal((8 * B, H, W, 2)).astype(np.float32), device="cuda")
    T = torch.empty((8 * B, H, W, 8), dtype=torch.float32, device="cuda")
    for j in range(8):
        teacher.forward(X[j * B:(j + 1) * B], T[j * B:(j + 1) * B])
    first = float(student.train_step(X[:B], T[:B], 0.0).item())
    for it in range(300):
        j = it % 8
        student.train_step(X[j * B:(j + 1) * B], T[j * B:(j + 1) * B], 2e-3)
    last = float(student.train_step(X[:B], T[:B], 0.0).item())
    assert last < 0.05 * first, (first, last)
    teacher.close()
    student.close()
