"""GPU part of the history starts (not in the paper): the vector arithmetic of
lbm_warm_combine and lbm_warm_dots against numpy, on a ragged length that spans several
grid strides, short lengths, in-place use, repeatability and argument errors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2609_31347_b300 import lbm
    assert torch.cuda.is_available()
    lbm.load_library()
    return lbm


@pytest.mark.parametrize("n", [1, 7, 1_000_003])
def test_combine_matches_numpy(L, n):
    rng = np.random.default_rng(n)
    V = rng.standard_normal((4, n))
    w = np.array([0.3, -1.7, 2.5, 1e-3])
    vs = [torch.as_tensor(v, device="cuda") for v in V]
    dst = torch.empty(n, dtype=torch.float64, device="cuda")
    for count in range(1, 5):
        L.warm_combine(w[:count], vs[:count], dst)
        ref = (w[:count, None] * V[:count]).sum(axis=0)
        scale = np.abs(w[:count, None] * V[:count]).sum(axis=0)
        assert np.all(np.abs(dst.cpu().numpy() - ref) <= 4e-16 * scale * count)
    # in place: the destination is the first source
    a = vs[0].clone()
    L.warm_combine([2.0, -1.0], [a, vs[1]], a)
    assert np.allclose(a.cpu().numpy(), 2 * V[0] - V[1], rtol=0, atol=1e-15 * 4)


@pytest.mark.parametrize("n", [1, 7, 1_000_003])
def test_dots_match_numpy_and_repeat(L, n):
    rng = np.random.default_rng(100 + n)
    V = rng.standard_normal((5, n))
    vs = [torch.as_tensor(v, device="cuda") for v in V]
    for m in range(1, 6):
        G = L.warm_dots(vs[:m])
        ref = V[:m] @ V[:m].T
        nrm = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
        assert G.shape == (m, m)
        assert np.all(np.abs(G - ref) <= 1e-13 * nrm + 1e-300)
        assert np.array_equal(G, G.T)
        assert np.array_equal(G, L.warm_dots(vs[:m]))  # fixed summation order


def test_history_calls_reject_bad_arguments(L):
    v = torch.zeros(16, dtype=torch.float64, device="cuda")
    for count in (5,):
        with pytest.raises(L.LBMError) as e:
            L.warm_combine([1.0] * count, [v] * count, v)
        assert e.value.status == L.LBM_ERR_ARG
    with pytest.raises(L.LBMError) as e:
        L.warm_dots([v] * 6)
    assert e.value.status == L.LBM_ERR_ARG
    with pytest.raises(ValueError):  # sizes differ
        L.warm_combine([1.0], [torch.zeros(8, dtype=torch.float64, device="cuda")], v)
