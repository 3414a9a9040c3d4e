"""The error model of the default sweep arithmetic, measured (LBM_KERNEL_AUTO: bulk nodes
in 64-bit fixed point scaled to the node's largest input; LBM_KERNEL_FP64: every
operation in binary64).

States whose nodes mix populations of size 1 with populations of size 2^-40: the node
f = (1, s1, 1, s3, s4, s5, s6, s7) has m10 = b1 + b3 - b4 with b1 = f0 - f2 = 0, so the
diagonal outputs of the collision (Section 3.1; the bulk diagonal populations depend
only on m11 and the bared first moments) are of size 2^-40 while the axis outputs are of
size 1.  Documented model, checked element by element after one sweep:
  - fixed point: |f_auto - f_exact| <= 4 * 2^-56 * (largest input of the source node),
    so a value 2^-40 of its node's maximum keeps only about 16 significant bits;
  - binary64: relative error of a few units of 2^-53 on every value, small or large.
The strict variant is the reference for the small values: its diagonal outputs are
formed from the small inputs alone.  The oracle pins both on the large values.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


@pytest.fixture(scope="module")
def lbm_mod():
    from paper_2609_31347_b300 import lbm
    assert torch.cuda.is_available()
    lbm.load_library()
    return lbm


def test_small_populations_next_to_large_ones(lbm_mod):
    nx = ny = 16
    N = nx * ny
    E, nu = 0.7, 0.25
    rng = np.random.default_rng(3)
    fS = rng.uniform(0.5, 1.0, (8, N)) * 2.0 ** -40 * rng.choice([-1, 1], (8, N))
    fS[0] = fS[2] = 1.0  # b1 = 0: the large pair enters only the axis outputs
    out = {}
    for kernel in ("auto", "fp64"):
        s = lbm_mod.LBMSolid(nx, ny, 1.0 / nx, E, nu, kernel=kernel)
        s.set_control(dev(np.zeros(2 * N)))
        s.set_populations(0, dev(fS))
        s.primal_solve(1, fixed_steps=True)
        out[kernel] = s.get_populations(0).cpu().numpy().reshape(8, N)
        s.close()
    a, b = out["auto"], out["fp64"]
    g = oracle.Grid(nx, ny, 1.0 / nx, nu)
    ref = oracle.primal(g, E, np.zeros((2, N)), 1, fS0=fS)
    node_max = 1.0  # every source node's largest input
    small = np.abs(b) < 2.0 ** -30
    assert small[4:].all() and not small[:4].any()  # diagonal small, axis large
    # large values: both variants equal the oracle to binary64 rounding
    assert np.abs(a[:4] - ref[:4]).max() <= 4 * 2.0 ** -53
    assert np.abs(b[:4] - ref[:4]).max() <= 4 * 2.0 ** -53
    # the fixed-point model: absolute error relative to the node's largest input
    assert np.abs(a[4:] - b[4:]).max() <= 4 * 2.0 ** -56 * node_max
    rel_small = np.abs(a[small] - b[small]) / np.abs(b[small])
    # ... which leaves the small values with ~16 significant bits, as documented
    assert rel_small.max() <= 4 * 2.0 ** -56 / np.abs(b[small]).min()
    assert rel_small.max() > 1e-9
    print("fixed point: small values relative error up to %.2e (binary64 would be ~1e-16)"
          % rel_small.max())
