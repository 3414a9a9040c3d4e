"""GPU test of lbm_objective_noalloc, the entry point for callers that cannot allocate
device memory (and so cannot create a handle, which allocates).

It is called through the C ABI on caller-owned device arrays and must return the same
objective as the handle's lbm_solid_objective, within the tolerance the other GPU
tests use for J (1e-12 relative), on two calls in a row: the second call reuses the
fixed device scratch that the first one left behind.  Kept in a file that pytest
collects last; it needs nothing from the other test files and also runs on its own.
"""
import ctypes

import numpy as np
import pytest

from paper_2609_31347_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

J_TOL = 1e-12


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


def ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def noalloc_J(lib, nx, ny, dx, fS, F, dstar, obs, stream):
    J = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.lbm_objective_noalloc(nx, ny, dx, ptr(fS), ptr(F), ptr(dstar), ptr(obs), ptr(J),
                                   ctypes.c_void_p(stream.cuda_stream))
    assert st == 0
    stream.synchronize()
    return float(J.item())


def test_noalloc_objective_matches_the_handle_objective_twice():
    from paper_2609_31347_b300 import lbm
    assert torch.cuda.is_available()
    lib = lbm.load_library()
    stream = torch.cuda.current_stream()
    nx, ny = 96, 70  # ragged against the 256-thread blocks
    dx = 1.0 / nx
    F = I.fourier_force(nx, ny=ny, seed=21, kmax=3)
    dstar = np.random.default_rng(22).standard_normal((2, nx * ny)) * 1e-3
    obs = (np.random.default_rng(23).random(nx * ny) > 0.3).astype(float)
    s = lbm.LBMSolid(nx, ny, dx, 0.5, 0.25, periodic=True, control="force_field", obs=obs)
    s.set_target(dev(dstar))
    F_dev, d_dev, o_dev = dev(F), dev(dstar), dev(obs)
    s.set_control(F_dev)
    results = []
    for steps in (17, 40):  # two calls in a row on different states
        s.primal_solve(steps, fixed_steps=True)
        J_ref = s.objective()
        fS = s.get_populations(0)
        J = noalloc_J(lib, nx, ny, dx, fS, F_dev, d_dev, o_dev, stream)
        assert abs(J - J_ref) <= J_TOL * abs(J_ref), (steps, J, J_ref)
        results.append(J)
    assert results[0] != results[1]
    # the same state twice gives the same value (scratch left by the last call is rewritten)
    assert noalloc_J(lib, nx, ny, dx, fS, F_dev, d_dev, o_dev, stream) == results[1]
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_2609_31347_b300 import lbm
    lib = lbm.load_library()
    big = torch.zeros(1, dtype=torch.float64, device="cuda")
    # (2^20 + 1) nodes exceed LBM_NOALLOC_MAX_NODES: rejected before any launch
    st = lib.lbm_objective_noalloc(1025, 1024, 1.0 / 1024, ptr(big), ptr(big), ptr(big), None,
                                   ptr(big), None)
    assert st == lbm.LBM_ERR_ARG
    st = lib.lbm_objective_noalloc(0, 8, 0.1, ptr(big), ptr(big), ptr(big), None, ptr(big), None)
    assert st == lbm.LBM_ERR_ARG
