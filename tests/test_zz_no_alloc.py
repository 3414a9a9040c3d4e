"""GPU test of lbm_objective_noalloc, the entry point for callers that cannot allocate
device memory (and so cannot create a handle, which allocates).

It is called through the C ABI on caller-owned device arrays and must return the same
objective as the handle's lbm_solid_objective, within the tolerance the other GPU tests
use for J (1e-12 relative), on two calls in a row: the second call reuses the fixed
device scratch that the first one left behind.  Cases: a periodic lattice and a small
elliptic plate, each with an observation mask and without one (on the plate the handle
then observes every active node, so the entry point is given the node mask as
weights).  Kept in a file that pytest collects last; it needs nothing from the other
test files and also runs on its own.
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
    J = torch.full((1,), 0.0, dtype=torch.float64, device="cuda")
    st = lib.lbm_objective_noalloc(nx, ny, dx, ptr(fS), ptr(F), ptr(dstar), ptr(obs), ptr(J),
                                   ctypes.c_void_p(stream.cuda_stream))
    assert st == 0
    stream.synchronize()
    return float(J.item())


def periodic_case(with_obs):
    nx, ny = 96, 70  # ragged against the 256-thread blocks
    F = I.fourier_force(nx, ny=ny, seed=21, kmax=3)
    dstar = np.random.default_rng(22).standard_normal((2, nx * ny)) * 1e-3
    obs = (np.random.default_rng(23).random(nx * ny) > 0.3).astype(float) if with_obs else None
    kw = dict(periodic=True, obs=obs)
    return nx, ny, 1.0 / nx, 0.5, 0.25, F, dstar, kw, obs


def plate_case(with_obs):
    geo = I.plate_geometry(20)
    dstar, sigma, F = I.plate_manufactured(geo.X, geo.Y)
    wd, wT = I.plate_wall_data(geo)
    act = geo.active.astype(float)
    obs = (np.random.default_rng(24).random(geo.nx * geo.nx) > 0.3) * act if with_obs else None
    kw = dict(periodic=False, node_mask=geo.active, link_bc=geo.link, wall_d=wd, wall_T=wT,
              wall_n=geo.normal, obs=obs)
    # the handle observes only active nodes: the entry point gets weights zero outside
    w = act if obs is None else obs
    return geo.nx, geo.nx, geo.dx, I.PLATE_E, I.PLATE_NU, F * geo.active, dstar, kw, w


@pytest.mark.parametrize("with_obs", [True, False])
@pytest.mark.parametrize("kind", ["periodic", "plate"])
def test_noalloc_objective_matches_the_handle_objective_twice(kind, with_obs):
    from paper_2609_31347_b300 import lbm
    assert torch.cuda.is_available()
    lib = lbm.load_library()
    stream = torch.cuda.current_stream()
    nx, ny, dx, E, nu, F, dstar, kw, w = (periodic_case if kind == "periodic"
                                          else plate_case)(with_obs)
    s = lbm.LBMSolid(nx, ny, dx, E, nu, control="force_field", **kw)
    s.set_target(dev(dstar))
    F_dev, d_dev = dev(F), dev(dstar)
    w_dev = None if w is None else dev(w)
    s.set_control(F_dev)
    results = []
    for steps in (17, 40):  # two calls in a row on different states
        s.primal_solve(steps, fixed_steps=True)
        J_ref = s.objective()
        fS = s.get_populations(0)
        J = noalloc_J(lib, nx, ny, dx, fS, F_dev, d_dev, w_dev, stream)
        assert abs(J - J_ref) <= J_TOL * abs(J_ref), (steps, J, J_ref)
        results.append(J)
    assert results[0] != results[1]
    # the same state twice gives the same value (scratch left by the last call is rewritten)
    assert noalloc_J(lib, nx, ny, dx, fS, F_dev, d_dev, w_dev, stream) == results[1]
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch_and_flags_a_zero_target():
    from paper_2609_31347_b300 import lbm
    lib = lbm.load_library()
    stream = torch.cuda.current_stream()
    big = torch.zeros(1, dtype=torch.float64, device="cuda")
    # (2^20 + 1) nodes exceed LBM_NOALLOC_MAX_NODES: rejected before any launch
    st = lib.lbm_objective_noalloc(1025, 1024, 1.0 / 1024, ptr(big), ptr(big), ptr(big), None,
                                   ptr(big), None)
    assert st == lbm.LBM_ERR_ARG
    st = lib.lbm_objective_noalloc(0, 8, 0.1, ptr(big), ptr(big), ptr(big), None, ptr(big), None)
    assert st == lbm.LBM_ERR_ARG
    # a target with zero weighted norm gives NaN
    nx = ny = 8
    fS = dev(np.random.default_rng(1).standard_normal(8 * nx * ny))
    z2 = dev(np.zeros(2 * nx * ny))
    assert np.isnan(noalloc_J(lib, nx, ny, 1.0 / nx, fS, z2, z2, None, stream))
