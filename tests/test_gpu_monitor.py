"""GPU parity of the convergence monitor and the paper's stopping rule (Eqs. convergence,
convergence_crit) against the oracle, through the C ABI.

The solve loop samples c once per chunk of check_every sweeps: the chunk that ends after
s sweeps contributes c of the state its last sweep collided, f_S(s - 1) (adjoint:
phi_S(s - 1)); the first chunk is skipped while s < 2.  The oracle's traces give c of
every state of the plain iteration, and its CV rule decides at which sample the solve
must stop.  Checked: every GPU sample equals the oracle's to 1e-12 relative, and the GPU
stops after the same number of sweeps, for both kernel variants, periodic and plate.
Tolerances are chosen so that the CV at the stopping sample is clearly below and the one
before it clearly above the threshold.
"""
import numpy as np
import pytest

import oracle
from paper_2609_31347_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLE_TOL = 1e-12


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


@pytest.fixture(scope="module")
def lbm_mod():
    from paper_2609_31347_b300 import lbm
    assert torch.cuda.is_available()
    lbm.load_library()
    return lbm


def expected_samples(trace, check_every, max_steps):
    """(sweep counts s, samples) of the solve loop from an oracle trace."""
    s_list, c_list = [], []
    s = 0
    while s < max_steps:
        s += min(check_every, max_steps - s)
        if s >= 2:
            s_list.append(s)
            c_list.append(trace[s - 1])
    return np.array(s_list), np.array(c_list)


def stop_point(samples, window, tol):
    i, cv = oracle.cv_stop(samples, window, tol)
    assert i >= window, "tolerance reached too early for a meaningful test"
    _, cv_prev = oracle.cv_stop(samples[:i], window, tol)
    assert cv < tol * (1 - 1e-6) and cv_prev > tol * (1 + 1e-6), (cv, cv_prev)
    return i


def periodic_case(nx):
    # a smooth target: a random one excites the wavevectors (N/2, 0), (0, N/2), where the
    # adjoint step has the eigenvalue -1 and c never settles
    F = I.fourier_force(nx, seed=nx, kmax=2)
    dstar = I.fourier_force(nx, seed=nx + 1, kmax=3) * 1e-3
    return oracle.Grid(nx, nx, 1.0 / nx, 0.3), F, dstar, 0.8, None


def plate_case(Nx):
    geo = I.plate_geometry(Nx)
    dstar, sigma, F = I.plate_manufactured(geo.X, geo.Y)
    wd, wT = I.plate_wall_data(geo)
    g = oracle.Grid(geo.nx, geo.nx, geo.dx, I.PLATE_NU, periodic=False,
                    node_type=geo.node_type, link=geo.link, wall_d=wd, wall_T=wT,
                    wall_n=geo.normal)
    extra = dict(periodic=False, node_mask=geo.active, link_bc=geo.link, wall_d=wd,
                 wall_T=wT, wall_n=geo.normal, obs=geo.active.astype(float))
    return g, F * geo.active, dstar, I.PLATE_E, extra


# 16^2 and 32^2 run cluster launches through L2, 48^2 the lattice held in distributed
# shared memory, the plate graph-replayed compact launches
CASES = [("periodic", 16, 16, 30, 1e-6), ("periodic", 32, 64, 30, 1e-6),
         ("periodic", 48, 64, 30, 1e-6), ("plate", 10, 16, 25, 1e-4)]


def make(lbm_mod, g, E, extra, kernel):
    kw = extra or {}
    return lbm_mod.LBMSolid(g.nx, g.ny, g.dx, E, g.nu, kernel=kernel, **kw)


@pytest.mark.parametrize("kernel", ["fp64", "auto"])
@pytest.mark.parametrize("kind,n,check_every,window,tol", CASES)
def test_primal_cv_rule_matches_the_oracle(lbm_mod, kind, n, check_every, window, tol, kernel):
    g, F, dstar, E, extra = periodic_case(n) if kind == "periodic" else plate_case(n)
    max_steps = 400 * n * n // 8 + 4000
    trace = oracle.primal_trace(g, E, F, max_steps)
    s_all, c_all = expected_samples(trace, check_every, max_steps)
    i = stop_point(c_all, window, tol)
    s = make(lbm_mod, g, E, extra, kernel)
    s.set_control(dev(F))
    info = s.primal_solve(max_steps, tol=tol, criterion=0, window=window,
                          check_every=check_every)
    got = s.monitor_samples()
    assert info.status == lbm_mod.LBM_OK
    assert info.steps == s_all[i], (info.steps, s_all[i])
    assert got.size == i + 1
    assert np.all(np.abs(got - c_all[: i + 1]) <= SAMPLE_TOL * np.abs(c_all[: i + 1]))
    s.close()


@pytest.mark.parametrize("kernel", ["fp64", "auto"])
@pytest.mark.parametrize("kind,n,check_every,window,tol", CASES)
def test_adjoint_cv_rule_matches_the_oracle(lbm_mod, kind, n, check_every, window, tol, kernel):
    g, F, dstar, E, extra = periodic_case(n) if kind == "periodic" else plate_case(n)
    obs = None if extra is None else extra["obs"]
    fS = oracle.primal(g, E, F, 3 * n * n)
    max_steps = 400 * n * n // 8 + 4000
    trace = oracle.adjoint_trace(g, E, F, fS, dstar, max_steps, obs=obs)
    s_all, c_all = expected_samples(trace, check_every, max_steps)
    i = stop_point(c_all, window, tol)
    s = make(lbm_mod, g, E, extra, kernel)
    s.set_target(dev(dstar))
    s.set_control(dev(F))
    s.set_populations(0, dev(fS))
    info = s.adjoint_solve(max_steps, tol=tol, criterion=0, window=window,
                           check_every=check_every)
    got = s.monitor_samples()
    assert info.status == lbm_mod.LBM_OK
    assert info.steps == s_all[i], (info.steps, s_all[i])
    assert got.size == i + 1
    assert np.all(np.abs(got - c_all[: i + 1]) <= SAMPLE_TOL * np.abs(c_all[: i + 1]))
    s.close()
