"""GPU forward-mode (f-AD) tangent solve against the GPU adjoint gradient and the oracle's
dual-number f-AD: the paper's two gradient methods (Sections 3.3.1 and 3.3.2) must agree
(Section 4.2.3 reports >= 11 significant digits between f-AD and ALBM)."""
import numpy as np
import pytest

import oracle
from paper_2609_31347_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


@pytest.fixture(scope="module")
def lbm():
    from paper_2609_31347_b300 import lbm as m
    assert torch.cuda.is_available()
    m.load_library()
    return m


def test_benchmark1_tangent_equals_adjoint_and_oracle_fad(lbm):
    nx = 20
    m = I.periodic_manufactured(nx)
    basis = I.paper_scale_basis(m["Fstar"])
    s = lbm.LBMSolid(nx, nx, m["dx"], I.PAPER_E, I.PAPER_NU, control="force_basis2",
                     force_basis=basis.reshape(-1))
    s.set_target(dev(m["dstar"]))
    s.set_control(dev([-1.0, -1.0]))
    s.primal_solve(2_000_000, tol=1e-14, criterion=1, check_every=64)
    s.adjoint_solve(2_000_000, tol=1e-14, criterion=1, check_every=64)
    g = s.gradient().cpu().numpy()
    t = np.array([s.tangent(dev(e), tol=1e-14) for e in ([1.0, 0.0], [0.0, 1.0])])
    assert np.all(np.abs(t - g) <= 1e-11 * np.abs(g)), (t, g)
    g_ = oracle.Grid(nx, nx, m["dx"], I.PAPER_NU)
    F = -m["Fstar"]
    steps = 30 * nx * nx
    for i in range(2):
        fSv, fSd = oracle.primal_tangent(g_, I.PAPER_E, F, steps, Fdot=basis[i])
        _, Jd = oracle.objective_tangent(g_, fSv, fSd, F, m["dstar"], Fdot=basis[i])
        assert abs(t[i] - Jd) <= 1e-10 * abs(Jd)
    s.close()


def test_force_field_tangent_along_a_random_direction(lbm):
    nx = 40
    c = I.config_amplitudes(nx)
    s = lbm.LBMSolid(nx, nx, c["dx"], c["E"], c["nu"])
    s.set_target(dev(c["dstar"]))
    s.set_control(dev(0.3 * np.tensordot([1.0, 0.5], c["basis"], axes=1)))
    s.primal_solve(2_000_000, tol=1e-14, criterion=1, check_every=64)
    s.adjoint_solve(2_000_000, tol=1e-14, criterion=1, check_every=64)
    g = s.gradient().cpu().numpy()
    v = I.fourier_force(nx, seed=9, kmax=3).ravel()  # zero-mean direction
    dJ = s.tangent(dev(v))
    assert abs(dJ - g @ v) <= 1e-11 * np.abs(g).max() * np.abs(v).sum()
    s.close()


def test_plate_young_tangent(lbm):
    Nx = 16
    geo = I.plate_geometry(Nx)
    dstar, sigma, F = I.plate_manufactured(geo.X, geo.Y)
    wd, wT = I.plate_wall_data(geo)
    F = F * geo.active
    s = lbm.LBMSolid(geo.nx, geo.nx, geo.dx, I.PLATE_E, I.PLATE_NU, periodic=False,
                     node_mask=geo.active, link_bc=geo.link, wall_d=wd, wall_T=wT,
                     wall_n=geo.normal, obs=geo.active.astype(float), control="young_scalar",
                     force=F)
    s.set_target(dev(dstar))
    a = np.sqrt(0.15)
    s.set_control(dev([a]))
    s.primal_solve(2_000_000, tol=1e-14, criterion=1, check_every=64)
    s.adjoint_solve(2_000_000, tol=1e-14, criterion=1, check_every=64)
    g = float(s.gradient()[0])
    t = s.tangent(dev([1.0]), tol=1e-14)
    assert abs(t - g) <= 1e-10 * abs(g), (t, g)
    go = oracle.Grid(geo.nx, geo.nx, geo.dx, I.PLATE_NU, periodic=False, node_type=geo.node_type,
                     link=geo.link, wall_d=wd, wall_T=wT, wall_n=geo.normal)
    steps = 40000
    fSv, fSd = oracle.primal_tangent(go, 0.15, F, steps, Edot=1.0)
    _, Jd = oracle.objective_tangent(go, fSv, fSd, F, dstar, obs=geo.active.astype(float))
    assert abs(t - 2 * a * Jd) <= 1e-9 * abs(2 * a * Jd)
    s.close()
