"""Oracle pins for the discrete adjoint and the gradient (Section 3.3), CPU only.

- adjoint dot-product identity <P x, y> = <x, P^T y> for the step operator, periodic
  and bounded (the adjoint streaming and collision are the exact transpose);
- f-AD tangents equal central differences (J and the state are smooth in the control);
- ALBM gradients equal f-AD gradients to >= 11 significant digits once both are
  converged (Section 4.2.3 reports >= 11 digits between the two methods);
- the distributed-control gradient equals central differences node-wise, and the
  one-sided FDQ of Eq. (FDQ_grad) differs from it by (h/2) d2J/dF2 (J is quadratic in
  a force control);
- at F = -F* the gradient vanishes on the diagonal at s = 1/4, 1/2, 3/4
  (Section 4.2.5).
"""
import numpy as np
import pytest

import oracle
from oracle import fourier
from paper_2609_31347_b300 import inputs as I


def plate_grid(Nx, E=I.PLATE_E, nu=I.PLATE_NU):
    geo = I.plate_geometry(Nx)
    dstar, sigma, F = I.plate_manufactured(geo.X, geo.Y, E=E, nu=nu)
    wd, wT = I.plate_wall_data(geo, E=E, nu=nu)
    g = oracle.Grid(geo.nx, geo.nx, geo.dx, nu, periodic=False, node_type=geo.node_type,
                    link=geo.link, wall_d=wd, wall_T=wT, wall_n=geo.normal)
    return g, geo, dstar, F * geo.active


def test_dot_product_periodic():
    nx = 9
    g = oracle.Grid(nx, nx, 1.0 / nx, 0.8)
    x = I.random_state(nx * nx, 1)
    y = I.random_state(nx * nx, 2)
    Px = oracle.apply_step(g, 0.11, x)
    PTy = oracle.apply_step_transpose(g, 0.11, y)
    lhs, rhs = np.sum(Px * y), np.sum(x * PTy)
    assert abs(lhs - rhs) <= 1e-14 * np.sqrt(np.sum(Px ** 2) * np.sum(y ** 2))


@pytest.mark.parametrize("E", [I.PLATE_E, 1.0])
def test_dot_product_plate(E):
    g, geo, _, _ = plate_grid(20, E=E)
    act = geo.active.astype(float)
    x = I.random_state(g.N, 3) * act
    y = I.random_state(g.N, 4) * act
    Px = oracle.apply_step(g, E, x)
    PTy = oracle.apply_step_transpose(g, E, y)
    lhs, rhs = np.sum(Px * y), np.sum(x * PTy)
    assert abs(lhs - rhs) <= 1e-13 * np.sqrt(np.sum(Px ** 2) * np.sum(y ** 2))
    # inactive nodes stay zero in both directions
    assert np.all(Px[:, geo.active == 0] == 0) and np.all(PTy[:, geo.active == 0] == 0)


def test_fad_tangent_equals_central_difference():
    g, geo, dstar, F = plate_grid(12)
    steps = 300
    rng = np.random.default_rng(5)
    Fdot = rng.standard_normal(F.shape) * geo.active
    fS, fSd = oracle.primal_tangent(g, I.PLATE_E, F, steps, Edot=1.0, Fdot=Fdot)
    h = 1e-5
    fp = oracle.primal(g, I.PLATE_E + h, F + h * Fdot, steps)
    fm = oracle.primal(g, I.PLATE_E - h, F - h * Fdot, steps)
    fd = (fp - fm) / (2 * h)
    assert np.allclose(fS, oracle.primal(g, I.PLATE_E, F, steps), rtol=0, atol=0)
    assert np.abs(fd - fSd).max() <= 1e-6 * np.abs(fSd).max()


def _benchmark1(nx):
    m = I.periodic_manufactured(nx)
    g = oracle.Grid(nx, nx, m["dx"], I.PAPER_NU)
    return g, m


def test_albm_equals_fad_benchmark1():
    # Benchmark (1): F = alpha o F* with alpha = (-1, -1) (first step of Section 4.2.3).
    nx = 10
    g, m = _benchmark1(nx)
    basis = I.paper_scale_basis(m["Fstar"])
    alpha = np.array([-1.0, -1.0])
    F = np.tensordot(alpha, basis, axes=1)
    steps = 6000
    fS = oracle.primal(g, I.PAPER_E, F, steps)
    _, phiS = oracle.adjoint(g, I.PAPER_E, F, fS, m["dstar"], steps)
    gF = oracle.gradient_force(g, I.PAPER_E, F, fS, phiS, m["dstar"])
    g_albm = np.array([np.sum(basis[i] * gF) for i in range(2)])
    g_fad = []
    for i in range(2):
        fSv, fSd = oracle.primal_tangent(g, I.PAPER_E, F, steps, Fdot=basis[i])
        _, Jd = oracle.objective_tangent(g, fSv, fSd, F, m["dstar"], Fdot=basis[i])
        g_fad.append(Jd)
    g_fad = np.array(g_fad)
    assert np.all(np.abs(g_albm - g_fad) <= 1e-11 * np.abs(g_fad))


def test_albm_equals_fad_distributed_nodes():
    # Benchmark (2) gradient at a few nodes and both components: f-AD seeded on e_{n,i}.
    nx = 8
    g, m = _benchmark1(nx)
    F = -m["Fstar"]
    steps = 5000
    fS = oracle.primal(g, I.PAPER_E, F, steps)
    _, phiS = oracle.adjoint(g, I.PAPER_E, F, fS, m["dstar"], steps)
    gF = oracle.gradient_force(g, I.PAPER_E, F, fS, phiS, m["dstar"])
    for n, i in [(0, 0), (9, 1), (37, 0), (63, 1)]:
        seed = np.zeros_like(F)
        seed[i, n] = 1.0
        fSv, fSd = oracle.primal_tangent(g, I.PAPER_E, F, steps, Fdot=seed)
        _, Jd = oracle.objective_tangent(g, fSv, fSd, F, m["dstar"], Fdot=seed)
        assert abs(gF[i, n] - Jd) <= 1e-11 * np.abs(gF).max(), (n, i, gF[i, n], Jd)


def test_distributed_gradient_vs_finite_differences():
    # J is quadratic in the force control, so central differences are exact up to
    # cancellation; the one-sided FDQ of Eq. (FDQ_grad) is off by (h/2) d2J/dF_n^2.
    nx = 10
    g, m = _benchmark1(nx)
    F = -m["Fstar"]
    steps = 6000
    J0, _ = oracle.objective(g, oracle.primal(g, I.PAPER_E, F, steps), F, m["dstar"])
    fS = oracle.primal(g, I.PAPER_E, F, steps)
    _, phiS = oracle.adjoint(g, I.PAPER_E, F, fS, m["dstar"], steps)
    gF = oracle.gradient_force(g, I.PAPER_E, F, fS, phiS, m["dstar"])
    h = 1e-5

    def J_at(Fp):
        return oracle.objective(g, oracle.primal(g, I.PAPER_E, Fp, steps), Fp, m["dstar"])[0]

    gmax = np.abs(gF).max()
    second = {}
    nodes = [(0, int(np.abs(gF[0]).argmax())), (1, int(np.abs(gF[1]).argmax())), (0, 23), (1, 23)]
    for i, n in nodes:
        e = np.zeros_like(F)
        e[i, n] = 1.0
        Jp, Jm = J_at(F + h * e), J_at(F - h * e)
        central = (Jp - Jm) / (2 * h)
        # cancellation error ~ eps J / h ~ 1e-11 of the largest gradient
        assert abs(central - gF[i, n]) <= 1e-9 * gmax, (i, n, central, gF[i, n])
        second.setdefault(i, []).append((Jp - 2 * J0 + Jm) / h ** 2)
        fdq = (Jp - J0) / h
        assert abs(fdq - gF[i, n] - 0.5 * h * second[i][-1]) <= 1e-9 * gmax
    # translation invariance: d2J/dF_{n,i}^2 does not depend on the node
    for i in (0, 1):
        assert second[i][0] > 0
        assert abs(second[i][0] - second[i][1]) <= 1e-4 * second[i][0]


def test_gradient_zeros_on_the_diagonal():
    # Section 4.2.5: at F = -F* the ALBM gradient vanishes at s in {1/4, 1/2, 3/4}.
    nx = 20
    g, m = _benchmark1(nx)
    F = -m["Fstar"]
    fS = fourier.periodic_fixed_point(nx, I.PAPER_E, I.PAPER_NU, F)
    _, phiS = oracle.adjoint(g, I.PAPER_E, F, fS, m["dstar"], 30 * nx * nx)
    gF = oracle.gradient_force(g, I.PAPER_E, F, fS, phiS, m["dstar"])
    gmax = np.abs(gF).max()
    for s in (5, 10, 15):
        n = s * nx + s
        assert np.abs(gF[:, n]).max() <= 1e-10 * gmax
    assert np.abs(gF[:, 3 * nx + 3]).max() > 1e-3 * gmax


def test_plate_young_albm_equals_fad():
    # Benchmark (3) derivative dJ/dE through omega(E), gamma(E) and the E-dependent
    # Neumann rule, ALBM (with the streaming term of the Lagrangian) vs f-AD.
    g, geo, dstar, F = plate_grid(12)
    E = 0.15
    obs = geo.active.astype(float)
    steps = 20000
    fS = oracle.primal(g, E, F, steps)
    phiC, phiS = oracle.adjoint(g, E, F, fS, dstar, steps, obs=obs)
    gn, gtot = oracle.gradient_young(g, E, F, fS, phiS, phiC)
    fSv, fSd = oracle.primal_tangent(g, E, F, steps, Edot=1.0)
    _, Jd = oracle.objective_tangent(g, fSv, fSd, F, dstar, obs=obs)
    assert abs(gtot - Jd) <= 1e-10 * abs(Jd), (gtot, Jd)
    # per-node field: f-AD seeded on single nodes (interior and boundary)
    interior = np.where(geo.node_type == 1)[0]
    boundary = np.where(geo.node_type == 2)[0]
    for n in (interior[len(interior) // 2], boundary[0], boundary[len(boundary) // 3]):
        seed = np.zeros(g.N)
        seed[n] = 1.0
        fSv, fSd = oracle.primal_tangent(g, E, F, steps, Edot=seed)
        _, Jd = oracle.objective_tangent(g, fSv, fSd, F, dstar, obs=obs)
        assert abs(gn[n] - Jd) <= 1e-9 * max(abs(Jd), 1e-3 * abs(gn).max()), (n, gn[n], Jd)


def test_plate_force_gradient_albm_equals_fad():
    g, geo, dstar, F = plate_grid(12)
    obs = geo.active.astype(float)
    steps = 20000
    fS = oracle.primal(g, I.PLATE_E, F, steps)
    _, phiS = oracle.adjoint(g, I.PLATE_E, F, fS, dstar, steps, obs=obs)
    gF = oracle.gradient_force(g, I.PLATE_E, F, fS, phiS, dstar, obs=obs)
    bnd = np.where(geo.node_type == 2)[0]
    for n, i in [(bnd[0], 0), (bnd[len(bnd) // 2], 1), (np.where(geo.node_type == 1)[0][5], 0)]:
        seed = np.zeros_like(F)
        seed[i, n] = 1.0
        fSv, fSd = oracle.primal_tangent(g, I.PLATE_E, F, steps, Fdot=seed)
        _, Jd = oracle.objective_tangent(g, fSv, fSd, F, dstar, Fdot=seed, obs=obs)
        assert abs(gF[i, n] - Jd) <= 1e-9 * abs(Jd), (n, i)
