"""GPU tests of the gradient-based optimisation layer (autograd function + L-BFGS with
strong-Wolfe line search, Algorithm 2) on the paper's benchmarks.

The reference optima come from the oracle's exact periodic fixed point: the steady
displacement is linear in a force control, so J is quadratic and its minimiser solves a
small normal system built from the steady responses to the control's basis fields.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import fourier
from paper_2609_31347_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


@pytest.fixture(scope="module")
def mods():
    from paper_2609_31347_b300 import gbo, lbm
    assert torch.cuda.is_available()
    lbm.load_library()
    return lbm, gbo


def exact_fit(nx, E, nu, basis, dstar):
    """alpha minimising J over F = sum_i alpha_i Phi_i (normal equations, exact steady
    states from the per-wavevector fixed point)."""
    dx = 1.0 / nx
    D = [fourier.displacement(fourier.periodic_fixed_point(nx, E, nu, b), b, dx).ravel()
         for b in basis]
    D = np.array(D)
    return np.linalg.solve(D @ D.T, D @ dstar.ravel())


def test_autograd_gradient_is_the_adjoint_gradient(mods):
    lbm, gbo = mods
    nx = 16
    m = I.periodic_manufactured(nx)
    basis = I.paper_scale_basis(m["Fstar"])
    s = lbm.LBMSolid(nx, nx, m["dx"], I.PAPER_E, I.PAPER_NU, control="force_basis2",
                     force_basis=basis.reshape(-1))
    s.set_target(dev(m["dstar"]))
    a = torch.tensor([0.3, -0.7], dtype=torch.float64, device="cuda", requires_grad=True)
    J = gbo.objective(a, s)
    J.backward()
    g = a.grad.cpu().numpy()
    # J is quadratic in alpha: central differences are exact up to cancellation
    h = 1e-3
    for i in range(2):
        e = np.zeros(2)
        e[i] = h
        Jp = float(gbo.objective(dev(a.detach().cpu().numpy() + e), s))
        Jm = float(gbo.objective(dev(a.detach().cpu().numpy() - e), s))
        assert abs((Jp - Jm) / (2 * h) - g[i]) <= 1e-7 * np.abs(g).max()
    # the backward restores the checkpointed steady state if another forward ran first
    a2 = torch.tensor([0.3, -0.7], dtype=torch.float64, device="cuda", requires_grad=True)
    J2 = gbo.objective(a2, s)
    gbo.objective(dev([1.0, 1.0]), s)  # overwrites the handle's state
    J2.backward()
    assert np.allclose(a2.grad.cpu().numpy(), g, rtol=1e-9, atol=0)
    s.close()


def test_benchmark1_identification_reaches_the_exact_fit(mods):
    # Section 4.2.3: alpha^(0) = (-1, -1), l = 20, lambda0 = 1, eps = 1e-10 (Table 2)
    lbm, gbo = mods
    nx = 20
    m = I.periodic_manufactured(nx)
    basis = I.paper_scale_basis(m["Fstar"])
    s = lbm.LBMSolid(nx, nx, m["dx"], I.PAPER_E, I.PAPER_NU, control="force_basis2",
                     force_basis=basis.reshape(-1))
    s.set_target(dev(m["dstar"]))
    r = gbo.lbfgs(gbo.make_fg(s), dev([-1.0, -1.0]), m_max=50, eps=1e-10)
    a = r.alpha.cpu().numpy()
    a_opt = exact_fit(nx, I.PAPER_E, I.PAPER_NU, basis, m["dstar"])
    assert r.steps <= 20, r
    assert r.J <= 1e-20  # target exactly representable: J at round-off level
    assert np.abs(a - a_opt).max() <= 1e-8 * np.abs(a_opt).max()
    # control-error floor = amplitude error of the scheme, O(dx^2)
    assert 1e-3 < np.linalg.norm(a - 1.0) / np.sqrt(2) < 5e-2
    s.close()


def test_two_amplitude_identification(mods):
    # two-amplitude workload: lambda = mu = 1, alpha_ref = (1, 0.5), start (0, 0)
    lbm, gbo = mods
    nx = 32
    c = I.config_amplitudes(nx)
    s = lbm.LBMSolid(nx, nx, c["dx"], c["E"], c["nu"], control="force_basis2",
                     force_basis=c["basis"].reshape(-1))
    s.set_target(dev(c["dstar"]))
    r = gbo.lbfgs(gbo.make_fg(s), dev([0.0, 0.0]), m_max=50, eps=1e-8)
    a_opt = exact_fit(nx, c["E"], c["nu"], c["basis"], c["dstar"])
    assert r.reason in ("gradient", "control change"), r.reason
    assert np.abs(r.alpha.cpu().numpy() - a_opt).max() <= 1e-7
    s.close()


def test_distributed_control_with_projection(mods):
    # Section 4.2.4: F itself is the control (2N values), uninformed start (-1, -1)
    # projected to zero mean, projected gradients; the recovered force is the discrete
    # exact fit, which for this single-wavenumber target is alpha_opt o F*.
    lbm, gbo = mods
    nx = 10
    m = I.periodic_manufactured(nx)
    s = lbm.LBMSolid(nx, nx, m["dx"], I.PAPER_E, I.PAPER_NU, control="force_field")
    s.set_target(dev(m["dstar"]))
    a0 = -np.ones((2, nx * nx))
    a0 -= a0.mean(axis=1, keepdims=True)  # Eq. zero_mean_projection
    dx = m["dx"]
    l2 = lambda g: float(torch.sqrt(dx * dx * torch.sum(g * g)))  # noqa: E731
    r = gbo.lbfgs(gbo.make_fg(s, project=True), dev(a0), m_max=100, eps=1e-10, norm=l2)
    F = r.alpha.cpu().numpy().reshape(2, -1)
    a_opt = exact_fit(nx, I.PAPER_E, I.PAPER_NU, I.paper_scale_basis(m["Fstar"]), m["dstar"])
    F_opt = a_opt[:, None] * m["Fstar"]
    assert r.J <= 1e-18
    assert np.abs(F - F_opt).max() <= 1e-6 * np.abs(F_opt).max()
    assert abs(F.mean(axis=1)).max() <= 1e-12 * np.abs(F).max()
    s.close()


def test_plate_young_identification(mods):
    # Section 4.3.3: E = alpha^2, E^(0) = 0.15, E* = 0.1, f-AD in the paper (ALBM here)
    lbm, gbo = mods
    Nx = 24
    geo = I.plate_geometry(Nx)
    dstar, sigma, F = I.plate_manufactured(geo.X, geo.Y)
    wd, wT = I.plate_wall_data(geo)
    s = lbm.LBMSolid(geo.nx, geo.nx, geo.dx, I.PLATE_E, I.PLATE_NU, periodic=False,
                     node_mask=geo.active, link_bc=geo.link, wall_d=wd, wall_T=wT,
                     wall_n=geo.normal, obs=geo.active.astype(float), control="young_scalar",
                     force=F * geo.active)
    s.set_target(dev(dstar))
    # near E = 0.2 (nu = 0.7) tau_s = 1/2 and the boundary gamma is singular (Eq. gamma); a
    # trial control where the iteration diverges gets J = inf and the line search steps back
    opts = gbo.SolveOpts(tol=1e-12, max_steps=400_000)
    r = gbo.lbfgs(gbo.make_fg(s, opts, opts), dev([np.sqrt(0.15)]), m_max=30, eps=1e-10)
    E = float(r.alpha[0]) ** 2
    # a stationary point of J(E): the gradient fell by orders of magnitude, and J there is
    # below J at the reference modulus and at the start
    assert r.reason in ("gradient", "control change", "line search"), r.reason
    assert r.grad_norm <= 1e-4 * r.history[0]["grad_norm"]
    fg = gbo.make_fg(s, opts, opts)
    J_ref, _ = fg(dev([np.sqrt(I.PLATE_E)]))
    assert r.J <= J_ref and r.J <= r.history[0]["J"]
    # The recovered modulus carries the boundary rules' discretisation error (first order,
    # large constant at N_x = 24); the paper's own rules give 2.23 % at N_x = 40.  Only the
    # order of magnitude is pinned here.
    assert 0.05 < E < 0.3, E
    s.close()


def test_plate_identification_from_previous_steady_states(mods):
    # clamped / tensioned plate, target = its own state at E = 1, L-BFGS from E = 0.5.  The
    # evaluation points of the cold run are replayed with every solve started from the
    # history of steady states: same objectives and gradients (every solve converges to
    # the same residual), fewer sweeps.  history = 1 restarts from the last state;
    # history = 3 extrapolates the primal state in 1/E and fits the adjoint source.
    lbm, gbo = mods
    from paper_2609_31347_b300 import warmstart as W
    geo, wd, wT = I.baseline_plate(24)

    def solver():
        s = lbm.LBMSolid(geo.nx, geo.nx, geo.dx, 1.0, 0.3, periodic=False,
                         node_mask=geo.active, link_bc=geo.link, wall_d=wd, wall_T=wT,
                         wall_n=geo.normal, control="young_scalar")
        s.set_control(dev([1.0]))
        s.primal_solve(1_000_000, tol=1e-13, criterion=1)
        s.set_target(s.displacement())
        s.sweeps.clear()
        return s

    opts = gbo.SolveOpts(tol=1e-11, max_steps=1_000_000)
    s = solver()
    fg = gbo.make_fg(s, opts, opts)
    pts, ref = [], []

    def rec(a):
        pts.append(a.detach().clone())
        ref.append(fg(a))
        return ref[-1]
    # stop once the gradient fell by 1e-5 (E within ~1e-5): beyond that the objective
    # reaches the level of the solves' own residual error
    _, gs = fg(dev([np.sqrt(0.5)]))
    s.sweeps.clear()
    r = gbo.lbfgs(rec, dev([np.sqrt(0.5)]), m_max=20, eps=1e-5 * float(gs.abs().max()))
    cold = s.sweeps["primal_solve"] + s.sweeps["adjoint_solve"]
    s.close()
    assert r.reason == "gradient", r.reason
    assert abs(float(r.alpha[0]) ** 2 - 1.0) < 1e-4, float(r.alpha[0]) ** 2
    assert len(pts) >= 4
    s = solver()
    with pytest.raises(ValueError):  # the networks map periodic force fields only
        gbo.make_fg(s, opts, opts, warm=W.WarmStarter(primal=object()))(pts[0])
    s.close()
    J0, g0 = ref[0][0], float(ref[0][1].abs().max())
    sweeps = {}
    for history in (1, 3):
        s = solver()
        fgw = gbo.make_fg(s, opts, opts, warm=W.WarmStarter(history=history))
        for a, (J, g) in zip(pts, ref):
            Jw, gw = fgw(a)
            if math.isinf(J):  # a trial modulus with no steady state diverges from any start
                assert math.isinf(Jw)
                continue
            assert abs(Jw - J) <= 1e-6 * J0, (history, Jw, J)
            assert float((gw - g).abs().max()) <= 1e-5 * g0, history
        sweeps[history] = s.sweeps["primal_solve"] + s.sweeps["adjoint_solve"]
        s.close()
    # the last state alone is no better than rest for the adjoint (its source shrinks
    # towards the optimum), the combinations are
    assert sweeps[3] < 0.85 * cold and sweeps[3] < 0.85 * sweeps[1], (sweeps, cold)


def test_distributed_gradient_central_fd_at_64_random_nodes(mods):
    # 80^2 distributed force control (12,800 controls) at zero control, seed 0: the ALBM
    # gradient against central differences with h = 1e-6 at 64 random (node, component)
    # pairs.  On the periodic lattice a point force has nonzero mean and no steady state
    # (Section 2, compatibility), so each perturbation is projected to zero mean
    # (Eq. zero_mean_projection) and compared with the projected gradient.  J is
    # quadratic in F, so the only FD error is cancellation ~ eps J / h.
    # A point perturbation also excites the wavevectors (N/2, 0) and (0, N/2), where the
    # primal step has the eigenvalue -1 (tests/test_oracle_periodic.py): those components
    # alternate and never pass the residual test, so the perturbed solves stop at an even
    # max_steps, where the alternating part is zero; it is orthogonal to the smooth
    # target, so it does not enter the derivative at F = 0.
    lbm, gbo = mods
    nx = 80
    N = nx * nx
    c = I.config_amplitudes(nx)
    s = lbm.LBMSolid(nx, nx, c["dx"], c["E"], c["nu"], control="force_field")
    s.set_target(dev(c["dstar"]))
    opts = gbo.SolveOpts(tol=1e-13)
    pert = gbo.SolveOpts(tol=1e-13, max_steps=64 * 128)  # smooth part converged by ~2000
    F0 = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    J0, g = gbo.make_fg(s, opts, opts, project=True)(F0)
    g = g.cpu().numpy()
    rng = np.random.default_rng(0)
    picks = rng.choice(2 * N, size=64, replace=False)
    h = 1e-6
    worst = 0.0
    for p in picks:
        comp = p // N
        e = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
        e[comp * N:(comp + 1) * N] = -1.0 / N
        e[p] += 1.0
        Jp = float(gbo.objective(F0 + h * e, s, pert, opts))
        Jm = float(gbo.objective(F0 - h * e, s, pert, opts))
        # directional derivative along the projected unit vector = projected gradient
        worst = max(worst, abs((Jp - Jm) / (2 * h) - g[p]))
    # cancellation bound of central differences: a few eps |J| / h
    assert worst <= 10 * 2.2e-16 * abs(J0) / h + 1e-9 * np.abs(g).max(), (worst, J0)
    s.close()


def test_plate_identification_error_on_the_paper_ladder(mods):
    # Section 4.3.3 with Table 4 settings (E^(0) = 0.15, E* = 0.1, eps = 1e-10, solves capped
    # at T_max = 60): the recovered control's error falls under refinement, at the order
    # of the printed errors (2.23 % at N_x = 40, 0.55 % at N_x = 80).  The paper's boundary
    # rules are not given and ours are first order of their own, so only the order of
    # magnitude and the decrease are pinned (measured here: 6.5 % and 2.0 %).
    lbm, gbo = mods
    errs = []
    for Nx, paper in ((40, 0.0223), (80, 0.0055)):
        geo = I.plate_geometry(Nx)
        dstar, sigma, F = I.plate_manufactured(geo.X, geo.Y)
        wd, wT = I.plate_wall_data(geo)
        s = lbm.LBMSolid(geo.nx, geo.nx, geo.dx, I.PLATE_E, I.PLATE_NU, periodic=False,
                         node_mask=geo.active, link_bc=geo.link, wall_d=wd, wall_T=wT,
                         wall_n=geo.normal, obs=geo.active.astype(float),
                         control="young_scalar", force=F * geo.active)
        s.set_target(dev(dstar))
        opts = gbo.SolveOpts(tol=1e-10, max_steps=int(60 * Nx * Nx / 2.25))
        r = gbo.lbfgs(gbo.make_fg(s, opts, opts), dev([np.sqrt(0.15)]), m_max=50, eps=1e-10,
                      k_max=20)
        a = abs(float(r.alpha[0]))
        err = abs(a - np.sqrt(I.PLATE_E)) / np.sqrt(I.PLATE_E)
        assert paper / 5 <= err <= 5 * paper, (Nx, err)
        errs.append(err)
        s.close()
    assert errs[1] < 0.5 * errs[0]
