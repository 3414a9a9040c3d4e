"""Oracle pins of the convergence monitor and stopping rule (Eqs. convergence,
convergence_crit), and of the oracle's thread count, CPU only.

- The stopping rule on hand-made sequences: the first index whose trailing window has
  population standard deviation / mean below the tolerance (a case where the sample
  standard deviation would not fire yet), and a constant zero window.
- The c(t) traces equal the monitor of the states the plain stepping reaches.
- Results are bitwise the same with one thread and with all of them.
"""
import numpy as np
import pytest

import oracle
from paper_2609_31347_b300 import inputs as I


def test_cv_rule_on_hand_sequences():
    c = [1.0, 2.0, 3.0, 3.0, 3.0]
    # windows of 3: [1,2,3] CV = sqrt(2/3)/2 = 0.408; [2,3,3] CV = sqrt(2/9)/(8/3) = 0.177;
    # [3,3,3] CV = 0
    i, m = oracle.cv_stop(c, 3, 0.2)
    assert i == 3 and m == pytest.approx(np.sqrt(2.0 / 9.0) / (8.0 / 3.0), rel=1e-14)
    # the sample standard deviation (divided by 2) would give 0.2165 there: not below 0.2
    i, m = oracle.cv_stop(c, 3, 0.1)
    assert i == 4 and m == 0.0
    i, m = oracle.cv_stop(c, 3, 1e-3)
    assert i == 4
    assert oracle.cv_stop([1.0, 2.0, 4.0, 8.0], 2, 0.1)[0] == -1  # never holds
    assert oracle.cv_stop([0.0, 0.0, 0.0], 2, 1e-9)[0] == 1     # constant zero window
    assert oracle.cv_stop([5.0], 2, 1.0)[0] == -1               # window never full


def _plate(Nx=10):
    geo = I.plate_geometry(Nx)
    dstar, sigma, F = I.plate_manufactured(geo.X, geo.Y)
    wd, wT = I.plate_wall_data(geo)
    g = oracle.Grid(geo.nx, geo.nx, geo.dx, I.PLATE_NU, periodic=False,
                    node_type=geo.node_type, link=geo.link, wall_d=wd, wall_T=wT,
                    wall_n=geo.normal)
    return g, F * geo.active, dstar


def test_primal_trace_is_the_monitor_of_the_stepped_states():
    nx = 9
    g = oracle.Grid(nx, nx, 1.0 / nx, 0.3)
    F = I.fourier_force(nx, seed=4, kmax=3)
    E = 0.7
    tr = oracle.primal_trace(g, E, F, 12)
    # at rest d = g / 2 (the half force of Eq. moments_bar_1/2)
    assert tr[0] == oracle.monitor(g, np.zeros((8, nx * nx)), F) > 0.0
    for t in (1, 5, 12):
        assert tr[t] == oracle.monitor(g, oracle.primal(g, E, F, t), F)
    gp, Fp, _ = _plate()
    tr = oracle.primal_trace(gp, I.PLATE_E, Fp, 9)
    for t in (3, 9):
        assert tr[t] == oracle.monitor(gp, oracle.primal(gp, I.PLATE_E, Fp, t), Fp)


def test_adjoint_trace_is_the_adjoint_displacement_of_phi_S():
    nx = 8
    g = oracle.Grid(nx, nx, 1.0 / nx, 0.3)
    F = I.fourier_force(nx, seed=5, kmax=2)
    dstar = np.random.default_rng(5).standard_normal((2, nx * nx)) * 1e-3
    E = 0.9
    fS = oracle.primal(g, E, F, 40)
    tr = oracle.adjoint_trace(g, E, F, fS, dstar, 10)
    assert tr[0] == 0.0
    for i in (1, 4, 10):
        _, phiS = oracle.adjoint(g, E, F, fS, dstar, i)
        dphi = np.vstack([I.CX @ phiS, I.CY @ phiS])
        assert tr[i] == pytest.approx(np.mean((dphi ** 2).sum(0)), rel=1e-13)


def test_results_do_not_depend_on_the_thread_count():
    gp, Fp, dstar = _plate(12)
    nx = 16
    gq = oracle.Grid(nx, nx, 1.0 / nx, 0.3)
    Fq = I.fourier_force(nx, seed=6)
    dq = np.random.default_rng(6).standard_normal((2, nx * nx)) * 1e-3
    out = []
    for th in (1, 0):
        oracle.set_threads(th)
        res = []
        for g, F, ds, E in ((gq, Fq, dq, 0.8), (gp, Fp, dstar, I.PLATE_E)):
            fS = oracle.primal(g, E, F, 30)
            pc, ps = oracle.adjoint(g, E, F, fS, ds, 30)
            res += [fS, pc, ps, oracle.gradient_force(g, E, F, fS, ps, ds),
                    oracle.primal_trace(g, E, F, 5)]
        out.append(res)
    oracle.set_threads(0)
    for a, b in zip(*out):
        assert np.array_equal(a, b)
