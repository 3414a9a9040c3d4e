"""Starts from the history of an optimisation loop (not in the paper), CPU part: the
weight rules, and why they work on the plate, shown with the oracle's exact steady
states.

- Lagrange weights reproduce polynomials of degree < k (extrapolation included);
- the affine-fit weights sum to 1, reproduce a vector in the affine span of the
  previous ones and leave a residual orthogonal to their differences otherwise;
- the source-fit weights are the least-squares solution;
- on the clamped / tensioned plate the steady state is close to affine in 1/E, so
  extrapolating in 1/E from two steady states lands about 30 times closer to the new
  steady state than the last state alone (from three, closer still); and the last
  adjoint state alone is further from the new one than a start from rest, while the
  adjoint states combined with the weights that fit the new source land within 2 %.
"""
import numpy as np
import pytest

import oracle
from paper_2609_31347_b300 import inputs as I
from paper_2609_31347_b300.warmstart import (affine_fit_weights, lagrange_weights,
                                             source_fit_weights)


def gram(vs):
    V = np.stack(vs)
    return V @ V.T


def test_lagrange_weights_reproduce_low_degree_polynomials():
    rng = np.random.default_rng(0)
    xs = [0.5, 2.0, 1.1]
    for x in (1.0, 3.0, -0.4, 0.5):
        w = lagrange_weights(xs, x)
        for deg in range(3):
            c = rng.standard_normal(deg + 1)
            p = np.polynomial.polynomial.polyval
            assert abs(sum(wi * p(xi, c) for wi, xi in zip(w, xs)) - p(x, c)) <= 1e-12 * (
                1 + abs(p(x, c)))
    assert np.allclose(lagrange_weights(xs, 2.0), [0, 1, 0])
    # degree 3 is not reproduced by three points
    w = lagrange_weights(xs, 3.0)
    assert abs(sum(wi * xi ** 3 for wi, xi in zip(w, xs)) - 27.0) > 1.0


def test_affine_fit_weights():
    rng = np.random.default_rng(1)
    A = [rng.standard_normal(50) for _ in range(3)]
    # a point of the affine span is reproduced exactly
    lam = np.array([0.3, -1.2, 1.9])
    a = sum(l * v for l, v in zip(lam, A))
    w = affine_fit_weights(gram(A + [a]))
    assert abs(w.sum() - 1.0) < 1e-12
    assert np.abs(sum(wi * v for wi, v in zip(w, A)) - a).max() < 1e-10
    # otherwise the residual is orthogonal to the span's directions
    b = rng.standard_normal(50)
    w = affine_fit_weights(gram(A + [b]))
    res = sum(wi * v for wi, v in zip(w, A)) - b
    assert abs(w.sum() - 1.0) < 1e-12
    for v in A[:-1]:
        assert abs(res @ (v - A[-1])) < 1e-9 * np.linalg.norm(res) * np.linalg.norm(v)
    # collinear controls along a line search: the new point on the line is reproduced
    x, d = rng.standard_normal(50), rng.standard_normal(50)
    L = [x, x + 0.7 * d, x + 0.2 * d]
    w = affine_fit_weights(gram(L + [x + 1.5 * d]))
    assert np.abs(sum(wi * v for wi, v in zip(w, L)) - (x + 1.5 * d)).max() < 1e-9
    assert np.array_equal(affine_fit_weights(gram([x, d])), [1.0])


def test_source_fit_weights_are_least_squares():
    rng = np.random.default_rng(2)
    R = [rng.standard_normal(40) for _ in range(3)]
    r = rng.standard_normal(40)
    w = source_fit_weights(gram(R + [r]))
    ref = np.linalg.lstsq(np.stack(R, 1), r, rcond=None)[0]
    assert np.allclose(w, ref, rtol=1e-10, atol=1e-12)
    assert np.array_equal(source_fit_weights(gram([np.zeros(40), r])), [0.0])


@pytest.fixture(scope="module")
def plate():
    geo, wd, wT = I.baseline_plate(10)
    g = oracle.Grid(geo.nx, geo.nx, geo.dx, 0.3, periodic=False, node_type=geo.node_type,
                    link=geo.link, wall_d=wd, wall_T=wT, wall_n=geo.normal)
    N = g.N
    F = np.zeros(2 * N)
    idx = np.nonzero(np.repeat(geo.node_type[None, :] > 0, 8, axis=0).ravel())[0]

    def step_matrix(E, transpose):
        n = idx.size
        A = np.zeros((n, n))
        apply = oracle.apply_step_transpose if transpose else oracle.apply_step
        for j, k in enumerate(idx):
            e = np.zeros(8 * N)
            e[k] = 1.0
            A[:, j] = apply(g, E, e).ravel()[idx]
        return A

    def primal(E):
        # exact steady f_S: the fixed point of f -> A f + b with b = one step from rest
        b = oracle.primal(g, E, F, 1).ravel()[idx]
        f = np.zeros(8 * N)
        f[idx] = np.linalg.solve(np.eye(idx.size) - step_matrix(E, False), b)
        return f

    Es = (0.6, 0.8, 0.95, 1.0)
    S = {E: primal(E) for E in Es}
    for E in Es:  # one oracle step from the solved state stays there
        f1 = oracle.primal(g, E, F, 1, fS0=S[E]).ravel()
        assert np.abs(f1 - S[E]).max() <= 1e-12 * np.abs(S[E]).max()
    dstar = oracle.displacement(g, S[1.0], F).ravel()

    def adjoint(E):
        # exact steady phi_C: the fixed point of the transposed step with the source of
        # one adjoint iteration from rest
        pc1, _ = oracle.adjoint(g, E, F, S[E], dstar, 1)
        p = np.zeros(8 * N)
        p[idx] = np.linalg.solve(np.eye(idx.size) - step_matrix(E, True), pc1.ravel()[idx])
        return p, pc1.ravel()  # pc1 = -(c . r): linear in the source r

    P = {E: adjoint(E) for E in Es[:3]}
    return S, P, Es


def test_plate_state_extrapolates_in_inverse_modulus(plate):
    S, P, Es = plate
    assert all(np.abs(S[E]).max() > 0 for E in Es)
    f_new = S[Es[3]]
    reuse = np.abs(S[Es[2]] - f_new).max()
    w = lagrange_weights([1 / Es[1], 1 / Es[2]], 1 / Es[3])
    lin = np.abs(w[0] * S[Es[1]] + w[1] * S[Es[2]] - f_new).max()
    w = lagrange_weights([1 / E for E in Es[:3]], 1 / Es[3])
    quad = np.abs(sum(wi * S[E] for wi, E in zip(w, Es[:3])) - f_new).max()
    assert lin < 0.1 * reuse, (lin, reuse)
    assert quad < 0.5 * lin, (quad, lin)


def test_plate_adjoint_state_from_source_fit(plate):
    S, P, Es = plate
    p_new, r_new = P[Es[2]]
    reuse = np.abs(P[Es[1]][0] - p_new).max()
    G = gram([P[Es[0]][1], P[Es[1]][1], r_new])
    w = source_fit_weights(G)
    fit = np.abs(w[0] * P[Es[0]][0] + w[1] * P[Es[1]][0] - p_new).max()
    assert fit < 0.05 * reuse, (fit, reuse)
    assert fit < 0.05 * np.abs(p_new).max()


# ---- WarmStarter's choices, with the library's two vector calls done in numpy ------

class FakeSolver:
    """Just what WarmStarter touches: control kind, geometry, the steady states."""

    def __init__(self, control, periodic=False, N=5):
        import torch
        self.control, self.periodic, self.N, self.nx, self.dx = control, periodic, N, N, 1.0
        self.f = torch.zeros(8 * N, dtype=torch.float64)
        self.p = torch.zeros(8 * N, dtype=torch.float64)
        self.r = torch.zeros(2 * N, dtype=torch.float64)
        self.sets = []

    def get_populations(self, which):
        return self.f if which == 0 else self.p

    def set_populations(self, which, t):
        self.sets.append((which, t.clone()))

    def adjoint_source(self):
        return self.r.clone()


@pytest.fixture
def W(monkeypatch):
    import torch
    from paper_2609_31347_b300 import warmstart

    def dots(vs):
        V = torch.stack([v.reshape(-1) for v in vs]).numpy()
        return V @ V.T

    def combine(w, srcs, dst):
        dst.copy_(sum(float(wi) * s for wi, s in zip(w, srcs)))
        return dst

    monkeypatch.setattr(warmstart.L, "warm_dots", dots)
    monkeypatch.setattr(warmstart.L, "warm_combine", combine)
    return warmstart


def test_scalar_modulus_start_is_the_extrapolation_in_inverse_modulus(W):
    import torch
    rng = np.random.default_rng(3)
    a, b, c = (torch.as_tensor(rng.standard_normal(40)) for _ in range(3))
    state = lambda E: a + b / E + c / E ** 2  # quadratic in 1/E: reproduced exactly
    s = FakeSolver("young_scalar")
    ws = W.WarmStarter(history=3)
    ctrl = lambda E: torch.tensor([np.sqrt(E)], dtype=torch.float64)
    ws.before_primal(s, ctrl(0.5))
    assert s.sets == []  # no history, no network: from rest
    for E in (0.5, 0.8, 1.2):
        s.f = state(E)
        ws.after_primal(s, ctrl(E))
    ws.before_primal(s, ctrl(1.0))
    which, f0 = s.sets[-1]
    assert which == 0
    assert torch.allclose(f0, state(1.0), rtol=0, atol=1e-12)
    # history = 1: the last state
    ws1 = W.WarmStarter(history=1)
    for E in (0.5, 0.8, 1.2):
        s.f = state(E)
        ws1.after_primal(s, ctrl(E))
    ws1.before_primal(s, ctrl(1.0))
    assert torch.equal(s.sets[-1][1], state(1.2))
    # states crowded together and a far target: weights above the bound, so the
    # oldest entries are dropped down to the last state
    ws2 = W.WarmStarter(history=3)
    for E in (1.0, 1.001, 1.002):
        s.f = state(E)
        ws2.after_primal(s, ctrl(E))
    ws2.before_primal(s, ctrl(0.3))
    assert torch.equal(s.sets[-1][1], state(1.002))


def test_force_control_start_is_the_affine_fit(W):
    import torch
    rng = np.random.default_rng(4)
    K = torch.as_tensor(rng.standard_normal((40, 10)))
    f_of = lambda F: K @ F + 1.0  # steady state affine in the control
    s = FakeSolver("force_field", periodic=True, N=5)
    ws = W.WarmStarter(history=3)
    x, d = torch.as_tensor(rng.standard_normal(10)), torch.as_tensor(rng.standard_normal(10))
    for t in (0.0, 1.0, 0.4):  # points of one line search
        s.f = f_of(x + t * d)
        ws.after_primal(s, x + t * d)
    ws.before_primal(s, x + 0.7 * d)
    assert torch.allclose(s.sets[-1][1], f_of(x + 0.7 * d), rtol=0, atol=1e-11)


def test_adjoint_start_fits_the_source_or_starts_from_rest(W):
    import torch
    rng = np.random.default_rng(5)
    K = torch.as_tensor(rng.standard_normal((40, 10)))  # steady state linear in r
    s = FakeSolver("young_scalar", N=5)
    ws = W.WarmStarter(history=3)
    R = [torch.as_tensor(rng.standard_normal(10)) for _ in range(2)]
    ws.before_adjoint(s)
    assert s.sets == []
    for r in R:
        s.r, s.p = r, K @ r
        ws.before_adjoint(s)
        ws.after_adjoint(s)
    s.sets.clear()
    s.r = 0.3 * R[0] - 0.7 * R[1]
    ws.before_adjoint(s)
    which, p0 = s.sets[-1]
    assert which == 2
    assert torch.allclose(p0, K @ s.r, rtol=0, atol=1e-12)
    # a source the previous ones do not explain: from rest
    s.sets.clear()
    Q, _ = np.linalg.qr(np.stack([R[0].numpy(), R[1].numpy(), rng.standard_normal(10)], 1))
    s.r = torch.as_tensor(Q[:, 2].copy())
    ws.before_adjoint(s)
    assert s.sets == []


def test_networks_are_refused_off_the_periodic_force_field(W):
    s = FakeSolver("young_scalar")
    with pytest.raises(ValueError):
        W.WarmStarter(primal=object()).before_primal(s, None)
    with pytest.raises(ValueError):
        W.WarmStarter(history=5)
