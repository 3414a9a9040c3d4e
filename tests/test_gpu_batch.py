"""GPU tests of the batched path (many periodic instances, one launch per sweep): each
instance equals a single-lattice handle with the same kernel, the autotuner keeps the
state, and a batch of node-wise finite-difference perturbations reproduces the adjoint
gradient (Section 4.2.5's gradient validation, done as one batched run)."""
import numpy as np
import pytest

import oracle
from paper_2609_31347_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def lbm():
    from paper_2609_31347_b300 import lbm as m
    assert torch.cuda.is_available()
    m.load_library()
    return m


SIZES = [(3, 5), (17, 9), (64, 33), (130, 67), (257, 3), (40, 40)]


@pytest.mark.parametrize("kernel", ["fp64", "auto"])
def test_batch_instances_equal_single_handles(lbm, kernel):
    E, nu, T, K = 0.7, 0.25, 37, 29
    b = lbm.LBMBatch(SIZES, E, nu, kernel=kernel)
    # lay out per instance: [Fx plane, Fy plane] at 2*off_i
    Fb = np.zeros(2 * b.total)
    Db = np.zeros(2 * b.total)
    for i, (nx, ny) in enumerate(SIZES):
        o, n = b.offsets[i], nx * ny
        Fi = I.fourier_force(nx, ny=ny, seed=i, kmax=2)
        Di = np.random.default_rng(50 + i).standard_normal((2, n)) * 1e-3
        Fb[2 * o:2 * (o + n)] = Fi.ravel()
        Db[2 * o:2 * (o + n)] = Di.ravel()
    b.set_target(dev(Db))
    b.set_force(dev(Fb))
    b.primal(T)
    Jb = host(b.objective())
    b.adjoint(K)
    fS = b.get_populations(0)
    pC = b.get_populations(2)
    gB = b.gradient()
    for i, (nx, ny) in enumerate(SIZES):
        o, n = b.offsets[i], nx * ny
        s = lbm.LBMSolid(nx, ny, 1.0 / nx, E, nu, kernel=kernel)
        s.set_target(dev(Db[2 * o:2 * (o + n)]))
        s.set_control(dev(Fb[2 * o:2 * (o + n)]))
        s.primal_solve(T, fixed_steps=True)
        f1 = host(s.get_populations(0)).reshape(8, n)
        assert np.array_equal(host(b.pop_view(fS, i)), f1), i  # same arithmetic, bit for bit
        J1 = s.objective()
        assert abs(Jb[i] - J1) <= 1e-13 * abs(J1)
        s.adjoint_solve(K, fixed_steps=True)
        p1 = host(s.get_populations(2)).reshape(8, n)
        assert np.abs(host(b.pop_view(pC, i)) - p1).max() <= 1e-13 * np.abs(p1).max()
        g1 = host(s.gradient()).reshape(2, n)
        assert np.abs(host(b.field_view(gB, i)) - g1).max() <= 1e-12 * np.abs(g1).max()
        s.close()
    # and one instance against the oracle
    nx, ny = SIZES[1]
    o, n = b.offsets[1], nx * ny
    g = oracle.Grid(nx, ny, 1.0 / nx, nu)
    ref = oracle.primal(g, E, Fb[2 * o:2 * (o + n)].reshape(2, n), T)
    got = host(b.pop_view(fS, 1))
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    b.close()


def test_tuner_keeps_the_state(lbm):
    sizes = [(96, 80), (200, 50), (31, 77)]
    b = lbm.LBMBatch(sizes, 1.0, 0.3)
    Fb = np.zeros(2 * b.total)
    for i, (nx, ny) in enumerate(sizes):
        o, n = b.offsets[i], nx * ny
        Fb[2 * o:2 * (o + n)] = I.fourier_force(nx, ny=ny, seed=7 + i, kmax=2).ravel()
    b.set_force(dev(Fb))
    b.primal(10)
    before = host(b.get_populations(0))
    bx = b.tune(8)
    assert bx in (32, 64, 128, 256)
    assert np.array_equal(host(b.get_populations(0)), before)
    b.primal(10)
    ref = lbm.LBMBatch(sizes, 1.0, 0.3)
    ref.set_force(dev(Fb))
    ref.primal(20)
    assert np.array_equal(host(b.get_populations(0)), host(ref.get_populations(0)))
    b.close()
    ref.close()


def test_batched_finite_difference_perturbations(lbm):
    # 80^2 distributed force control at half the reference force: 2 x 16 perturbed
    # copies (zero-mean unit perturbations at 16 random (node, component) pairs, +-h)
    # run as one batch; central differences equal the adjoint gradient (J is quadratic).
    nx, T = 80, 4000
    N = nx * nx
    c = I.config_amplitudes(nx)
    F0 = 0.5 * np.tensordot([1.0, 0.5], c["basis"], axes=1).ravel()
    s = lbm.LBMSolid(nx, nx, c["dx"], c["E"], c["nu"])
    s.set_target(dev(c["dstar"]))
    s.set_control(dev(F0))
    s.primal_solve(T, fixed_steps=True)
    s.adjoint_solve(T, fixed_steps=True)
    g = host(s.gradient(project_zero_mean=True))
    s.close()
    rng = np.random.default_rng(0)
    picks = rng.choice(2 * N, size=16, replace=False)
    h = 1e-4
    m = 2 * len(picks)
    b = lbm.LBMBatch([(nx, nx)] * m, c["E"], c["nu"])
    Fb = np.tile(F0, m)
    for j, p in enumerate(picks):
        comp = p // N
        e = np.zeros(2 * N)
        e[comp * N:(comp + 1) * N] = -1.0 / N
        e[p] += 1.0
        Fb[(2 * j) * 2 * N:(2 * j + 1) * 2 * N] += h * e
        Fb[(2 * j + 1) * 2 * N:(2 * j + 2) * 2 * N] -= h * e
    b.set_target(dev(np.tile(c["dstar"].ravel(), m)))
    b.set_force(dev(Fb))
    b.primal(T)
    J = host(b.objective())
    fd = (J[0::2] - J[1::2]) / (2 * h)
    assert np.abs(fd - g[picks]).max() <= 1e-7 * np.abs(g).max()
    b.close()


@pytest.mark.parametrize("kernel", ["fp64", "auto"])
def test_batch_adjoint_and_gradient_match_the_oracle(lbm, kernel):
    # uneven instances compared directly with the oracle: primal state, objective,
    # adjoint phi_C (Eq. adjoint_iteration) and the nodal force gradient (Eq. optimality)
    sizes = [(17, 9), (40, 23), (5, 31)]
    E, nu, T, K = 0.7, 0.25, 41, 33
    b = lbm.LBMBatch(sizes, E, nu, kernel=kernel)
    Fb = np.zeros(2 * b.total)
    Db = np.zeros(2 * b.total)
    for i, (nx, ny) in enumerate(sizes):
        o, n = b.offsets[i], nx * ny
        Fb[2 * o:2 * (o + n)] = I.fourier_force(nx, ny=ny, seed=60 + i, kmax=2).ravel()
        Db[2 * o:2 * (o + n)] = np.random.default_rng(70 + i).standard_normal(2 * n) * 1e-3
    b.set_target(dev(Db))
    b.set_force(dev(Fb))
    b.primal(T)
    Jb = host(b.objective())
    b.adjoint(K)
    fS, pC, gB = b.get_populations(0), b.get_populations(2), b.gradient()
    for i, (nx, ny) in enumerate(sizes):
        o, n = b.offsets[i], nx * ny
        g = oracle.Grid(nx, ny, 1.0 / nx, nu)
        F = Fb[2 * o:2 * (o + n)].reshape(2, n)
        D = Db[2 * o:2 * (o + n)].reshape(2, n)
        f_ref = oracle.primal(g, E, F, T)
        J_ref, _ = oracle.objective(g, f_ref, F, D)
        pc_ref, ps_ref = oracle.adjoint(g, E, F, f_ref, D, K)
        g_ref = oracle.gradient_force(g, E, F, f_ref, ps_ref, D)
        f_got = host(b.pop_view(fS, i))
        assert np.abs(f_got - f_ref).max() <= 1e-11 * np.abs(f_ref).max(), i
        assert abs(Jb[i] - J_ref) <= 1e-12 * abs(J_ref), i
        p_got = host(b.pop_view(pC, i))
        assert np.abs(p_got - pc_ref).max() <= 1e-11 * np.abs(pc_ref).max(), i
        g_got = host(b.field_view(gB, i))
        assert np.abs(g_got - g_ref).max() <= 1e-10 * np.abs(g_ref).max(), i
    b.close()
