"""Learned warm start on the GPU: the state <-> network conversions against the
moment definition (Appendix A.1), and what the trained networks gain: fewer primal
and adjoint sweeps to the same residual tolerance, the same fixed point, and an
optimisation loop that reaches the same control error in fewer sweeps."""
import numpy as np
import pytest

from oracle import fourier as Fo
from paper_2609_31347_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E, NU = 8.0 / 3.0, 1.0 / 3.0


@pytest.fixture(scope="module")
def lbm():
    from paper_2609_31347_b300 import lbm as m
    assert torch.cuda.is_available()
    m.load_library()
    return m


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


def ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def stream():
    import ctypes
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def drop_half_nyquist(p, nx, ny):
    """p (..., nx*ny) minus its Fourier components at (nx/2, 0) and (0, ny/2)."""
    i = np.arange(nx * ny)
    ex = np.where((i % nx) % 2, -1.0, 1.0)
    ey = np.where((i // nx) % 2, -1.0, 1.0)
    n = nx * ny
    return p - (p @ ex)[..., None] * ex / n - (p @ ey)[..., None] * ey / n


def drop_conserved(p, mode):
    """p (count, 8, N) with the k = 0 invariants of the iteration set to zero: primal
    (mode 1) mean m10, m01 removed along the stationary states v = M^-1 (e_m10 + e_m12/3)
    (resp. m01, m21); adjoint (mode 2) mean <v, phi> removed along c_x, c_y."""
    M = Fo.moment_matrix()
    e = np.eye(8)
    vx = np.linalg.solve(M, e[0] + e[5] / 3)
    vy = np.linalg.solve(M, e[1] + e[6] / 3)
    cx, cy = M[0], M[1]
    pairs = ((cx, vx), (cy, vy)) if mode == 1 else ((vx, cx), (vy, cy))  # (functional, direction)
    mean = p.mean(axis=2)  # (count, 8)
    out = p.copy()
    for w, u in pairs:
        out -= (mean @ w)[:, None, None] * u[None, :, None]
    return out


def test_targets_are_the_scaled_moments_and_decode_inverts_them(lbm):
    lib = lbm.load_library()
    nx, count = 32, 3
    N = nx * nx
    dx = 1.0 / 96  # any spacing
    rng = np.random.default_rng(0)
    pops = rng.standard_normal((count, 8, N))
    field = rng.standard_normal((count, 2, N))
    x = torch.empty((count, nx, nx, 2), dtype=torch.float32, device="cuda")
    s = torch.empty(count, dtype=torch.float32, device="cuda")
    assert lib.lbm_warm_encode(count, nx, nx, 1, ptr(dev(field)), None, ptr(x), ptr(s), stream()) == 0
    srms = np.sqrt((field ** 2).mean(axis=(1, 2)))
    assert np.allclose(s.cpu().numpy(), srms, rtol=1e-6)
    assert np.allclose(x.cpu().numpy(), (field / srms[:, None, None]).transpose(0, 2, 1)
                       .reshape(count, nx, nx, 2), rtol=1e-6, atol=1e-6)
    chan = torch.as_tensor(np.array([1, 2, 3, 4, 5, 6, 7, 8], np.float32), device="cuda")
    M = Fo.moment_matrix()
    for mode in (1, 2, 0):
        t = torch.empty((count, nx, nx, 8), dtype=torch.float32, device="cuda")
        assert lib.lbm_warm_targets(count, nx, nx, dx, mode, ptr(dev(pops)), ptr(s), ptr(chan),
                                    ptr(t), stream()) == 0
        m = np.einsum("ik,bkn->bin", M, pops)
        th, a = (1 / 3, 1.0) if mode == 1 else (2 / 3, dx * dx)
        if mode:
            z = a * np.stack([m[:, 0], m[:, 1], m[:, 2] / dx, m[:, 3] / dx, m[:, 4] / dx,
                              (m[:, 5] - th * m[:, 0]) / dx ** 2, (m[:, 6] - th * m[:, 1]) / dx ** 2,
                              m[:, 7] / dx], axis=1)
        else:
            z = m
        z = z / srms[:, None, None] / np.arange(1, 9)[None, :, None]
        got = t.cpu().numpy().reshape(count, N, 8).transpose(0, 2, 1)
        assert np.abs(got - z).max() <= 1e-6 * np.abs(z).max()
        back = torch.empty(count * 8 * N, dtype=torch.float64, device="cuda")
        assert lib.lbm_warm_decode(count, nx, nx, 1, dx, mode, ptr(t), ptr(s), ptr(chan),
                                   ptr(back), 0, stream()) == 0
        tol = 1e-6 if mode == 0 else 1e-4  # the dx^-2 channels carry FP32 rounding
        want = pops if mode == 0 else drop_conserved(drop_half_nyquist(pops, nx, nx), mode)
        err = np.abs(back.cpu().numpy().reshape(count, 8, N) - want).max()
        assert err <= tol * np.abs(pops).max(), (mode, err)
        # accumulate adds
        assert lib.lbm_warm_decode(count, nx, nx, 1, dx, mode, ptr(t), ptr(s), ptr(chan),
                                   ptr(back), 1, stream()) == 0
        got = back.cpu().numpy().reshape(count, 8, N)
        assert np.abs(got - 2 * want).max() <= 2 * tol * np.abs(pops).max()
        if mode:  # nothing left at (N/2, 0), (0, N/2) nor in the k = 0 invariants
            assert np.abs(got - drop_half_nyquist(got, nx, nx)).max() <= 1e-13 * np.abs(got).max()
            assert np.abs(got - drop_conserved(got, mode)).max() <= 1e-13 * np.abs(got).max()
    # c_i = 0: the channel is neither a target nor predicted
    chan0 = torch.as_tensor(np.array([1, 1, 1, 1, 1, 0, 0, 1], np.float32), device="cuda")
    assert lib.lbm_warm_targets(count, nx, nx, dx, 2, ptr(dev(pops)), ptr(s), ptr(chan0),
                                ptr(t), stream()) == 0
    tt = t.cpu().numpy()
    assert np.all(tt[..., 5:7] == 0) and np.all(np.isfinite(tt))
    # mode 3 (bounded grids): the targets of mode 1, decoded without the periodic steps
    t1 = torch.empty_like(t)
    assert lib.lbm_warm_targets(count, nx, nx, dx, 1, ptr(dev(pops)), ptr(s), None,
                                ptr(t1), stream()) == 0
    assert lib.lbm_warm_targets(count, nx, nx, dx, 3, ptr(dev(pops)), ptr(s), None,
                                ptr(t), stream()) == 0
    assert torch.equal(t, t1)
    back3 = torch.empty(count * 8 * N, dtype=torch.float64, device="cuda")
    back0 = torch.empty(count * 8 * N, dtype=torch.float64, device="cuda")
    assert lib.lbm_warm_decode(count, nx, nx, 1, dx, 3, ptr(t), ptr(s), None, ptr(back3), 0,
                               stream()) == 0
    assert np.abs(back3.cpu().numpy().reshape(count, 8, N) - pops).max() <= \
        1e-4 * np.abs(pops).max()
    assert lib.lbm_warm_targets(count, nx, nx, dx, 4, ptr(dev(pops)), ptr(s), None,
                                ptr(t), stream()) == lbm.LBM_ERR_ARG
    assert lib.lbm_warm_decode(count, nx, nx, 1, dx, 4, ptr(t), ptr(s), None, ptr(back0), 0,
                               stream()) == lbm.LBM_ERR_ARG


def test_restriction_and_prolongation(lbm):
    lib = lbm.load_library()
    nc, f = 16, 4
    nf = nc * f
    # fine field: block-constant values -> the coarse input is exactly those values
    v = np.random.default_rng(1).standard_normal((2, nc, nc))
    fine = np.repeat(np.repeat(v, f, axis=1), f, axis=2).reshape(1, 2, nf * nf)
    x = torch.empty((1, nc, nc, 2), dtype=torch.float32, device="cuda")
    s = torch.empty(1, dtype=torch.float32, device="cuda")
    ref = 0.5 * fine
    assert lib.lbm_warm_encode(1, nf, nf, f, ptr(dev(fine)), ptr(dev(ref)), ptr(x), ptr(s), stream()) == 0
    sr = np.sqrt(((0.5 * fine) ** 2).mean())
    assert abs(float(s.item()) - sr) <= 1e-6 * sr
    assert np.allclose(x.cpu().numpy()[0], 0.5 * v.transpose(1, 2, 0) / sr, rtol=1e-5, atol=1e-6)
    # prolongation of a smooth coarse field: second-order accurate at the fine nodes
    xc = (np.arange(nc) * f + 0.5 * (f - 1)) / nf  # coarse node = centre of its block
    Xc, Yc = np.meshgrid(xc, xc, indexing="xy")
    y = np.zeros((1, nc, nc, 8), np.float32)
    y[0, :, :, 0] = np.cos(2 * np.pi * Xc) * np.sin(2 * np.pi * Yc)
    one = torch.ones(1, dtype=torch.float32, device="cuda")
    out = torch.empty(8 * nf * nf, dtype=torch.float64, device="cuda")
    assert lib.lbm_warm_decode(1, nc, nc, f, 1.0 / nf, 0, ptr(torch.as_tensor(y, device="cuda")),
                               ptr(one), None, ptr(out), 0, stream()) == 0
    pops = out.cpu().numpy().reshape(8, nf * nf)
    m10 = Fo.moment_matrix()[0] @ pops
    xf = np.arange(nf) / nf
    Xf, Yf = np.meshgrid(xf, xf, indexing="xy")
    exact = (np.cos(2 * np.pi * Xf) * np.sin(2 * np.pi * Yf)).ravel()
    h = 2 * np.pi / nc
    assert np.abs(m10 - exact).max() <= 0.5 * h * h  # bilinear: |err| <= h^2/8 (|fxx|+|fyy|)


@pytest.fixture(scope="module")
def nets(lbm):
    from paper_2609_31347_b300 import warmstart as W
    out = {}
    for kind, count in (("primal", 2048), ("adjoint", 2048)):
        w = W.WarmStartNet(kind, nx=128, E=E, nu=NU, seed=0)
        X, T = w.generate(count, sweeps=5000, seed=1)
        log = w.fit(X, T, steps=2000, lr=1e-3)
        Xh, Th = w.generate(32, sweeps=5000, seed=99)
        out[kind] = (w, log, w.evaluate(Xh, Th))
        del X, T
    return out


def test_networks_learn_the_steady_states(nets):
    for kind, (w, log, err) in nets.items():
        assert log[-1][1] < 0.05 * log[0][1], (kind, log[0], log[-1])
        # held-out relative error of the predicted states (inputs include displacement-like
        # spectra, dominated by the lowest wavenumbers, where the network is least exact)
        assert err < 0.2, (kind, err)


def _primal(lbm, nx, F, f0=None):
    s = lbm.LBMSolid(nx, nx, 1.0 / nx, E, NU)
    s.set_control(F)
    if f0 is not None:
        s.set_populations(0, f0)
    info = s.primal_solve(4_000_000, tol=1e-10, criterion=1, check_every=64)
    f = s.get_populations(0).cpu().numpy()
    s.close()
    return info.steps, f


@pytest.mark.parametrize("nx", [128, 256])
def test_primal_warm_start_saves_sweeps_and_keeps_the_fixed_point(lbm, nets, nx):
    w = nets["primal"][0]
    for seed in (501, 502):
        F = I.fourier_fields(1, nx, seed=seed, kmax=4).reshape(-1).contiguous()
        cold, fc = _primal(lbm, nx, F)
        f0 = torch.empty(8 * nx * nx, dtype=torch.float64, device="cuda")
        w.predict(F, f0, nx_fine=nx)
        warm, fw = _primal(lbm, nx, F, f0)
        assert warm <= 0.85 * cold, (nx, cold, warm)
        assert np.abs(fw - fc).max() <= 5e-7 * np.abs(fc).max()


def test_adjoint_warm_start_saves_sweeps(lbm, nets):
    w = nets["adjoint"][0]
    nx = 128
    F = I.fourier_fields(1, nx, seed=7, kmax=4).reshape(-1).contiguous()
    dstar = I.fourier_fields(1, nx, seed=8, kmax=4).reshape(-1).contiguous() * 1e-2
    res = []
    for use in (False, True):  # the adjoint network is used at its own 128^2 here
        s = lbm.LBMSolid(nx, nx, 1.0 / nx, E, NU)
        s.set_target(dstar)
        s.set_control(F)
        s.primal_solve(4_000_000, tol=1e-12, criterion=1, check_every=64)
        if use:
            p0 = torch.empty(8 * nx * nx, dtype=torch.float64, device="cuda")
            w.predict(s.adjoint_source(), p0)
            s.set_populations(2, p0)
        info = s.adjoint_solve(4_000_000, tol=1e-10, criterion=1, check_every=64)
        res.append((info.steps, s.gradient().cpu().numpy()))
        s.close()
    (cold, gc), (warm, gw) = res
    assert warm <= 0.9 * cold, (cold, warm)
    assert np.abs(gw - gc).max() <= 1e-6 * np.abs(gc).max()


def test_optimisation_loop_same_evaluations_fewer_sweeps(lbm, nets):
    # distributed force control (2 x 128^2 values) towards the displacement of an 8-mode
    # force.  L-BFGS runs cold (every solve from rest, the paper's setting) and records
    # its evaluation points; the warm-started solver (network + previous states) then
    # evaluates the same points: the same objectives and gradients (each solve converged
    # to the same residual) from fewer sweeps.  Replaying the points separates the
    # warm start's effect from the optimiser's sensitivity to rounding-level changes.
    from paper_2609_31347_b300 import gbo, warmstart as W
    nx = 128
    Fstar = I.fourier_fields(1, nx, seed=21, kmax=4).reshape(-1).contiguous()
    s = lbm.LBMSolid(nx, nx, 1.0 / nx, E, NU)
    s.set_control(Fstar)
    s.primal_solve(4_000_000, tol=1e-12, criterion=1, check_every=64)
    dstar = s.displacement()
    s.close()
    pts, ref = [], []
    s = lbm.LBMSolid(nx, nx, 1.0 / nx, E, NU)
    s.set_target(dstar)
    fg = gbo.make_fg(s, gbo.SolveOpts(tol=1e-10), gbo.SolveOpts(tol=1e-10), project=True)

    def rec(a):
        pts.append(a.detach().clone())
        ref.append(fg(a))
        return ref[-1]
    r = gbo.lbfgs(rec, torch.zeros_like(Fstar), m_max=10, eps=1e-14)
    assert r.J < 1e-3 * ref[0][0]
    cold = s.sweeps["primal_solve"] + s.sweeps["adjoint_solve"]
    s.close()
    s = lbm.LBMSolid(nx, nx, 1.0 / nx, E, NU)
    s.set_target(dstar)
    fgw = gbo.make_fg(s, gbo.SolveOpts(tol=1e-10), gbo.SolveOpts(tol=1e-10), project=True,
                      warm=W.WarmStarter(nets["primal"][0], nets["adjoint"][0]))
    for a, (J, g) in zip(pts, ref):
        Jw, gw = fgw(a)
        assert abs(Jw - J) <= 1e-5 * J
        assert float((gw - g).abs().max()) <= 1e-3 * float(g.abs().max())
    warm = s.sweeps["primal_solve"] + s.sweeps["adjoint_solve"]
    s.close()
    assert warm <= 0.95 * cold, (cold, warm)
