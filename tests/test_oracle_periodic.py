"""Oracle pins on the periodic benchmarks (Section 4.2), CPU only.

- time stepping agrees with the exact per-wavevector fixed point (two independent
  routes to Eq. primal_fixed_point);
- the steady solution converges to the manufactured solution with the printed EOCs
  (Section 4.2.2: 1.99 / 1.99 / 2.00 / 2.00);
- a single-wavenumber force gives a single-wavenumber response (Section 4.2.3);
- the convergence monitor is Eq. (convergence).
"""
import numpy as np
import pytest

import oracle
from oracle import fourier
from paper_2609_31347_b300 import inputs as I
from tests.conftest import golden


@pytest.mark.parametrize("nx,E,nu,seed", [(8, 1.0, 0.3, 1), (10, 0.11, 0.8, 2), (7, 0.5, -0.2, 3)])
def test_stepping_matches_fourier_fixed_point(nx, E, nu, seed):
    F = I.fourier_force(nx, seed=seed, kmax=3)
    g = oracle.Grid(nx, nx, 1.0 / nx, nu)
    mu = E / (2 * (1 + nu))
    steps = int(60.0 / (mu * (2 * np.pi) ** 2) * nx * nx) + 200  # ~60 e-folds of the slowest mode
    fS = oracle.primal(g, E, F, steps)
    fF = fourier.periodic_fixed_point(nx, E, nu, F)
    assert np.abs(fS - fF).max() <= 1e-12 * np.abs(fF).max()


def _errors(nx, fS):
    m = I.periodic_manufactured(nx)
    d = fourier.displacement(fS, m["Fstar"], m["dx"])
    s = fourier.stress(fS, m["Fstar"], m["dx"], I.PAPER_E, I.PAPER_NU)
    fro = oracle.stress_frobenius_rows
    return (oracle.norm_L2(d - m["dstar"], m["dx"]) / oracle.norm_L2(m["dstar"], m["dx"]),
            oracle.norm_Linf(d - m["dstar"]) / oracle.norm_Linf(m["dstar"]),
            oracle.norm_L2(fro(s - m["sigma"]), m["dx"]) / oracle.norm_L2(fro(m["sigma"]), m["dx"]),
            oracle.norm_Linf(s - m["sigma"]) / oracle.norm_Linf(m["sigma"]))


def test_primal_eoc_matches_the_paper():
    gd = golden("periodic_primal_eoc.txt")
    nxs = [int(v) for v in gd["nx"]]
    errs = []
    for nx in nxs:
        m = I.periodic_manufactured(nx)
        fS = fourier.periodic_fixed_point(nx, I.PAPER_E, I.PAPER_NU, m["Fstar"])
        errs.append(_errors(nx, fS))
    errs = np.array(errs)
    for col, key in enumerate(["eoc_d_L2", "eoc_d_Linf", "eoc_sigma_L2", "eoc_sigma_Linf"]):
        eoc = oracle.eoc(nxs, errs[:, col])
        # printed to two decimals
        assert abs(eoc - gd[key][0]) <= 0.0101, (key, eoc)


def test_time_stepped_oracle_at_32_reproduces_the_fixed_point_errors():
    # Section 4.2.2 protocol: 30 N_x^2 steps from f_S = 0.
    nx = 32
    m = I.periodic_manufactured(nx)
    g = oracle.Grid(nx, nx, m["dx"], I.PAPER_NU)
    fS = oracle.primal(g, I.PAPER_E, m["Fstar"], 30 * nx * nx)
    fF = fourier.periodic_fixed_point(nx, I.PAPER_E, I.PAPER_NU, m["Fstar"])
    e_step, e_fix = _errors(nx, fS), _errors(nx, fF)
    assert np.allclose(e_step, e_fix, rtol=1e-9)
    # and the oracle's own displacement / stress routines agree with the fixed point's
    d = oracle.displacement(g, fS, m["Fstar"])
    assert np.allclose(d, fourier.displacement(fS, m["Fstar"], m["dx"]), atol=1e-18)
    s = oracle.stress(g, I.PAPER_E, fS, m["Fstar"])
    assert np.allclose(s, fourier.stress(fS, m["Fstar"], m["dx"], I.PAPER_E, I.PAPER_NU),
                       rtol=1e-12, atol=1e-16)


def test_single_wavenumber_is_preserved():
    # Section 4.2.3: a single-wavenumber force leaves a response that differs from d*
    # only by the amplitudes of its two components, with an O(dx^2) amplitude error.
    amp_err = []
    for nx in (10, 20, 40):
        m = I.periodic_manufactured(nx)
        fS = fourier.periodic_fixed_point(nx, I.PAPER_E, I.PAPER_NU, m["Fstar"])
        d = fourier.displacement(fS, m["Fstar"], m["dx"])
        errs = []
        for c in range(2):
            a = d[c] @ m["dstar"][c] / (m["dstar"][c] @ m["dstar"][c])
            assert np.abs(d[c] - a * m["dstar"][c]).max() <= 1e-13 * np.abs(d[c]).max()
            errs.append(abs(a - 1.0))
        amp_err.append(max(errs))
    assert 3.5 < amp_err[0] / amp_err[1] < 4.5 and 3.5 < amp_err[1] / amp_err[2] < 4.5


@pytest.mark.parametrize("axis", [0, 1])
def test_half_nyquist_force_is_never_damped(axis):
    # Degenerate case of the periodic scheme (Section 3.1 collision with omega_12 =
    # omega_21 = omega_f = 1, no rest population): at the wavevectors (N/2, 0) and
    # (0, N/2) one step multiplies a collision invariant by -1 under streaming, so the
    # iteration has the eigenvalue -1 there.  A force with that content is never
    # converged by iterating: the iterates alternate about the fixed point, which is
    # still well defined (I - P A has the eigenvalue 2 there) and is their average.
    nx, E, nu = 8, 8.0 / 3.0, 1.0 / 3.0
    g = oracle.Grid(nx, nx, 1.0 / nx, nu)
    i = np.arange(nx)
    X, Y = np.meshgrid(i, i, indexing="xy")
    F = np.zeros((2, nx * nx))
    F[axis] = ((-1.0) ** (X if axis == 0 else Y)).ravel()  # zero mean
    f = [oracle.primal(g, E, F, T) for T in (300, 301, 302)]
    scale = np.abs(f[1]).max()
    assert np.abs(f[2] - f[0]).max() <= 1e-12 * scale       # period two ...
    assert np.abs(f[1] - f[0]).max() >= 0.5 * scale          # ... and no decay
    fp = fourier.periodic_fixed_point(nx, E, nu, F)
    assert np.abs(0.5 * (f[0] + f[1]) - fp).max() <= 1e-12 * scale
    # any smooth force on the same grid converges
    Fs = I.fourier_force(nx, seed=3, kmax=2)
    a, b = oracle.primal(g, E, Fs, 400), oracle.primal(g, E, Fs, 401)
    assert np.abs(b - a).max() <= 1e-13 * np.abs(b).max()


def test_states_are_linear_in_the_force_and_the_tangent_is_a_primal():
    # From f_S(0) = 0 the periodic step is linear in the force (Section 3.1: affine
    # collision, permutation streaming), so the state after T steps for a1 F1 + a2 F2 is
    # a1 f(F1) + a2 f(F2), and the forward-mode tangent along a force direction Fd (at
    # any F, the modulus fixed) is the primal state driven by Fd alone.
    nx, T = 10, 150
    g = oracle.Grid(nx, nx, 1.0 / nx, 1.0 / 3.0)
    E = 8.0 / 3.0
    F1 = I.fourier_force(nx, seed=11, kmax=3)
    F2 = I.fourier_force(nx, seed=12, kmax=3)
    f1, f2 = oracle.primal(g, E, F1, T), oracle.primal(g, E, F2, T)
    f12 = oracle.primal(g, E, 0.7 * F1 - 1.3 * F2, T)
    scale = np.abs(f12).max()
    assert np.abs(f12 - (0.7 * f1 - 1.3 * f2)).max() <= 1e-13 * scale
    _, fd = oracle.primal_tangent(g, E, F1, T, Fdot=F2)
    assert np.abs(fd - f2).max() <= 1e-13 * np.abs(f2).max()


def test_monitor_is_mean_squared_displacement():
    nx = 6
    rng = np.random.default_rng(0)
    fS = rng.standard_normal((8, nx * nx))
    F = rng.standard_normal((2, nx * nx))
    g = oracle.Grid(nx, nx, 1.0 / nx, 0.3)
    d = fourier.displacement(fS, F, 1.0 / nx)
    assert oracle.monitor(g, fS, F) == pytest.approx(np.mean(d[0] ** 2 + d[1] ** 2), rel=1e-14)


def test_force_closed_form_is_navier_cauchy():
    # Eq. force_man_periodic equals -mu lap d* - K grad div d* (spectral derivatives
    # of the sampled d* are exact for this single mode).
    nx = 16
    m = I.periodic_manufactured(nx)
    mu, K = I.lame(I.PAPER_E, I.PAPER_NU)
    k = 2 * np.pi * np.fft.fftfreq(nx) * nx
    KY, KX = np.meshgrid(k, k, indexing="ij")

    def der(f, ax, ay):
        fh = np.fft.fft2(f.reshape(nx, nx))
        return np.fft.ifft2(fh * (1j * KX) ** ax * (1j * KY) ** ay).real.ravel()

    u, v = m["dstar"]
    Fx = -mu * (der(u, 2, 0) + der(u, 0, 2)) - K * (der(u, 2, 0) + der(v, 1, 1))
    Fy = -mu * (der(v, 2, 0) + der(v, 0, 2)) - K * (der(u, 1, 1) + der(v, 0, 2))
    assert np.allclose(np.vstack([Fx, Fy]), m["Fstar"], atol=1e-12)
    s11 = K * (der(u, 1, 0) + der(v, 0, 1)) + mu * (der(u, 1, 0) - der(v, 0, 1))
    s12 = mu * (der(u, 0, 1) + der(v, 1, 0))
    assert np.allclose(s11, m["sigma"][0], atol=1e-14)
    assert np.allclose(s12, m["sigma"][2], atol=1e-14)
