"""Oracle pins: moment matrix, material map and one local collision (CPU only).

Each check compares the oracle with something fixed outside it: the matrix printed
in Appendix A.1, the raw-moment definition m_ab = sum i^a j^b f (Eq. moments), the
relaxation rules (Eqs. moments_c, moments_bar_1/2, moments_c_10/01, Table A.1) read
off the output populations with an independent moment sum, and closed-form
special cases of the plane-stress moduli.
"""
import numpy as np
import pytest

import oracle
from tests.conftest import golden

CX = np.array([1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 1, 0, -1, 1, 1, -1, -1])


def raw(f, a, b):
    return float(np.sum((CX ** a) * (CY ** b) * f))


def test_moment_matrix_is_the_printed_one():
    M, Mi = oracle.moment_matrix(0.0)
    g = golden("moment_matrix.txt")
    printed = np.array([g["row%d" % r] for r in range(8)])
    assert np.array_equal(M, printed)
    assert np.allclose(M @ Mi, np.eye(8), atol=1e-15)


@pytest.mark.parametrize("gamma", [-0.5, 0.25, 1.0])
def test_gamma_row(gamma):
    # Appendix A.1: the last row becomes (g, g, g, g, 1+2g, 1+2g, 1+2g, 1+2g)
    M, Mi = oracle.moment_matrix(gamma)
    assert np.allclose(M[7], [gamma] * 4 + [1 + 2 * gamma] * 4, atol=0)
    M0, _ = oracle.moment_matrix(0.0)
    assert np.array_equal(M[:7], M0[:7])
    assert np.allclose(M @ Mi, np.eye(8), atol=1e-14)


def test_paper_plate_gamma_and_conditioning():
    # E = 0.1, nu = 0.7 (Section 4.3.1): K = 1/6, tau_s = 1/4, gamma = -1/2 and the
    # last row (-1/2, ..., 0, ...) still gives an invertible M.
    w, gb = oracle.material(0.1, 0.7)
    assert gb == pytest.approx(-0.5, rel=1e-14)
    M, _ = oracle.moment_matrix(gb)
    assert np.allclose(M[7], [-0.5] * 4 + [0.0] * 4)
    assert np.linalg.cond(M) < 10.0


def test_material_closed_forms():
    # lambda = mu = 1 <=> nu = 1/3, E = 8/3 (plane stress): K = 2, tau_11 = mu/theta = 3,
    # tau_s = 2K/(1+theta) = 3, tau_d = 2mu/(1-theta) = 3 -> omega = 1/(3 + 1/2).
    w, gb = oracle.material(8.0 / 3.0, 1.0 / 3.0)
    assert np.allclose(w[:3], 1.0 / 3.5, rtol=1e-14)
    assert np.allclose(w[3:], 1.0, rtol=0)  # tau_12 = tau_21 = tau_f = 1/2
    # gamma = theta tau_f / ((1+theta)(tau_s - tau_f)) = (1/6)/((4/3)(5/2)) = 1/20
    assert gb == pytest.approx(1.0 / 20.0, rel=1e-14)
    with pytest.raises(ValueError):
        oracle.material(-1.0, 0.3)
    # tau_s = 1/2 makes gamma singular: K = 1/3 -> E = 2K(1-nu)
    with pytest.raises(ValueError):
        oracle.material(2.0 / 3.0 * (1 - 0.5), 0.5)


@pytest.mark.parametrize("boundary", [False, True])
def test_collision_follows_the_moment_rules(boundary):
    rng = np.random.default_rng(7)
    E, nu = 0.37, 0.21
    mu, K = E / (2 * (1 + nu)), E / (2 * (1 - nu))
    th = 1.0 / 3.0
    tau = {"11": mu / th, "s": 2 * K / (1 + th), "d": 2 * mu / (1 - th)}
    w = {b: 1.0 / (t + 0.5) for b, t in tau.items()}
    _, gb = oracle.material(E, nu)
    gam = gb if boundary else 0.0
    for _ in range(5):
        f = rng.standard_normal(8)
        gx, gy = rng.standard_normal(2)
        c = oracle.collide(E, nu, f, gx, gy, boundary=boundary)
        m10, m01 = raw(f, 1, 0), raw(f, 0, 1)
        b10, b01 = m10 + gx / 2, m01 + gy / 2
        # first-order moments: second half of the force (Eqs. moments_c_10/01)
        assert raw(c, 1, 0) == pytest.approx(b10 + gx / 2, abs=1e-13)
        assert raw(c, 0, 1) == pytest.approx(b01 + gy / 2, abs=1e-13)
        # relaxed second-order moments towards zero equilibrium
        assert raw(c, 1, 1) == pytest.approx((1 - w["11"]) * raw(f, 1, 1), abs=1e-13)
        ms, md = raw(f, 2, 0) + raw(f, 0, 2), raw(f, 2, 0) - raw(f, 0, 2)
        assert raw(c, 2, 0) + raw(c, 0, 2) == pytest.approx((1 - w["s"]) * ms, abs=1e-13)
        assert raw(c, 2, 0) - raw(c, 0, 2) == pytest.approx((1 - w["d"]) * md, abs=1e-13)
        # omega_12 = omega_21 = omega_f = 1: third-order moments set to theta * bared
        assert raw(c, 1, 2) == pytest.approx(th * b10, abs=1e-13)
        assert raw(c, 2, 1) == pytest.approx(th * b01, abs=1e-13)
        # m_f^C = 0 -> m22^C = -gamma m_s^C
        assert raw(c, 2, 2) == pytest.approx(-gam * (1 - w["s"]) * ms, abs=1e-13)


def test_equilibrium_is_a_fixed_point_without_force():
    # f^eq = M^-1 N d: collision with g = 0 leaves it unchanged (m^eq = m).
    E, nu = 0.11, 0.8
    _, Mi = oracle.moment_matrix(0.0)
    for d in ([1.0, 0.0], [0.3, -0.7]):
        m = np.array([d[0], d[1], 0, 0, 0, d[0] / 3, d[1] / 3, 0])
        feq = Mi @ m
        assert np.allclose(oracle.collide(E, nu, feq, 0.0, 0.0), feq, atol=1e-15)
