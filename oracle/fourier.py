"""Exact periodic fixed point of the solid LBM, one wavevector at a time.

TEST INFRASTRUCTURE ONLY (part of the oracle).  On the periodic lattice the primal
step f_S <- S (A f_S + B g) has translation-invariant coefficients, so its steady
state (Eq. primal_fixed_point) decouples per discrete wavevector k:
    (I - P_k A) f^_S(k) = P_k B g^(k),  P_k = diag(exp(-2 pi i k.c_j / n)),
where A = dC/df_S and B = dC/dg are the (constant) Jacobians of the local collision
(Eq. local_collide).  The k = 0 mode is the rigid translation that the zero initial
state and a zero-mean force keep at zero (Section 2, compatibility).

This is an independent route to the state the time-stepping oracle converges to:
numpy linear algebra instead of stepping, so it pins the stepping, the streaming
direction and the index wrap, and it reaches N_x = 256 in seconds.
"""
from __future__ import annotations

import numpy as np

CX = np.array([1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 1, 0, -1, 1, 1, -1, -1])
THETA = 1.0 / 3.0


def moment_matrix(gamma: float = 0.0) -> np.ndarray:
    """Rows m10, m01, m11, m_s, m_d, m12, m21, m_f = m22 + gamma m_s (Appendix A.1)."""
    i, j = CX.astype(float), CY.astype(float)
    return np.vstack([i, j, i * j, i * i + j * j, i * i - j * j, i * j * j, i * i * j,
                      i * i * j * j + gamma * (i * i + j * j)])


def collision_affine(E: float, nu: float, gamma: float = 0.0):
    """(A, B) with C(f, g) = A f + B g (Section 3.1 collision, Table A.1)."""
    mu = E / (2 * (1 + nu))
    K = E / (2 * (1 - nu))
    tau = np.array([mu / THETA, 2 * K / (1 + THETA), 2 * mu / (1 - THETA), 0.5, 0.5, 0.5])
    w = 1.0 / (tau + 0.5)
    M = moment_matrix(gamma)
    Mi = np.linalg.inv(M)
    # moment-space map m^C = R m + G g:
    # m^C_10 = m10 + g_x, m^C_01 = m01 + g_y, m^C_b = (1-w_b) m_b + w_b m^eq_b,
    # m^eq_12 = theta (m10 + g_x/2), m^eq_21 = theta (m01 + g_y/2), others 0.
    R = np.zeros((8, 8))
    G = np.zeros((8, 2))
    R[0, 0] = R[1, 1] = 1.0
    G[0, 0] = G[1, 1] = 1.0
    for b in range(2, 8):
        R[b, b] = 1.0 - w[b - 2]
    R[5, 0] += w[3] * THETA
    G[5, 0] += w[3] * THETA * 0.5
    R[6, 1] += w[4] * THETA
    G[6, 1] += w[4] * THETA * 0.5
    return Mi @ R @ M, Mi @ G


def periodic_fixed_point(nx: int, E: float, nu: float, F: np.ndarray, ny: int | None = None):
    """Steady f_S (8, N) for a zero-mean force F (2, N) on the periodic grid, dx = 1/nx."""
    ny = nx if ny is None else ny
    dx = 1.0 / nx
    A, B = collision_affine(E, nu)
    g = (dx * dx) * np.asarray(F, dtype=np.float64).reshape(2, ny, nx)
    gh = np.fft.fft2(g, axes=(1, 2))  # (2, ny, nx)
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.fftfreq(nx) * nx
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    phase = np.exp(-2j * np.pi * (KX[..., None] * CX / nx + KY[..., None] * CY / ny))  # (ny,nx,8)
    Pa = phase[..., :, None] * A[None, None]  # P_k A
    lhs = np.eye(8)[None, None] - Pa
    rhs = phase * np.einsum("kc,cyx->yxk", B, gh)  # P_k B g^
    lhs[0, 0] = np.eye(8)
    rhs[0, 0] = 0.0
    fh = np.linalg.solve(lhs, rhs[..., None])[..., 0]  # (ny, nx, 8)
    f = np.fft.ifft2(np.moveaxis(fh, -1, 0), axes=(1, 2)).real
    return f.reshape(8, nx * ny)


def displacement(fS: np.ndarray, F: np.ndarray, dx: float) -> np.ndarray:
    """d = (m10 + g_x/2, m01 + g_y/2), g = dx^2 F (Eq. disp_from_moments)."""
    return np.vstack([CX @ fS, CY @ fS]) + 0.5 * dx * dx * np.asarray(F)


def stress(fS: np.ndarray, F: np.ndarray, dx: float, E: float, nu: float) -> np.ndarray:
    """Physical (s11, s22, s12) = -(bared second moments)/dx (Eq. stress_from_moments)."""
    A, B = collision_affine(E, nu)
    fC = A @ fS + B @ ((dx * dx) * np.asarray(F))
    M = moment_matrix()
    mb = 0.5 * (M @ fS + M @ fC)
    return np.vstack([-0.5 * (mb[3] + mb[4]), -0.5 * (mb[3] - mb[4]), -mb[2]]) / dx
