"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the lattice Boltzmann arithmetic: it only builds the data
the solver is given (body forces, target displacements, the elliptic-plate geometry
and its boundary data, material fields and random states).  Both the CUDA path and
the CPU oracle receive the same arrays from here.

Layout: node n = y*nx + x; two-component fields are (2, N) SoA arrays; link data is
(8, N) in the D2Q8 order Q of Eq. (direction_order).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

# D2Q8 velocities in the order Q (Eq. direction_order); geometry needs them to decide
# which links leave the domain.
CX = np.array([1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 1, 0, -1, 1, 1, -1, -1])

TWO_PI = 2.0 * np.pi


def lame(E, nu):
    """Plane-stress moduli (Eqs. lambda, mu, K): returns (mu, K)."""
    mu = E / (2.0 * (1.0 + nu))
    K = E / (2.0 * (1.0 - nu))
    return mu, K


def periodic_coords(nx: int):
    """Periodic unit square: x_i = i dx, dx = 1/nx (nodes at i = 0..nx-1)."""
    dx = 1.0 / nx
    i = np.arange(nx)
    X, Y = np.meshgrid(i * dx, i * dx, indexing="xy")
    return X.ravel(), Y.ravel(), dx


# ---- benchmarks (1)/(2): periodic manufactured solution (Section 4.2.1) -------------
PAPER_DELTA = (9e-4, 7e-4)
PAPER_E, PAPER_NU = 0.11, 0.8


def periodic_manufactured(nx: int, E=PAPER_E, nu=PAPER_NU, delta=PAPER_DELTA):
    """d* (Eq. disp_man_periodic), F* (Eq. force_man_periodic), sigma* (Eq. stress).

    Returns dict with dstar (2,N), Fstar (2,N), sigma (3,N: s11, s22, s12), dx.
    """
    X, Y, dx = periodic_coords(nx)
    d1, d2 = delta
    mu, K = lame(E, nu)
    c1, s1 = np.cos(TWO_PI * X), np.sin(TWO_PI * X)
    c2, s2 = np.cos(TWO_PI * Y), np.sin(TWO_PI * Y)
    dstar = np.vstack([d1 * c1 * s2, d2 * s1 * c2])
    Fstar = 4.0 * np.pi ** 2 * np.vstack([(K * (d1 + d2) + 2 * mu * d1) * c1 * s2,
                                          (K * (d1 + d2) + 2 * mu * d2) * s1 * c2])
    # gradients of d*
    du1dx = -TWO_PI * d1 * s1 * s2
    du1dy = TWO_PI * d1 * c1 * c2
    du2dx = TWO_PI * d2 * c1 * c2
    du2dy = -TWO_PI * d2 * s1 * s2
    sigma = _stress_from_grad(du1dx, du1dy, du2dx, du2dy, mu, K)
    return dict(dstar=dstar, Fstar=Fstar, sigma=sigma, dx=dx)


def _stress_from_grad(a11, a12, a21, a22, mu, K):
    """sigma = K div(d) I + mu [grad d + grad d^T - div(d) I] (Eq. stress).

    a_ij = d d_i / d x_j.  Returns (s11, s22, s12)."""
    div = a11 + a22
    s11 = K * div + mu * (2 * a11 - div)
    s22 = K * div + mu * (2 * a22 - div)
    s12 = mu * (a12 + a21)
    return np.vstack([s11, s22, s12])


def config_amplitudes(nx: int, alpha=(1.0, 0.5)):
    """Two-amplitude periodic workload with lambda = mu = 1 (E = 8/3, nu = 1/3, K = 2):
    u = (a1 sin2pix sin2piy, a2 cos2pix cos2piy) and its closed-form Navier-Cauchy force
    F = 4pi^2 ([2mu a1 + K(a1-a2)] sin sin, [2mu a2 - K(a1-a2)] cos cos).

    F is linear in (a1, a2): F = a1 Phi1 + a2 Phi2.  Returns dstar(alpha) (2,N), the
    basis (2, 2, N) = (Phi1, Phi2), dx, E, nu.
    """
    X, Y, dx = periodic_coords(nx)
    mu, K = 1.0, 2.0
    a1, a2 = alpha
    ss = np.sin(TWO_PI * X) * np.sin(TWO_PI * Y)
    cc = np.cos(TWO_PI * X) * np.cos(TWO_PI * Y)
    dstar = np.vstack([a1 * ss, a2 * cc])
    q = 4.0 * np.pi ** 2
    phi1 = q * np.vstack([(2 * mu + K) * ss, -K * cc])
    phi2 = q * np.vstack([-K * ss, (2 * mu + K) * cc])
    return dict(dstar=dstar, basis=np.stack([phi1, phi2]), dx=dx, E=8.0 / 3.0, nu=1.0 / 3.0)


def paper_scale_basis(Fstar):
    """Benchmark (1) control F = alpha o F* (Eq. control_param_periodic) written as a
    two-field basis: Phi1 = (F*_1, 0), Phi2 = (0, F*_2)."""
    z = np.zeros_like(Fstar[0])
    return np.stack([np.vstack([Fstar[0], z]), np.vstack([z, Fstar[1]])])


def fourier_force(nx: int, modes: int = 8, kmax: int = 4, seed: int = 1, ny: Optional[int] = None):
    """Smooth zero-mean random force: `modes` Fourier modes with wavevectors
    2pi (kx, ky), kx, ky in {1..kmax}, N(0,1) amplitudes for sin/cos x 2 components."""
    ny = nx if ny is None else ny
    rng = np.random.default_rng(seed)
    dx, dy = 1.0 / nx, 1.0 / ny
    x = np.arange(nx) * dx
    y = np.arange(ny) * dy
    X, Y = np.meshgrid(x, y, indexing="xy")
    F = np.zeros((2, ny, nx))
    for _ in range(modes):
        kx, ky = rng.integers(1, kmax + 1, size=2)
        amp = rng.standard_normal(4)
        ph = TWO_PI * (kx * X + ky * Y)
        F[0] += amp[0] * np.sin(ph) + amp[1] * np.cos(ph)
        F[1] += amp[2] * np.sin(ph) + amp[3] * np.cos(ph)
    F -= F.mean(axis=(1, 2), keepdims=True)  # exact compatibility (Section 2)
    return F.reshape(2, nx * ny)


def fourier_fields(count: int, nx: int, seed: int, modes: int = 8, kmax: int = 8,
                   unit_norm: bool = False, exponents=(1.0,), device: str = "cuda"):
    """`count` random zero-mean two-component fields on the periodic nx^2 grid, as a
    (count, 2, nx*nx) float64 torch tensor on `device` (the layout of a batch of equal
    lattices).  Each field is `modes` Fourier modes with wavevectors 2 pi (kx, ky),
    kx, ky in {-kmax..kmax} not both zero, and N(0, |k|^(-2p)) sin/cos amplitudes per
    component, the spectral exponent p drawn per field from `exponents` (p = 1: force-like
    fields; p = 3: displacement-like fields, as the response to a p = 1 force decays by
    two more powers).  unit_norm scales every field to Euclidean norm 1 over its 2N
    values."""
    import torch
    rng = np.random.default_rng(seed)
    k = rng.integers(-kmax, kmax + 1, size=(count, modes, 2))
    zero = (k[..., 0] == 0) & (k[..., 1] == 0)
    k[zero, 0] = 1
    p = rng.choice(np.asarray(exponents, dtype=float), size=(count, 1))
    amp = rng.standard_normal((count, modes, 4)) * \
        (np.hypot(k[..., 0], k[..., 1]) ** -p)[..., None]
    x = torch.arange(nx, dtype=torch.float64, device=device) / nx
    Y, X = torch.meshgrid(x, x, indexing="ij")
    kt = torch.as_tensor(k, dtype=torch.float64, device=device)
    at = torch.as_tensor(amp, dtype=torch.float64, device=device)
    out = torch.empty((count, 2, nx * nx), dtype=torch.float64, device=device)
    for b in range(count):
        ph = TWO_PI * (kt[b, :, 0, None, None] * X + kt[b, :, 1, None, None] * Y)  # (modes, nx, nx)
        s, c = torch.sin(ph), torch.cos(ph)
        a = at[b]
        out[b, 0] = (a[:, 0, None, None] * s + a[:, 1, None, None] * c).sum(0).reshape(-1)
        out[b, 1] = (a[:, 2, None, None] * s + a[:, 3, None, None] * c).sum(0).reshape(-1)
    out -= out.mean(dim=2, keepdim=True)
    if unit_norm:
        out /= torch.linalg.vector_norm(out, dim=(1, 2), keepdim=True)
    return out


def random_state(n: int, seed: int, scale: float = 1.0):
    """Random populations / adjoint states (8, n), N(0, scale^2)."""
    return np.random.default_rng(seed).standard_normal((8, n)) * scale


# ---- benchmark (3): elliptic plate (Section 4.3.1, Table ellipseparameter) ----------
# (a^2, b^2, x_c, y_c, phi) with L = 1
PLATE_ELLIPSES = (
    (0.48, 0.30, 0.750, 0.750, -np.pi / 9.0),  # outer (Neumann)
    (0.010, 0.018, 0.950, 0.600, 0.0),          # inner hole (Dirichlet)
    (0.035, 0.010, 0.500, 0.900, 0.0),          # inner hole (Dirichlet)
)
PLATE_E, PLATE_NU = 0.1, 0.7


def _ellipse_level(e, X, Y):
    """Level function xi1^2/a^2 + xi2^2/b^2 - 1 with xi = R(-phi)(x - x_c), and its
    gradient (for the outward normal)."""
    a2, b2, xc, yc, phi = e
    c, s = np.cos(phi), np.sin(phi)
    px, py = X - xc, Y - yc
    xi1 = c * px + s * py
    xi2 = -s * px + c * py
    lev = xi1 ** 2 / a2 + xi2 ** 2 / b2 - 1.0
    g1, g2 = 2 * xi1 / a2, 2 * xi2 / b2
    gx = c * g1 - s * g2  # R(phi) (g1, g2)
    gy = s * g1 + c * g2
    return lev, gx, gy


def plate_manufactured(X, Y, E=PLATE_E, nu=PLATE_NU, delta=PAPER_DELTA):
    """d* (Eq. disp_man_ellipse), sigma* (Eq. stress) and F* = -mu lap d* - K grad div d*.

    Closed-form derivatives of d* = (d1 sin(2 pi x y), d2 cos(2 pi y)(1 + x^2))."""
    d1, d2 = delta
    mu, K = lame(E, nu)
    p = TWO_PI
    sxy, cxy = np.sin(p * X * Y), np.cos(p * X * Y)
    cy, sy = np.cos(p * Y), np.sin(p * Y)
    dstar = np.vstack([d1 * sxy, d2 * cy * (1 + X ** 2)])
    a11 = d1 * p * Y * cxy
    a12 = d1 * p * X * cxy
    a21 = d2 * cy * 2 * X
    a22 = -d2 * p * sy * (1 + X ** 2)
    sigma = _stress_from_grad(a11, a12, a21, a22, mu, K)
    # second derivatives
    u_xx = -d1 * p * p * Y * Y * sxy
    u_yy = -d1 * p * p * X * X * sxy
    u_xy = d1 * p * cxy - d1 * p * p * X * Y * sxy
    v_xx = 2 * d2 * cy
    v_yy = -d2 * p * p * cy * (1 + X ** 2)
    v_xy = -d2 * p * sy * 2 * X
    # F = -mu lap d - K grad(div d)
    Fx = -mu * (u_xx + u_yy) - K * (u_xx + v_xy)
    Fy = -mu * (v_xx + v_yy) - K * (u_xy + v_yy)
    return dstar, sigma, np.vstack([Fx, Fy])


@dataclass
class PlateGeometry:
    nx: int                 # nodes per direction (N_x + 1 in the paper's notation)
    dx: float
    X: np.ndarray
    Y: np.ndarray
    active: np.ndarray      # (N,) uint8: node inside Omega^E
    link: np.ndarray        # (8, N) uint8: 0 regular, 1 Dirichlet-missing, 2 Neumann-missing
    node_type: np.ndarray   # (N,) uint8: 0 outside, 1 interior, 2 boundary
    normal: np.ndarray      # (2, N) outward unit normal of the outer ellipse (boundary nodes)
    normal_hole: Optional[np.ndarray] = None  # (2, N) normal into the nearest hole (out of Omega^E)


def plate_geometry(Nx: int, ellipses=PLATE_ELLIPSES, box: float = 1.5) -> PlateGeometry:
    """Lattice of N_x + 1 nodes per direction on [0, box]^2 (Section 4.3.1): Omega^E is
    inside ellipse 1 and outside ellipses 2, 3.  A link k of an active node n is missing
    when its source node n - c_k is not active; it is Dirichlet when that source lies
    inside an inner ellipse and Neumann otherwise (outside the outer ellipse)."""
    nx = Nx + 1
    dx = box / Nx
    i = np.arange(nx)
    Xg, Yg = np.meshgrid(i * dx, i * dx, indexing="xy")
    X, Y = Xg.ravel(), Yg.ravel()
    lev = [_ellipse_level(e, X, Y) for e in ellipses]
    inside_outer = lev[0][0] <= 0.0
    in_hole = np.zeros_like(inside_outer)
    for (l, _, _) in lev[1:]:
        in_hole |= l <= 0.0
    active = (inside_outer & ~in_hole).astype(np.uint8)
    N = nx * nx
    link = np.zeros((8, N), dtype=np.uint8)
    xi, yi = np.arange(N) % nx, np.arange(N) // nx
    for k in range(8):
        xs, ys = xi - CX[k], yi - CY[k]
        ok = (xs >= 0) & (xs < nx) & (ys >= 0) & (ys < nx)
        src = np.where(ok, ys * nx + xs, 0)
        src_active = ok & (active[src] == 1)
        missing = (active == 1) & ~src_active
        src_hole = ok & in_hole[src]
        link[k][missing & src_hole] = 1
        link[k][missing & ~src_hole] = 2
    node_type = active.copy()
    node_type[(active == 1) & (link != 0).any(axis=0)] = 2
    _, gx, gy = lev[0]
    gn = np.sqrt(gx * gx + gy * gy)
    gn[gn == 0] = 1.0
    normal = np.vstack([gx / gn, gy / gn])
    # normal into the nearest inner ellipse (the outward normal of Omega^E at the holes)
    hl, hx, hy = lev[1]
    for (l2, gx2, gy2) in lev[2:]:
        m = l2 < hl
        hl, hx, hy = np.where(m, l2, hl), np.where(m, gx2, hx), np.where(m, gy2, hy)
    hn = np.sqrt(hx * hx + hy * hy)
    hn[hn == 0] = 1.0
    normal_hole = np.vstack([-hx / hn, -hy / hn])
    return PlateGeometry(nx, dx, X, Y, active, link, node_type, normal, normal_hole)


def plate_wall_data(geo: PlateGeometry, E=PLATE_E, nu=PLATE_NU, delta=PAPER_DELTA):
    """Per-node wall data of the manufactured solution, evaluated where the halfway-wall
    boundary rules place the wall: half a cell outward from the node along the outward
    normal of Omega^E.  Dirichlet: d_D = d*(x_n + dx/2 n_hole); Neumann:
    T = sigma*(x_n + dx/2 n) n with n the outer ellipse's outward normal."""
    h = 0.5 * geo.dx
    nh = geo.normal_hole
    dD, _, _ = plate_manufactured(geo.X + h * nh[0], geo.Y + h * nh[1], E=E, nu=nu, delta=delta)
    _, sN, _ = plate_manufactured(geo.X + h * geo.normal[0], geo.Y + h * geo.normal[1], E=E,
                                  nu=nu, delta=delta)
    T = np.vstack([sN[0] * geo.normal[0] + sN[2] * geo.normal[1],
                   sN[2] * geo.normal[0] + sN[1] * geo.normal[1]])
    return dD, T


def baseline_plate(Nx: int, traction: float = 0.01):
    """Clamped-left / uniform-tension plate: ellipse with semi-axes 1.0 and 0.5 centred
    in a [0, 2.2] x [0, 1.2] box is not square, so it is embedded in a square box of
    side 2.2 with N_x + 1 nodes per direction.  Dirichlet d = 0 on boundary links whose
    outward normal has n_x <= -1/2 (the left arc); Neumann T = traction * n elsewhere.
    Zero body force.  Returns geometry and wall data (the target is a solve at E_ref)."""
    box = 2.2
    e = (1.0, 0.25, 1.1, 1.1, 0.0)
    nx = Nx + 1
    dx = box / Nx
    i = np.arange(nx)
    Xg, Yg = np.meshgrid(i * dx, i * dx, indexing="xy")
    X, Y = Xg.ravel(), Yg.ravel()
    lev, gx, gy = _ellipse_level(e, X, Y)
    active = (lev <= 0.0).astype(np.uint8)
    gn = np.sqrt(gx * gx + gy * gy)
    gn[gn == 0] = 1.0
    normal = np.vstack([gx / gn, gy / gn])
    N = nx * nx
    link = np.zeros((8, N), dtype=np.uint8)
    xi, yi = np.arange(N) % nx, np.arange(N) // nx
    left = normal[0] <= -0.5
    for k in range(8):
        xs, ys = xi - CX[k], yi - CY[k]
        ok = (xs >= 0) & (xs < nx) & (ys >= 0) & (ys < nx)
        src = np.where(ok, ys * nx + xs, 0)
        src_active = ok & (active[src] == 1)
        missing = (active == 1) & ~src_active
        link[k][missing & left] = 1
        link[k][missing & ~left] = 2
    node_type = active.copy()
    node_type[(active == 1) & (link != 0).any(axis=0)] = 2
    geo = PlateGeometry(nx, dx, X, Y, active, link, node_type, normal)
    wall_d = np.zeros((2, N))
    wall_T = traction * normal
    return geo, wall_d, wall_T


def lognormal_E(N: int, E_ref: float = 1.0, sigma: float = 0.2, seed: int = 0):
    """Mean-preserving lognormal per-node modulus E_n = E_ref exp(sigma z - sigma^2/2)."""
    z = np.random.default_rng(seed).standard_normal(N)
    return E_ref * np.exp(sigma * z - 0.5 * sigma * sigma)
