"""CPU FP64 oracle for the solid LBM, its discrete adjoint and gradients.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the product path (the CUDA library and
its Python binding) never does.  The oracle shares no code with the CUDA path.

The C++ core (``lbm_oracle.cpp``) follows the paper step by step (Section 3.1
collision/streaming, Section 3.2 objective, Section 3.3.2 adjoint, Eq. optimality,
Section 3.3.1 f-AD).  ``fourier.py`` adds the exact periodic fixed point per
wavevector.  This module is a ctypes wrapper plus the build step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.cpp")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (g++, -O2, OpenMP, no fast-math) into oracle/liblbm_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h"))
    ):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
             "-ffp-contract=off", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I, D, L = ctypes.c_int, ctypes.c_double, ctypes.c_long
        sig = {
            "orc_moment_matrix": [D, P, P],
            "orc_material": [D, D, P, P],
            "orc_collide": [D, D, I, P, D, D, P],
            "orc_primal": [P, P, P, P, L, P, P],
            "orc_primal_tangent": [P, P, P, P, P, L, P, P],
            "orc_objective": [P, P, P, P, P, P, P],
            "orc_objective_tangent": [P, P, P, P, P, P, P, P, P],
            "orc_displacement": [P, P, P, P],
            "orc_stress": [P, P, P, P, P],
            "orc_monitor": [P, P, P, P],
            "orc_primal_trace": [P, P, P, L, P],
            "orc_adjoint_trace": [P, P, P, P, P, P, L, P],
            "orc_set_threads": [I],
            "orc_threads": [],
            "orc_apply_step": [P, P, P, P],
            "orc_apply_step_transpose": [P, P, P, P],
            "orc_adjoint": [P, P, P, P, P, P, L, P, P],
            "orc_gradient_force": [P, P, P, P, P, P, P, P],
            "orc_gradient_young": [P, P, P, P, P, P, P, P],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = I
        lib.orc_cv_stop.argtypes = [P, L, L, D, P]
        lib.orc_cv_stop.restype = L
        _lib = lib
    return _lib


class _CGrid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("periodic", ctypes.c_int),
        ("dx", ctypes.c_double), ("nu", ctypes.c_double),
        ("node_type", ctypes.c_void_p), ("link", ctypes.c_void_p),
        ("wall_d", ctypes.c_void_p), ("wall_T", ctypes.c_void_p), ("wall_n", ctypes.c_void_p),
    ]


@dataclass
class Grid:
    """Lattice description.  Periodic grids leave the bounded-domain fields None.

    node_type: (N,) uint8, 0 outside / 1 interior / 2 boundary.
    link: (8, N) uint8, 0 regular / 1 Dirichlet-missing / 2 Neumann-missing.
    wall_d, wall_T, wall_n: (2, N) float64 (Dirichlet data, traction, outward normal).
    """
    nx: int
    ny: int
    dx: float
    nu: float
    periodic: bool = True
    node_type: Optional[np.ndarray] = None
    link: Optional[np.ndarray] = None
    wall_d: Optional[np.ndarray] = None
    wall_T: Optional[np.ndarray] = None
    wall_n: Optional[np.ndarray] = None

    @property
    def N(self) -> int:
        return self.nx * self.ny

    def _c(self):
        keep = []

        def ptr(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a.ctypes.data

        cg = _CGrid(self.nx, self.ny, 1 if self.periodic else 0, float(self.dx), float(self.nu),
                    ptr(self.node_type, np.uint8), ptr(self.link, np.uint8),
                    ptr(self.wall_d, np.float64), ptr(self.wall_T, np.float64),
                    ptr(self.wall_n, np.float64))
        return cg, keep


def _arr(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _E(grid: Grid, E):
    E = np.asarray(E, dtype=np.float64)
    if E.ndim == 0:
        E = np.full(grid.N, float(E))
    return _arr(E, grid.N)


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with code %d" % (what, rc))


def moment_matrix(gamma: float = 0.0):
    M = np.zeros(64)
    Mi = np.zeros(64)
    rc = _load().orc_moment_matrix(float(gamma), M.ctypes.data, Mi.ctypes.data)
    _check(rc, "moment_matrix")
    return M.reshape(8, 8), Mi.reshape(8, 8)


def material(E: float, nu: float):
    w = np.zeros(6)
    gb = ctypes.c_double()
    rc = _load().orc_material(float(E), float(nu), w.ctypes.data, ctypes.addressof(gb))
    _check(rc, "material")
    return w, gb.value


def collide(E, nu, fS8, gx, gy, boundary=False):
    f = _arr(fS8, 8)
    out = np.zeros(8)
    rc = _load().orc_collide(float(E), float(nu), 1 if boundary else 0, f.ctypes.data,
                             float(gx), float(gy), out.ctypes.data)
    _check(rc, "collide")
    return out


def primal(grid: Grid, E, F, steps: int, fS0=None, return_fC: bool = False):
    """f_S after `steps` collide+stream steps from f_S(0) = fS0 (default 0).  (8, N)."""
    cg, keep = grid._c()
    N = grid.N
    E = _E(grid, E)
    F = _arr(F, 2 * N)
    f0 = None if fS0 is None else _arr(fS0, 8 * N)
    fS = np.zeros(8 * N)
    fC = np.zeros(8 * N) if return_fC else None
    rc = _load().orc_primal(ctypes.byref(cg), E.ctypes.data, F.ctypes.data,
                            None if f0 is None else f0.ctypes.data, int(steps), fS.ctypes.data,
                            None if fC is None else fC.ctypes.data)
    _check(rc, "primal")
    if return_fC:
        return fS.reshape(8, N), fC.reshape(8, N)
    return fS.reshape(8, N)


def primal_tangent(grid: Grid, E, F, steps: int, Edot=None, Fdot=None):
    """f-AD: (f_S, df_S) for the seeds Edot (N) and Fdot (2N)."""
    cg, keep = grid._c()
    N = grid.N
    E = _E(grid, E)
    F = _arr(F, 2 * N)
    Ed = None if Edot is None else _E(grid, Edot)
    Fd = None if Fdot is None else _arr(Fdot, 2 * N)
    fS = np.zeros(8 * N)
    fSd = np.zeros(8 * N)
    rc = _load().orc_primal_tangent(ctypes.byref(cg), E.ctypes.data,
                                    None if Ed is None else Ed.ctypes.data, F.ctypes.data,
                                    None if Fd is None else Fd.ctypes.data, int(steps),
                                    fS.ctypes.data, fSd.ctypes.data)
    _check(rc, "primal_tangent")
    return fS.reshape(8, N), fSd.reshape(8, N)


def objective(grid: Grid, fS, F, dstar, obs=None):
    cg, keep = grid._c()
    N = grid.N
    fS, F, ds = _arr(fS, 8 * N), _arr(F, 2 * N), _arr(dstar, 2 * N)
    ob = None if obs is None else _arr(obs, N)
    J, C = ctypes.c_double(), ctypes.c_double()
    rc = _load().orc_objective(ctypes.byref(cg), fS.ctypes.data, F.ctypes.data, ds.ctypes.data,
                               None if ob is None else ob.ctypes.data, ctypes.addressof(J),
                               ctypes.addressof(C))
    _check(rc, "objective")
    return J.value, C.value


def objective_tangent(grid: Grid, fS, fSdot, F, dstar, Fdot=None, obs=None):
    cg, keep = grid._c()
    N = grid.N
    fS, fSd, F, ds = _arr(fS, 8 * N), _arr(fSdot, 8 * N), _arr(F, 2 * N), _arr(dstar, 2 * N)
    Fd = None if Fdot is None else _arr(Fdot, 2 * N)
    ob = None if obs is None else _arr(obs, N)
    J, Jd = ctypes.c_double(), ctypes.c_double()
    rc = _load().orc_objective_tangent(ctypes.byref(cg), fS.ctypes.data, fSd.ctypes.data,
                                       F.ctypes.data, None if Fd is None else Fd.ctypes.data,
                                       ds.ctypes.data, None if ob is None else ob.ctypes.data,
                                       ctypes.addressof(J), ctypes.addressof(Jd))
    _check(rc, "objective_tangent")
    return J.value, Jd.value


def displacement(grid: Grid, fS, F):
    cg, keep = grid._c()
    N = grid.N
    fS, F = _arr(fS, 8 * N), _arr(F, 2 * N)
    d = np.zeros(2 * N)
    _check(_load().orc_displacement(ctypes.byref(cg), fS.ctypes.data, F.ctypes.data,
                                    d.ctypes.data), "displacement")
    return d.reshape(2, N)


def stress(grid: Grid, E, fS, F):
    """Physical stress (sigma11, sigma22, sigma12), (3, N)."""
    cg, keep = grid._c()
    N = grid.N
    E = _E(grid, E)
    fS, F = _arr(fS, 8 * N), _arr(F, 2 * N)
    s = np.zeros(3 * N)
    _check(_load().orc_stress(ctypes.byref(cg), E.ctypes.data, fS.ctypes.data, F.ctypes.data,
                              s.ctypes.data), "stress")
    return s.reshape(3, N)


def monitor(grid: Grid, fS, F):
    cg, keep = grid._c()
    N = grid.N
    fS, F = _arr(fS, 8 * N), _arr(F, 2 * N)
    c = ctypes.c_double()
    _check(_load().orc_monitor(ctypes.byref(cg), fS.ctypes.data, F.ctypes.data,
                               ctypes.addressof(c)), "monitor")
    return c.value


def primal_trace(grid: Grid, E, F, steps: int):
    """c(t) of Eq. (convergence) for t = 0 .. steps of the primal from rest, (steps+1,)."""
    cg, keep = grid._c()
    E, F = _E(grid, E), _arr(F, 2 * grid.N)
    c = np.zeros(int(steps) + 1)
    _check(_load().orc_primal_trace(ctypes.byref(cg), E.ctypes.data, F.ctypes.data,
                                    int(steps), c.ctypes.data), "primal_trace")
    return c


def adjoint_trace(grid: Grid, E, F, fS, dstar, steps: int, obs=None):
    """c of the adjoint displacement of phi_S(i), i = 0 .. steps, (steps+1,)."""
    cg, keep = grid._c()
    N = grid.N
    E, F, fS, ds = _E(grid, E), _arr(F, 2 * N), _arr(fS, 8 * N), _arr(dstar, 2 * N)
    ob = None if obs is None else _arr(obs, N)
    c = np.zeros(int(steps) + 1)
    _check(_load().orc_adjoint_trace(ctypes.byref(cg), E.ctypes.data, F.ctypes.data,
                                     fS.ctypes.data, ds.ctypes.data,
                                     None if ob is None else ob.ctypes.data, int(steps),
                                     c.ctypes.data), "adjoint_trace")
    return c


def cv_stop(samples, window: int, tol: float):
    """Eq. (convergence_crit) on a sample sequence: (first index where the trailing
    window's std/mean < tol, or -1; last CV evaluated)."""
    c = _arr(samples)
    m = ctypes.c_double(float("nan"))
    i = _load().orc_cv_stop(c.ctypes.data, c.size, int(window), float(tol), ctypes.addressof(m))
    if i < -1:
        raise ValueError("cv_stop: bad input")
    return int(i), m.value


def set_threads(n: int = 0) -> int:
    """OpenMP threads of the oracle's node loops (0 = all processors); results do not
    depend on it."""
    return int(_load().orc_set_threads(int(n)))


def threads() -> int:
    return int(_load().orc_threads())


def apply_step(grid: Grid, E, x):
    cg, keep = grid._c()
    N = grid.N
    E, x = _E(grid, E), _arr(x, 8 * N)
    y = np.zeros(8 * N)
    _check(_load().orc_apply_step(ctypes.byref(cg), E.ctypes.data, x.ctypes.data,
                                  y.ctypes.data), "apply_step")
    return y.reshape(8, N)


def apply_step_transpose(grid: Grid, E, y):
    cg, keep = grid._c()
    N = grid.N
    E, y = _E(grid, E), _arr(y, 8 * N)
    x = np.zeros(8 * N)
    _check(_load().orc_apply_step_transpose(ctypes.byref(cg), E.ctypes.data, y.ctypes.data,
                                            x.ctypes.data), "apply_step_transpose")
    return x.reshape(8, N)


def adjoint(grid: Grid, E, F, fS, dstar, steps: int, obs=None):
    """(phi_C, phi_S) after `steps` adjoint iterations from phi_C = 0 at state fS."""
    cg, keep = grid._c()
    N = grid.N
    E, F, fS, ds = _E(grid, E), _arr(F, 2 * N), _arr(fS, 8 * N), _arr(dstar, 2 * N)
    ob = None if obs is None else _arr(obs, N)
    pc = np.zeros(8 * N)
    ps = np.zeros(8 * N)
    rc = _load().orc_adjoint(ctypes.byref(cg), E.ctypes.data, F.ctypes.data, fS.ctypes.data,
                             ds.ctypes.data, None if ob is None else ob.ctypes.data, int(steps),
                             pc.ctypes.data, ps.ctypes.data)
    _check(rc, "adjoint")
    return pc.reshape(8, N), ps.reshape(8, N)


def gradient_force(grid: Grid, E, F, fS, phiS, dstar, obs=None):
    """dJ/dF_n (2, N) for the nodal force control (Eq. optimality)."""
    cg, keep = grid._c()
    N = grid.N
    E, F, fS, ps, ds = (_E(grid, E), _arr(F, 2 * N), _arr(fS, 8 * N), _arr(phiS, 8 * N),
                        _arr(dstar, 2 * N))
    ob = None if obs is None else _arr(obs, N)
    g = np.zeros(2 * N)
    rc = _load().orc_gradient_force(ctypes.byref(cg), E.ctypes.data, F.ctypes.data,
                                    fS.ctypes.data, ps.ctypes.data, ds.ctypes.data,
                                    None if ob is None else ob.ctypes.data, g.ctypes.data)
    _check(rc, "gradient_force")
    return g.reshape(2, N)


def gradient_young(grid: Grid, E, F, fS, phiS, phiC):
    """(dJ/dE_n per node (N,), their sum) at the fixed point (Eq. optimality)."""
    cg, keep = grid._c()
    N = grid.N
    E, F, fS, ps, pc = (_E(grid, E), _arr(F, 2 * N), _arr(fS, 8 * N), _arr(phiS, 8 * N),
                        _arr(phiC, 8 * N))
    gn = np.zeros(N)
    tot = ctypes.c_double()
    rc = _load().orc_gradient_young(ctypes.byref(cg), E.ctypes.data, F.ctypes.data,
                                    fS.ctypes.data, ps.ctypes.data, pc.ctypes.data,
                                    gn.ctypes.data, ctypes.addressof(tot))
    _check(rc, "gradient_young")
    return gn, tot.value


# ---- error measures (Section 4.1) ------------------------------------------------
def norm_L2(chi, dx):
    """Discrete L2 norm (Eq. L2_norm): (dx^2 sum_n |chi_n|_2^2)^(1/2); chi (c, N)."""
    chi = np.atleast_2d(chi)
    return float(np.sqrt(dx * dx * np.sum(chi * chi)))


def norm_Linf(chi):
    """Discrete Linf norm (Eq. Linf_norm): max_n |chi_n|_inf."""
    return float(np.max(np.abs(chi)))


def stress_frobenius_rows(s):
    """(s11, s22, s12) -> rows whose squared sum is the squared Frobenius norm."""
    return np.vstack([s[0], s[1], np.sqrt(2.0) * s[2]])


def eoc(nxs, errs):
    """Negative least-squares slope of log e over log N_x (Eq. EOC)."""
    x = np.log(np.asarray(nxs, dtype=np.float64))
    y = np.log(np.asarray(errs, dtype=np.float64))
    xm, ym = x.mean(), y.mean()
    return float(-np.sum((x - xm) * (y - ym)) / np.sum((x - xm) ** 2))
