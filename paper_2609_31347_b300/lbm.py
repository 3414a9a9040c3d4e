"""Python binding of the C ABI in include/lbm_solid.h (ctypes; argument marshalling only).

Every step of the primal / adjoint / gradient path runs in the CUDA library
``lib/liblbmsolid.so``; this module only converts arguments.  Device arrays are torch
CUDA float64 tensors; the library enqueues on torch's current stream unless a stream
is given.  Loading fails loudly when the library or a CUDA device is missing: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_STATE = 0, 1, 2, 3, 4
LBM_ERR_NOT_CONVERGED, LBM_ERR_DIVERGED = 5, 6
CONTROLS = {"force_field": 0, "force_basis2": 1, "young_scalar": 2, "young_field": 3}
KERNELS = {"auto": 0, "fp64": 1}

EXPORTED = [
    "lbm_solid_create", "lbm_solid_destroy", "lbm_solid_set_control", "lbm_solid_set_target",
    "lbm_solid_primal_solve", "lbm_solid_objective", "lbm_solid_adjoint_solve",
    "lbm_solid_gradient", "lbm_solid_get_populations", "lbm_solid_set_populations",
    "lbm_solid_displacement", "lbm_solid_launch_count", "lbm_status_string",
    "lbm_solid_last_error", "lbm_objective_noalloc",
]


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double),
        ("periodic", ctypes.c_int), ("E", ctypes.c_double), ("nu", ctypes.c_double),
        ("node_mask", ctypes.c_void_p), ("link_bc", ctypes.c_void_p),
        ("wall_d", ctypes.c_void_p), ("wall_T", ctypes.c_void_p), ("wall_n", ctypes.c_void_p),
        ("obs_mask", ctypes.c_void_p), ("control", ctypes.c_int), ("force", ctypes.c_void_p),
        ("force_basis", ctypes.c_void_p), ("kernel", ctypes.c_int),
    ]


class _Opts(ctypes.Structure):
    _fields_ = [("max_steps", ctypes.c_long), ("tol", ctypes.c_double),
                ("criterion", ctypes.c_int), ("window", ctypes.c_long),
                ("check_every", ctypes.c_long), ("fixed_steps", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_long), ("last_metric", ctypes.c_double),
                ("seconds", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (built in-tree by ``build.build()``) and declare signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("CUDA library %s is missing: run paper_2609_31347_b300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sigs = {
        "lbm_solid_create": ([ctypes.POINTER(_Desc), P, ctypes.POINTER(P)], I),
        "lbm_solid_destroy": ([P], I),
        "lbm_solid_set_control": ([P, P, S, I], I),
        "lbm_solid_set_target": ([P, P], I),
        "lbm_solid_primal_solve": ([P, ctypes.POINTER(_Opts), ctypes.POINTER(_Info)], I),
        "lbm_solid_objective": ([P, ctypes.POINTER(D)], I),
        "lbm_solid_adjoint_solve": ([P, ctypes.POINTER(_Opts), ctypes.POINTER(_Info)], I),
        "lbm_solid_gradient": ([P, P, S, I], I),
        "lbm_solid_get_populations": ([P, I, P], I),
        "lbm_solid_set_populations": ([P, I, P], I),
        "lbm_solid_displacement": ([P, P], I),
        "lbm_solid_launch_count": ([P], ctypes.c_long),
        "lbm_status_string": ([I], ctypes.c_char_p),
        "lbm_solid_last_error": ([P], ctypes.c_char_p),
        "lbm_objective_noalloc": ([I, I, D, P, P, P, P, P, P], I),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


@dataclass
class SolveInfo:
    steps: int
    last_metric: float
    seconds: float
    status: int


def _host(a, dtype, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=dtype).ravel())
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _dev_ptr(t, n=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError("expected a CUDA float64 tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError("expected %d values, got %d" % (n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


class LBMSolid:
    """One lattice on the GPU: primal sweep, objective, adjoint sweep, gradient."""

    def __init__(self, nx: int, ny: int, dx: float, E: float, nu: float, periodic: bool = True,
                 node_mask=None, link_bc=None, wall_d=None, wall_T=None, wall_n=None,
                 obs=None, control: str = "force_field", force=None, force_basis=None,
                 kernel: str = "auto", stream=None):
        import torch
        self._lib = load_library()
        self.nx, self.ny, self.N = int(nx), int(ny), int(nx) * int(ny)
        self.control = control
        N = self.N
        keep = [_host(node_mask, np.uint8, N), _host(link_bc, np.uint8, 8 * N),
                _host(wall_d, np.float64, 2 * N), _host(wall_T, np.float64, 2 * N),
                _host(wall_n, np.float64, 2 * N), _host(obs, np.float64, N),
                _host(force, np.float64, 2 * N), _host(force_basis, np.float64, 4 * N)]
        ptr = [None if a is None else a.ctypes.data for a in keep]
        d = _Desc(self.nx, self.ny, float(dx), 1 if periodic else 0, float(E), float(nu),
                  ptr[0], ptr[1], ptr[2], ptr[3], ptr[4], ptr[5], CONTROLS[control], ptr[6],
                  ptr[7], KERNELS[kernel])
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = self._lib.lbm_solid_create(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream),
                                        ctypes.byref(h))
        if st != LBM_OK:
            raise LBMError(st, "lbm_solid_create: " +
                           self._lib.lbm_status_string(st).decode())
        self._h = h

    # -- helpers ---------------------------------------------------------------------
    def _check(self, st, what):
        if st != LBM_OK:
            raise LBMError(st, "%s: %s" % (what, self._lib.lbm_solid_last_error(self._h).decode()))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_solid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launch_count(self) -> int:
        return int(self._lib.lbm_solid_launch_count(self._h))

    @staticmethod
    def _opts(max_steps, tol, criterion, window, check_every, fixed_steps):
        return _Opts(int(max_steps), float(tol), int(criterion), int(window), int(check_every),
                     1 if fixed_steps else 0)

    # -- C ABI calls -------------------------------------------------------------------
    def set_control(self, alpha, keep_state: bool = False):
        self._check(self._lib.lbm_solid_set_control(self._h, _dev_ptr(alpha), alpha.numel(),
                                                    1 if keep_state else 0), "set_control")

    def set_target(self, dstar):
        self._check(self._lib.lbm_solid_set_target(self._h, _dev_ptr(dstar, 2 * self.N)),
                    "set_target")

    def _solve(self, fn, what, max_steps, tol, criterion, window, check_every, fixed_steps,
               allow_not_converged):
        o = self._opts(max_steps, tol, criterion, window, check_every, fixed_steps)
        info = _Info()
        st = fn(self._h, ctypes.byref(o), ctypes.byref(info))
        if st != LBM_OK and not (allow_not_converged and
                                 st in (LBM_ERR_NOT_CONVERGED, LBM_ERR_DIVERGED)):
            self._check(st, what)
        return SolveInfo(info.steps, info.last_metric, info.seconds, st)

    def primal_solve(self, max_steps: int, tol: float = 1e-10, criterion: int = 1,
                     window: int = 100, check_every: int = 100, fixed_steps: bool = False,
                     allow_not_converged: bool = False) -> SolveInfo:
        return self._solve(self._lib.lbm_solid_primal_solve, "primal_solve", max_steps, tol,
                           criterion, window, check_every, fixed_steps, allow_not_converged)

    def adjoint_solve(self, max_steps: int, tol: float = 1e-10, criterion: int = 1,
                      window: int = 100, check_every: int = 100, fixed_steps: bool = False,
                      allow_not_converged: bool = False) -> SolveInfo:
        return self._solve(self._lib.lbm_solid_adjoint_solve, "adjoint_solve", max_steps, tol,
                           criterion, window, check_every, fixed_steps, allow_not_converged)

    def objective(self) -> float:
        J = ctypes.c_double()
        self._check(self._lib.lbm_solid_objective(self._h, ctypes.byref(J)), "objective")
        return J.value

    def gradient(self, out=None, project_zero_mean: bool = False):
        import torch
        n = {"force_field": 2 * self.N, "force_basis2": 2, "young_scalar": 1,
             "young_field": self.N}[self.control]
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device="cuda")
        self._check(self._lib.lbm_solid_gradient(self._h, _dev_ptr(out, n), n,
                                                 1 if project_zero_mean else 0), "gradient")
        return out

    def get_populations(self, which: int = 0, out=None):
        import torch
        if out is None:
            out = torch.empty(8 * self.N, dtype=torch.float64, device="cuda")
        self._check(self._lib.lbm_solid_get_populations(self._h, int(which),
                                                        _dev_ptr(out, 8 * self.N)),
                    "get_populations")
        return out

    def set_populations(self, which: int, src):
        self._check(self._lib.lbm_solid_set_populations(self._h, int(which),
                                                        _dev_ptr(src, 8 * self.N)),
                    "set_populations")

    def displacement(self, out=None):
        import torch
        if out is None:
            out = torch.empty(2 * self.N, dtype=torch.float64, device="cuda")
        self._check(self._lib.lbm_solid_displacement(self._h, _dev_ptr(out, 2 * self.N)),
                    "displacement")
        return out
