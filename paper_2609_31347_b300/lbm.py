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
    "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_offset", "lbm_batch_set_force",
    "lbm_batch_set_target", "lbm_batch_primal", "lbm_batch_objective", "lbm_batch_adjoint",
    "lbm_batch_gradient", "lbm_batch_get_populations", "lbm_batch_tune", "lbm_solid_tangent",
    "lbm_unet_create", "lbm_unet_destroy", "lbm_unet_param_count", "lbm_unet_get_params",
    "lbm_unet_set_params", "lbm_unet_forward", "lbm_unet_train_step", "lbm_unet_status",
    "lbm_solid_adjoint_source", "lbm_warm_encode", "lbm_warm_targets", "lbm_warm_decode", "lbm_warm_channel_rms",
    "lbm_warm_combine", "lbm_warm_dot_work_size", "lbm_warm_dots",
    "lbm_solid_monitor_samples", "lbm_plate_batch_create", "lbm_plate_batch_destroy",
    "lbm_plate_batch_set_control", "lbm_plate_batch_primal", "lbm_plate_batch_get_populations",
    "lbm_warm_encode_modulus", "lbm_warm_crop",
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
        "lbm_solid_monitor_samples": ([P, P, ctypes.c_long], ctypes.c_long),
        "lbm_plate_batch_create": ([ctypes.POINTER(_Desc), I, P, ctypes.POINTER(P)], I),
        "lbm_plate_batch_destroy": ([P], I),
        "lbm_plate_batch_set_control": ([P, P], I),
        "lbm_plate_batch_primal": ([P, ctypes.c_long], I),
        "lbm_plate_batch_get_populations": ([P, P], I),
        "lbm_warm_encode_modulus": ([I, I, I, I, P, P, D, I, I, I, P, P], I),
        "lbm_warm_crop": ([I, I, I, I, I, I, P, P, P, P], I),
        "lbm_status_string": ([I], ctypes.c_char_p),
        "lbm_solid_last_error": ([P], ctypes.c_char_p),
        "lbm_objective_noalloc": ([I, I, D, P, P, P, P, P, P], I),
        "lbm_batch_create": ([I, P, P, P, D, D, I, P, ctypes.POINTER(P)], I),
        "lbm_batch_destroy": ([P], I),
        "lbm_batch_offset": ([P, I], ctypes.c_long),
        "lbm_batch_set_force": ([P, P], I),
        "lbm_batch_set_target": ([P, P], I),
        "lbm_batch_primal": ([P, ctypes.c_long], I),
        "lbm_batch_objective": ([P, P], I),
        "lbm_batch_adjoint": ([P, ctypes.c_long], I),
        "lbm_batch_gradient": ([P, P], I),
        "lbm_batch_get_populations": ([P, I, P], I),
        "lbm_batch_tune": ([P, I, ctypes.POINTER(I)], I),
        "lbm_solid_tangent": ([P, P, S, ctypes.POINTER(_Opts), ctypes.POINTER(D),
                               ctypes.POINTER(_Info)], I),
        "lbm_unet_create": ([I, I, I, I, I, ctypes.c_ulonglong, P, ctypes.POINTER(P)], I),
        "lbm_unet_destroy": ([P], I),
        "lbm_unet_param_count": ([P], ctypes.c_long),
        "lbm_unet_get_params": ([P, P, I], I),
        "lbm_unet_set_params": ([P, P], I),
        "lbm_unet_status": ([P], I),
        "lbm_unet_forward": ([P, P, P, I], I),
        "lbm_unet_train_step": ([P, P, P, ctypes.c_float, P], I),
        "lbm_solid_adjoint_source": ([P, P], I),
        "lbm_warm_encode": ([I, I, I, I, P, P, P, P, P], I),
        "lbm_warm_targets": ([I, I, I, D, I, P, P, P, P, P], I),
        "lbm_warm_decode": ([I, I, I, I, D, I, P, P, P, P, I, P], I),
        "lbm_warm_channel_rms": ([P, ctypes.c_long, P, P], I),
        "lbm_warm_combine": ([I, ctypes.c_long, P, P, P, P], I),
        "lbm_warm_dot_work_size": ([], ctypes.c_long),
        "lbm_warm_dots": ([I, ctypes.c_long, P, P, P, P], I),
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


def _dev_ptr(t, n=None, dtype=None):
    import torch
    dtype = torch.float64 if dtype is None else dtype
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype):
        raise TypeError("expected a CUDA %s tensor" % dtype)
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError("expected %d values, got %d" % (n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _ptr_array(tensors, n):
    arr = (ctypes.c_void_p * len(tensors))()
    for j, t in enumerate(tensors):
        arr[j] = _dev_ptr(t, n).value
    return arr


def warm_combine(weights, srcs, dst):
    """dst = sum_j weights[j] * srcs[j] (1 to 4 device FP64 vectors of dst's size) on the
    current stream; dst may be one of srcs."""
    import torch
    lib = load_library()
    n = dst.numel()
    w = _host(weights, np.float64, len(srcs))
    st = lib.lbm_warm_combine(len(srcs), n, w.ctypes.data, _ptr_array(srcs, n),
                              _dev_ptr(dst, n), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != LBM_OK:
        raise LBMError(st, "lbm_warm_combine: " + lib.lbm_status_string(st).decode())
    return dst


_dot_work = {}


def warm_dots(vectors):
    """Matrix of inner products of 1 to 5 device FP64 vectors of one size (host, m x m),
    summed in a fixed order; synchronises the current stream."""
    import torch
    lib = load_library()
    dev = vectors[0].device
    work = _dot_work.get(dev)
    if work is None:
        work = torch.empty(int(lib.lbm_warm_dot_work_size()), dtype=torch.float64, device=dev)
        _dot_work[dev] = work
    n, m = vectors[0].numel(), len(vectors)
    out = np.zeros(m * m)
    st = lib.lbm_warm_dots(m, n, _ptr_array(vectors, n), _dev_ptr(work), out.ctypes.data,
                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != LBM_OK:
        raise LBMError(st, "lbm_warm_dots: " + lib.lbm_status_string(st).decode())
    return out.reshape(m, m)


def _desc(nx, ny, dx, E, nu, periodic, node_mask, link_bc, wall_d, wall_T, wall_n, obs,
          control, force, force_basis, kernel):
    """(lbm_solid_desc, host arrays it points to)."""
    N = int(nx) * int(ny)
    keep = [_host(node_mask, np.uint8, N), _host(link_bc, np.uint8, 8 * N),
            _host(wall_d, np.float64, 2 * N), _host(wall_T, np.float64, 2 * N),
            _host(wall_n, np.float64, 2 * N), _host(obs, np.float64, N),
            _host(force, np.float64, 2 * N), _host(force_basis, np.float64, 4 * N)]
    ptr = [None if a is None else a.ctypes.data for a in keep]
    d = _Desc(int(nx), int(ny), float(dx), 1 if periodic else 0, float(E), float(nu),
              ptr[0], ptr[1], ptr[2], ptr[3], ptr[4], ptr[5], CONTROLS[control], ptr[6],
              ptr[7], KERNELS[kernel])
    return d, keep


class LBMPlateBatch:
    """count instances of one bounded geometry, each with its own per-node modulus
    (E_n = alpha_n^2), advanced by one launch per sweep."""

    def __init__(self, count: int, nx: int, ny: int, dx: float, E: float, nu: float,
                 node_mask, link_bc, wall_d=None, wall_T=None, wall_n=None, force=None,
                 kernel: str = "auto", stream=None):
        import torch
        self._lib = load_library()
        self.count, self.nx, self.ny, self.N = int(count), int(nx), int(ny), int(nx) * int(ny)
        d, keep = _desc(nx, ny, dx, E, nu, False, node_mask, link_bc, wall_d, wall_T, wall_n,
                        None, "young_field", force, None, kernel)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        h = ctypes.c_void_p()
        st = self._lib.lbm_plate_batch_create(ctypes.byref(d), int(count),
                                              ctypes.c_void_p(self.stream.cuda_stream),
                                              ctypes.byref(h))
        if st != LBM_OK:
            raise LBMError(st, "lbm_plate_batch_create: " +
                           self._lib.lbm_status_string(st).decode())
        self._h = h

    def _check(self, st, what):
        if st != LBM_OK:
            raise LBMError(st, "%s: %s" % (what, self._lib.lbm_status_string(st).decode()))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_plate_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_control(self, alpha):
        """count * N controls (device float64); resets every instance to rest."""
        self._check(self._lib.lbm_plate_batch_set_control(
            self._h, _dev_ptr(alpha, self.count * self.N)), "set_control")

    def primal(self, sweeps: int):
        self._check(self._lib.lbm_plate_batch_primal(self._h, int(sweeps)), "primal")

    def get_populations(self, out=None):
        import torch
        if out is None:
            out = torch.empty(8 * self.count * self.N, dtype=torch.float64, device="cuda")
        self._check(self._lib.lbm_plate_batch_get_populations(
            self._h, _dev_ptr(out, 8 * self.count * self.N)), "get_populations")
        return out


class LBMSolid:
    """One lattice on the GPU: primal sweep, objective, adjoint sweep, gradient."""

    def __init__(self, nx: int, ny: int, dx: float, E: float, nu: float, periodic: bool = True,
                 node_mask=None, link_bc=None, wall_d=None, wall_T=None, wall_n=None,
                 obs=None, control: str = "force_field", force=None, force_basis=None,
                 kernel: str = "auto", stream=None):
        import torch
        self._lib = load_library()
        self.nx, self.ny, self.N = int(nx), int(ny), int(nx) * int(ny)
        self.dx, self.periodic = float(dx), bool(periodic)
        self.sweeps = {}  # sweeps performed per solve kind ("primal_solve", ...)
        self.capped = {}  # solves per kind that ended at max_steps before their rule held
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

    def monitor_samples(self) -> np.ndarray:
        """Monitor samples c of the last criterion-0 solve (host array)."""
        n = int(self._lib.lbm_solid_monitor_samples(self._h, None, 0))
        out = np.zeros(max(n, 0))
        if n > 0:
            self._lib.lbm_solid_monitor_samples(self._h, out.ctypes.data, n)
        return out

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
        self.sweeps[what] = self.sweeps.get(what, 0) + int(info.steps)
        if st == LBM_ERR_NOT_CONVERGED:
            self.capped[what] = self.capped.get(what, 0) + 1
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

    def tangent(self, seed, max_steps: int = 2_000_000, tol: float = 1e-12,
                check_every: int = 64, fixed_steps: bool = False) -> float:
        """Forward-mode dJ along `seed` (device tensor) at the current primal state."""
        o = self._opts(max_steps, tol, 1, 2, check_every, fixed_steps)
        dJ, info = ctypes.c_double(), _Info()
        st = self._lib.lbm_solid_tangent(self._h, _dev_ptr(seed), seed.numel(), ctypes.byref(o),
                                         ctypes.byref(dJ), ctypes.byref(info))
        self._check(st, "tangent")
        return dJ.value

    def objective(self) -> float:
        J = ctypes.c_double()
        self._check(self._lib.lbm_solid_objective(self._h, ctypes.byref(J)), "objective")
        return J.value

    def adjoint_source(self, out=None):
        """r = (dx^2/Cbar) w (d - d*) of the current primal state (2N, device)."""
        import torch
        if out is None:
            out = torch.empty(2 * self.N, dtype=torch.float64, device="cuda")
        self._check(self._lib.lbm_solid_adjoint_source(self._h, _dev_ptr(out, 2 * self.N)),
                    "adjoint_source")
        return out

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


class LBMBatch:
    """Many periodic lattices of uneven size advanced together (one launch per sweep)."""

    def __init__(self, sizes, E: float, nu: float, dx=None, kernel: str = "auto", stream=None):
        import torch
        self._lib = load_library()
        sizes = [(int(a), int(b)) for a, b in sizes]
        self.count = len(sizes)
        nx = (ctypes.c_int * self.count)(*[a for a, _ in sizes])
        ny = (ctypes.c_int * self.count)(*[b for _, b in sizes])
        dxa = None if dx is None else (ctypes.c_double * self.count)(*[float(v) for v in dx])
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = self._lib.lbm_batch_create(self.count, nx, ny, dxa, float(E), float(nu),
                                        KERNELS[kernel], ctypes.c_void_p(stream.cuda_stream),
                                        ctypes.byref(h))
        if st != LBM_OK:
            raise LBMError(st, "lbm_batch_create: " + self._lib.lbm_status_string(st).decode())
        self._h = h
        self.sizes = sizes
        self.offsets = [int(self._lib.lbm_batch_offset(h, i)) for i in range(self.count + 1)]
        self.total = self.offsets[-1]

    def _check(self, st, what):
        if st != LBM_OK:
            raise LBMError(st, "%s: %s" % (what, self._lib.lbm_status_string(st).decode()))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_force(self, F):
        self._check(self._lib.lbm_batch_set_force(self._h, _dev_ptr(F, 2 * self.total)), "set_force")

    def set_target(self, dstar):
        self._check(self._lib.lbm_batch_set_target(self._h, _dev_ptr(dstar, 2 * self.total)),
                    "set_target")

    def primal(self, sweeps: int):
        self._check(self._lib.lbm_batch_primal(self._h, int(sweeps)), "primal")

    def adjoint(self, sweeps: int):
        self._check(self._lib.lbm_batch_adjoint(self._h, int(sweeps)), "adjoint")

    def objective(self, out=None):
        import torch
        if out is None:
            out = torch.empty(self.count, dtype=torch.float64, device="cuda")
        self._check(self._lib.lbm_batch_objective(self._h, _dev_ptr(out, self.count)), "objective")
        return out

    def gradient(self, out=None):
        import torch
        if out is None:
            out = torch.empty(2 * self.total, dtype=torch.float64, device="cuda")
        self._check(self._lib.lbm_batch_gradient(self._h, _dev_ptr(out, 2 * self.total)), "gradient")
        return out

    def get_populations(self, which: int = 0, out=None):
        import torch
        if out is None:
            out = torch.empty(8 * self.total, dtype=torch.float64, device="cuda")
        self._check(self._lib.lbm_batch_get_populations(self._h, int(which),
                                                        _dev_ptr(out, 8 * self.total)),
                    "get_populations")
        return out

    def tune(self, sweeps: int = 16) -> int:
        bx = ctypes.c_int()
        self._check(self._lib.lbm_batch_tune(self._h, int(sweeps), ctypes.byref(bx)), "tune")
        return bx.value

    # views of one instance inside concatenated arrays
    def pop_view(self, t, i):
        o, n = self.offsets[i], self.offsets[i + 1] - self.offsets[i]
        return t[8 * o: 8 * (o + n)].view(8, n)

    def field_view(self, t, i):
        o, n = self.offsets[i], self.offsets[i + 1] - self.offsets[i]
        return t[2 * o: 2 * (o + n)].view(2, n)


class UNet:
    """The warm-start network (include/lbm_solid.h, "Learned warm start"): FP32 CUDA tensors
    x (B, H, W, 2) and y, t (B, H, W, 8), NHWC."""

    def __init__(self, batch: int, H: int, W: int, base: int = 32, levels: int = 4,
                 seed: int = 0, stream=None):
        import torch
        self._lib = load_library()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.batch, self.H, self.W, self.base, self.levels = batch, H, W, base, levels
        h = ctypes.c_void_p()
        st = self._lib.lbm_unet_create(int(base), int(levels), int(batch), int(H), int(W),
                                       int(seed), ctypes.c_void_p(stream.cuda_stream),
                                       ctypes.byref(h))
        if st != LBM_OK:
            raise LBMError(st, "lbm_unet_create: " + self._lib.lbm_status_string(st).decode())
        self._h = h
        self.nparams = int(self._lib.lbm_unet_param_count(h))
        self._loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def _check(self, st, what):
        if st != LBM_OK:
            raise LBMError(st, "%s: %s" % (what, self._lib.lbm_status_string(st).decode()))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f32(self, t, n):
        import torch
        return _dev_ptr(t, n, torch.float32)

    def status(self):
        """Synchronise; raise if a tensor-core convolution gave up waiting."""
        self._check(self._lib.lbm_unet_status(self._h), "unet")

    def params(self, which: int = 0):
        """Copy of the FP32 parameter vector (0) or of the last gradient (1)."""
        import torch
        out = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        self._check(self._lib.lbm_unet_get_params(self._h, self._f32(out, self.nparams), which),
                    "get_params")
        return out

    def set_params(self, p):
        self._check(self._lib.lbm_unet_set_params(self._h, self._f32(p, self.nparams)),
                    "set_params")

    def forward(self, x, out=None, exact_acts: bool = False):
        """y = net(x); exact_acts: FP32 activations (split-BF16 products) instead of BF16."""
        import torch
        P = self.batch * self.H * self.W
        if out is None:
            out = torch.empty((self.batch, self.H, self.W, 8), dtype=torch.float32, device="cuda")
        self._check(self._lib.lbm_unet_forward(self._h, self._f32(x, 2 * P), self._f32(out, 8 * P),
                                               1 if exact_acts else 0), "forward")
        return out

    def train_step(self, x, t, lr: float):
        """One step; returns the loss as a 1-element device tensor (no synchronisation)."""
        P = self.batch * self.H * self.W
        self._check(self._lib.lbm_unet_train_step(self._h, self._f32(x, 2 * P), self._f32(t, 8 * P),
                                                  float(lr), self._f32(self._loss, 1)),
                    "train_step")
        return self._loss
