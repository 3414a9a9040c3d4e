"""Learned warm start of the primal and adjoint fixed-point iterations.

Not part of the paper's method: a network only proposes the initial populations; the
solver then iterates (primal collide + stream, Section 3.1; adjoint, Eq.
adjoint_iteration) to the same residual tolerance as from a cold start, so the fixed
point, and every objective and gradient computed from it, is the solver's own.  The
network changes iteration counts only.

Pieces (all arithmetic in the CUDA library, see include/lbm_solid.h "Learned warm
start"; this module orchestrates):

- ``WarmStartNet``: one U-Net (BF16 storage, FP32 accumulation) for the primal map
  force F -> steady f_S, or for the adjoint map source r -> steady phi_C, with its
  training data generated by the solver itself (a batch of periodic lattices driven by
  random smooth fields, iterated to near steady state) and trained by the library's
  own forward/backward/Adam kernels.  A network trained on nx^2 lattices is used on
  (factor * nx)^2 lattices by block-averaging the input and interpolating the predicted
  moments, which are scaled so that they do not depend on the grid spacing.
- ``PlateWarmStartNet``: the same network for the primal state of one bounded plate as a
  function of its Young's modulus (uniform or per node), trained on states of a batch
  of that plate with random moduli (one launch per sweep).
- ``WarmStarter``: supplies initial states to the solves of an optimisation loop.
  Since the steady states are affine in F (primal) and linear in r (adjoint), a
  combination of the loop's earlier steady states reproduces the state of any control
  (source) in the span of the earlier ones; the network then predicts only the state
  of what is left of the change, so its error is relative to that remainder, not to
  the whole state.  For a Young's-modulus control the primal states are extrapolated
  in 1/E instead (no network).
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

from . import inputs as I
from . import lbm as L


def _ptr(t):
    return L.ctypes.c_void_p(t.data_ptr()) if t is not None else None


class WarmStartNet:
    """A U-Net for one of the two fixed-point maps of a periodic nx x nx lattice."""

    def __init__(self, kind: str = "primal", nx: int = 128, E: float = 8.0 / 3.0,
                 nu: float = 1.0 / 3.0, base: int = 32, levels: int = 4, batch: int = 16,
                 seed: int = 0, stream=None):
        import torch
        if kind not in ("primal", "adjoint"):
            raise ValueError("kind must be 'primal' or 'adjoint'")
        self._lib = L.load_library()
        self.kind, self.nx, self.dx = kind, int(nx), 1.0 / nx
        self.E, self.nu = float(E), float(nu)
        self.base, self.levels, self.batch, self.seed = base, levels, batch, seed
        self.mode = 1 if kind == "primal" else 2  # resolution-free moments, see lbm_warm.cu
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.net = L.UNet(batch, nx, nx, base, levels, seed, stream=self.stream)
        self._infer: Optional[L.UNet] = None
        self.chan = None  # per-channel constants c_i (8 floats, device)
        self._x = torch.empty((1, nx, nx, 2), dtype=torch.float32, device="cuda")
        self._y = torch.empty((1, nx, nx, 8), dtype=torch.float32, device="cuda")
        self._s = torch.empty(1, dtype=torch.float32, device="cuda")

    def _st(self):
        return L.ctypes.c_void_p(self.stream.cuda_stream)

    def _check(self, st, what):
        if st != L.LBM_OK:
            raise L.LBMError(st, "%s: %s" % (what, self._lib.lbm_status_string(st).decode()))

    # ---- data -------------------------------------------------------------------
    def generate(self, count: int, sweeps: int, seed: int = 1, chunk: int = 256,
                 modes: int = 8, kmax: int = 4, exponents=(1.0, 2.0, 3.0)):
        """`count` (input, target) pairs from the solver: random smooth fields (``modes``
        Fourier modes, |k| up to kmax * 2 pi, amplitude spectra |k|^-p with p drawn from
        `exponents`, from force-like to displacement-like inputs) drive a batch of
        lattices for `sweeps` sweeps from rest.  Returns device tensors
        X (count, nx, nx, 2) and T (count, nx, nx, 8), FP32."""
        import torch
        nx, N = self.nx, self.nx * self.nx
        X = torch.empty((count, nx, nx, 2), dtype=torch.float32, device="cuda")
        T = torch.empty((count, nx, nx, 8), dtype=torch.float32, device="cuda")
        sc = torch.empty(chunk, dtype=torch.float32, device="cuda")
        for start in range(0, count, chunk):
            m = min(chunk, count - start)
            fields = I.fourier_fields(m, nx, seed=seed * 1_000_003 + start, modes=modes,
                                      kmax=kmax, unit_norm=self.kind == "adjoint",
                                      exponents=exponents)
            b = L.LBMBatch([(nx, nx)] * m, self.E, self.nu, dx=[self.dx] * m, stream=self.stream)
            if self.kind == "primal":
                b.set_force(fields.reshape(-1))
                b.primal(sweeps)
                pops = b.get_populations(0)
                src = fields
            else:
                # F = 0 keeps d = 0, so r = (dx^2/Cbar)(0 - d*) = -d* for a unit-norm d*
                b.set_force(torch.zeros(2 * m * N, dtype=torch.float64, device="cuda"))
                b.set_target(fields.reshape(-1))
                b.adjoint(sweeps)
                pops = b.get_populations(2)
                src = -fields
            self._check(self._lib.lbm_warm_encode(m, nx, nx, 1, _ptr(src), None, _ptr(X[start:]),
                                                  _ptr(sc), self._st()), "encode")
            if self.chan is None:
                self._check(self._lib.lbm_warm_targets(m, nx, nx, self.dx, self.mode, _ptr(pops),
                                                       _ptr(sc), None, _ptr(T[start:]),
                                                       self._st()), "targets")
                rms = torch.empty(8, dtype=torch.float32, device="cuda")
                self._check(self._lib.lbm_warm_channel_rms(_ptr(T[start:]), m * N, _ptr(rms),
                                                           self._st()), "channel_rms")
                r = rms.cpu().numpy()
                # channels that vanish identically at the fixed point (the adjoint's
                # m12 - (1 - theta) m10, m21 - (1 - theta) m01) are not predicted: c_i = 0
                r = np.where(r > 1e-6 * r.max(), r, 0.0)
                self.chan = torch.as_tensor(r.astype(np.float32), device="cuda")
            self._check(self._lib.lbm_warm_targets(m, nx, nx, self.dx, self.mode, _ptr(pops),
                                                   _ptr(sc), _ptr(self.chan), _ptr(T[start:]),
                                                   self._st()), "targets")
            b.close()
        return X, T

    # ---- training ---------------------------------------------------------------
    def fit(self, X, T, steps: int, lr: float = 1e-3, lr_min: float = 1e-5,
            log_every: int = 50, seed: int = 0):
        """Adam on mini-batches of the data set with a cosine learning-rate schedule.
        Returns the logged losses [(step, loss)]."""
        B = self.batch
        nb = X.shape[0] // B
        if nb < 1:
            raise ValueError("need at least one full batch of %d samples" % B)
        rng = np.random.default_rng(seed)
        order = rng.permutation(nb)
        log = []
        for it in range(steps):
            if it and it % nb == 0:
                order = rng.permutation(nb)
            j = int(order[it % nb])
            lr_t = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * it / steps))
            loss = self.net.train_step(X[j * B:(j + 1) * B], T[j * B:(j + 1) * B], lr_t)
            if it % log_every == 0 or it == steps - 1:
                log.append((it, float(loss)))
        self._infer = None
        return log

    def evaluate(self, X, T):
        """Relative L2 error of the predictions (FP32 activations, as used for warm starts)
        over a data set (full batches)."""
        import torch
        B = self.batch
        num = den = 0.0
        out = torch.empty((B,) + tuple(T.shape[1:]), dtype=torch.float32, device="cuda")
        for j in range(X.shape[0] // B):
            self.net.forward(X[j * B:(j + 1) * B], out, exact_acts=True)
            t = T[j * B:(j + 1) * B]
            num += float(torch.sum((out.double() - t.double()) ** 2))
            den += float(torch.sum(t.double() ** 2))
        return math.sqrt(num / den)

    # ---- inference ---------------------------------------------------------------
    def _inference_net(self):
        if self._infer is None:
            self._infer = L.UNet(1, self.nx, self.nx, self.base, self.levels, self.seed,
                                 stream=self.stream)
            self._infer.set_params(self.net.params(0))
        return self._infer

    def predict(self, field, out, nx_fine: Optional[int] = None, dx_fine: Optional[float] = None,
                ref=None, accumulate: bool = False):
        """Initial populations (8 N_fine, FP64 device tensor `out`) for the state driven by
        `field` (2 N_fine; minus `ref` if given) on an nx_fine^2 periodic lattice with
        spacing dx_fine (default 1/nx_fine); added to `out` if accumulate."""
        if self.chan is None:
            raise RuntimeError("the network has no data normalisation yet: call generate()")
        nxf = self.nx if nx_fine is None else int(nx_fine)
        if nxf % self.nx:
            raise ValueError("lattice size %d is not a multiple of the network's %d" % (nxf, self.nx))
        factor = nxf // self.nx
        N = nxf * nxf
        L._dev_ptr(field, 2 * N)  # CUDA float64, contiguous, right size (raises otherwise)
        L._dev_ptr(out, 8 * N)
        if ref is not None:
            L._dev_ptr(ref, 2 * N)
        dxf = 1.0 / nxf if dx_fine is None else float(dx_fine)
        net = self._inference_net()
        self._check(self._lib.lbm_warm_encode(1, nxf, nxf, factor, _ptr(field), _ptr(ref),
                                              _ptr(self._x), _ptr(self._s), self._st()), "encode")
        net.forward(self._x, self._y, exact_acts=True)
        self._check(self._lib.lbm_warm_decode(1, self.nx, self.nx, factor, dxf, self.mode,
                                              _ptr(self._y), _ptr(self._s), _ptr(self.chan),
                                              _ptr(out), 1 if accumulate else 0, self._st()),
                    "decode")
        return out


class PlateWarmStartNet:
    """A U-Net for the steady primal state of one bounded geometry (the plate, its wall
    data and loads fixed) as a function of its Young's modulus, uniform or per node.

    Input: block means over the network's grid of the compliance mask E_ref / E and of the
    domain mask (for loads that do not depend on E the steady displacement of a uniform
    modulus is proportional to the compliance, which a linear network represents);
    output: the eight resolution-free moments of the steady state (the primal
    scaling of WarmStartNet, without the periodic steps).  The network's grid is the
    Nx x Nx crop of the (Nx + 1)^2 box (the domain lies inside it).  Training states are
    generated by the solver itself: a batch of the plate with random moduli, advanced
    by one launch per sweep (LBMPlateBatch).  A network trained at Nx serves the same
    physical plate at factor * Nx (input block-averaged, moments interpolated)."""

    net_on_change = False  # the map E -> state is not linear: no state-of-a-change use

    def __init__(self, make_geometry, Nx: int = 64, E_ref: float = 1.0, nu: float = 0.3,
                 base: int = 32, levels: int = 3, batch: int = 16, seed: int = 0,
                 stream=None):
        import torch
        self._lib = L.load_library()
        self.make_geometry = make_geometry
        self.Nx, self.nx = int(Nx), int(Nx)
        self.E_ref, self.nu = float(E_ref), float(nu)
        self.base, self.levels, self.batch, self.seed = base, levels, batch, seed
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.net = L.UNet(batch, self.Nx, self.Nx, base, levels, seed, stream=self.stream)
        self._infer = None
        self.chan = None
        self._geo = {}
        self._one = torch.ones(1, dtype=torch.float32, device="cuda")
        self._x = torch.empty((1, self.Nx, self.Nx, 2), dtype=torch.float32, device="cuda")
        self._y = torch.empty((1, self.Nx, self.Nx, 8), dtype=torch.float32, device="cuda")

    _st = WarmStartNet._st
    _check = WarmStartNet._check
    fit = WarmStartNet.fit
    evaluate = WarmStartNet.evaluate
    _inference_net = WarmStartNet._inference_net

    def geometry(self, Nx):
        """(geometry, wall_d, wall_T, device mask) of the plate at resolution Nx."""
        import torch
        if Nx not in self._geo:
            geo, wd, wT = self.make_geometry(Nx)
            mask = torch.as_tensor(geo.active.astype(np.uint8), device="cuda")
            self._geo[Nx] = (geo, wd, wT, mask)
        return self._geo[Nx]

    def generate(self, count: int, sweeps: int, seed: int = 1, chunk: int = 256,
                 E_range=(0.5, 2.0), sigma: float = 0.2, field_frac: float = 0.5):
        """`count` (input, target) pairs: moduli E_0 log-uniform in E_range, and for a
        fraction field_frac of the samples a per-node lognormal field E_0 exp(sigma z -
        sigma^2 / 2) (z i.i.d. normal); `sweeps` sweeps from rest.  Returns device tensors
        X (count, Nx, Nx, 2) and T (count, Nx, Nx, 8), FP32."""
        import torch
        geo, wd, wT, mask = self.geometry(self.Nx)
        nxb, Nx = geo.nx, self.Nx
        Nb = nxb * nxb
        rng = np.random.default_rng(seed)
        X = torch.empty((count, Nx, Nx, 2), dtype=torch.float32, device="cuda")
        T = torch.empty((count, Nx, Nx, 8), dtype=torch.float32, device="cuda")
        ones = torch.ones(chunk, dtype=torch.float32, device="cuda")
        for start in range(0, count, chunk):
            m = min(chunk, count - start)
            E0 = np.exp(rng.uniform(np.log(E_range[0]), np.log(E_range[1]), size=m))
            z = rng.standard_normal((m, Nb))
            field = rng.random(m) < field_frac
            E = E0[:, None] * np.where(field[:, None], np.exp(sigma * z - 0.5 * sigma * sigma),
                                       1.0)
            alpha = torch.as_tensor(np.sqrt(E).ravel(), device="cuda")
            b = L.LBMPlateBatch(m, nxb, nxb, geo.dx, self.E_ref, self.nu, node_mask=geo.active,
                                link_bc=geo.link, wall_d=wd, wall_T=wT, wall_n=geo.normal,
                                stream=self.stream)
            b.set_control(alpha)
            b.primal(sweeps)
            pops = b.get_populations()
            b.close()
            crop = torch.empty(m * 8 * Nx * Nx, dtype=torch.float64, device="cuda")
            self._check(self._lib.lbm_warm_crop(m, nxb, nxb, Nx, Nx, 0, None, _ptr(pops),
                                                _ptr(crop), self._st()), "crop")
            self._check(self._lib.lbm_warm_encode_modulus(
                m, nxb, nxb, 1, _ptr(alpha), _ptr(mask), self.E_ref, Nx, Nx, 1,
                _ptr(X[start:]), self._st()), "encode_modulus")
            if self.chan is None:
                self._check(self._lib.lbm_warm_targets(m, Nx, Nx, geo.dx, 3, _ptr(crop),
                                                       _ptr(ones), None, _ptr(T[start:]),
                                                       self._st()), "targets")
                rms = torch.empty(8, dtype=torch.float32, device="cuda")
                self._check(self._lib.lbm_warm_channel_rms(_ptr(T[start:]), m * Nx * Nx,
                                                           _ptr(rms), self._st()), "channel_rms")
                r = rms.cpu().numpy()
                r = np.where(r > 1e-6 * r.max(), r, 0.0)
                self.chan = torch.as_tensor(r.astype(np.float32), device="cuda")
            self._check(self._lib.lbm_warm_targets(m, Nx, Nx, geo.dx, 3, _ptr(crop), _ptr(ones),
                                                   _ptr(self.chan), _ptr(T[start:]),
                                                   self._st()), "targets")
        return X, T

    def predict(self, alpha, out, Nx_fine: int):
        """Initial populations (8 (Nx_fine + 1)^2, FP64 device tensor `out`) of the plate at
        resolution Nx_fine for the modulus E = alpha^2 (alpha: one value, or one per box
        node)."""
        import torch
        if self.chan is None:
            raise RuntimeError("the network has no data normalisation yet: call generate()")
        if Nx_fine % self.Nx:
            raise ValueError("resolution %d is not a multiple of the network's %d"
                             % (Nx_fine, self.Nx))
        factor = Nx_fine // self.Nx
        geo, _, _, mask = self.geometry(Nx_fine)
        nxb = geo.nx
        per_node = alpha.numel() == nxb * nxb
        if not per_node and alpha.numel() != 1:
            raise ValueError("alpha must hold one value or one per box node")
        L._dev_ptr(alpha, alpha.numel())
        L._dev_ptr(out, 8 * nxb * nxb)
        net = self._inference_net()
        self._check(self._lib.lbm_warm_encode_modulus(
            1, nxb, nxb, 1 if per_node else 0, _ptr(alpha), _ptr(mask), self.E_ref, Nx_fine,
            Nx_fine, factor, _ptr(self._x), self._st()), "encode_modulus")
        net.forward(self._x, self._y, exact_acts=True)
        crop = torch.empty(8 * Nx_fine * Nx_fine, dtype=torch.float64, device="cuda")
        self._check(self._lib.lbm_warm_decode(1, self.Nx, self.Nx, factor, geo.dx, 3,
                                              _ptr(self._y), _ptr(self._one), _ptr(self.chan),
                                              _ptr(crop), 0, self._st()), "decode")
        self._check(self._lib.lbm_warm_crop(1, nxb, nxb, Nx_fine, Nx_fine, 1, _ptr(mask),
                                            _ptr(crop), _ptr(out), self._st()), "uncrop")
        return out


def lagrange_weights(xs, x):
    """w with sum_j w_j p(xs_j) = p(x) for every polynomial p of degree < len(xs)
    (Lagrange interpolation/extrapolation at x from distinct abscissae xs)."""
    xs = [float(v) for v in xs]
    w = []
    for i, xi in enumerate(xs):
        t = 1.0
        for j, xj in enumerate(xs):
            if j != i:
                t *= (x - xj) / (xi - xj)
        w.append(t)
    return np.array(w)


def affine_fit_weights(G):
    """Weights of the affine combination of vectors a_0..a_{k-1} closest to a new vector a
    (sum_j w_j = 1, min |sum_j w_j a_j - a|), from the (k+1) x (k+1) inner products of
    (a_0, ..., a_{k-1}, a); minimum-norm solution when the a_j are affinely dependent."""
    k = G.shape[0] - 1
    if k == 1:
        return np.ones(1)
    # a_j - a_last for j < k - 1 and a - a_last, in terms of G
    L = k - 1
    D = np.empty((L, L))
    y = np.empty(L)
    for i in range(L):
        for j in range(L):
            D[i, j] = G[i, j] - G[i, L] - G[L, j] + G[L, L]
        y[i] = G[i, k] - G[i, L] - G[L, k] + G[L, L]
    v = np.linalg.lstsq(D, y, rcond=1e-12)[0]
    return np.concatenate([v, [1.0 - v.sum()]])


def source_fit_weights(G):
    """Least-squares weights of r_0..r_{k-1} for a new r (min |sum_j w_j r_j - r|), from
    the (k+1) x (k+1) inner products of (r_0, ..., r_{k-1}, r)."""
    k = G.shape[0] - 1
    if not np.any(G[:k, :k]):
        return np.zeros(k)
    return np.linalg.lstsq(G[:k, :k], G[:k, k], rcond=1e-12)[0]


def fit_residual(G, w):
    """|sum_j w_j r_j - r| / |r| from the inner products G of (r_0, ..., r_{k-1}, r)."""
    k = G.shape[0] - 1
    c = G[k, k]
    if c <= 0.0:
        return 0.0
    res2 = c - 2.0 * float(w @ G[:k, k]) + float(w @ G[:k, :k] @ w)
    return math.sqrt(max(res2, 0.0) / c)


class WarmStarter:
    """Initial states for the solves of an optimisation loop.

    The solver still iterates every solve to its tolerance; a start only changes the
    number of sweeps.  Sources of a start, in the order they are tried:

    - ``reuse`` with ``history`` >= 2: a combination of the last ``history`` steady
      states.  Primal: the steady state is affine in a force control, so for force
      controls the weights are those of the affine combination of the previous controls
      closest to the new one (exact when the new control lies in their affine span, as
      along a line search); for a scalar Young's modulus E = alpha^2 they extrapolate
      (Lagrange, up to degree history - 1) in 1/E, since the steady displacement scales
      with 1/E for loads that do not depend on E; other controls reuse the last state.
      Adjoint: the steady state is linear in the source r, so the previous adjoint states
      are combined with the least-squares weights that fit the new r by the previous
      ones; if that fit leaves more than ``max_residual`` of |r| unexplained (near an
      optimum r is mostly the primal solve's own residual error, unrelated to the earlier
      sources), the adjoint starts from rest.  A fit whose weights exceed
      ``max_weight`` in magnitude drops its oldest entries.
    - ``reuse`` with ``history`` = 1: the previous steady state.
    - primal / adjoint: trained ``WarmStartNet`` (periodic force-field controls only).
      Without a previous state the network predicts the state; with one, the primal
      network predicts the state of the control's change from the combined (or
      previous) control and it is added; the adjoint network is used only when there is
      no previous state, unless ``adjoint_change`` is set (then previous state + the
      network's state of the change of r; measured over an L-BFGS run on the 512^2
      lattice, that cost more adjoint sweeps than the previous state alone).
    With neither a network nor reuse every solve starts from rest, as in the paper."""

    def __init__(self, primal: Optional[WarmStartNet] = None,
                 adjoint: Optional[WarmStartNet] = None, reuse: bool = True,
                 adjoint_change: bool = False, history: int = 3, max_weight: float = 20.0,
                 max_residual: float = 0.5):
        if not 1 <= history <= 4:
            raise ValueError("history must be 1..4")
        self.primal, self.adjoint, self.reuse = primal, adjoint, reuse
        self.adjoint_change = adjoint_change
        self.history, self.max_weight = int(history), float(max_weight)
        self.max_residual = float(max_residual)
        self.hist_f = []  # (control, feature, steady f_S), newest last
        self.hist_p = []  # (source r, steady adjoint state), newest last
        self._r = None
        self._buf = None

    @property
    def f_prev(self):
        return self.hist_f[-1][2] if self.hist_f else None

    @property
    def p_prev(self):
        return self.hist_p[-1][1] if self.hist_p else None

    def _check(self, solver):
        if isinstance(self.primal, PlateWarmStartNet):
            if solver.periodic or solver.control not in ("young_scalar", "young_field") or \
                    self.adjoint is not None:
                raise ValueError("a plate network serves the primal of Young's-modulus "
                                 "controls on its bounded geometry")
            return
        if (self.primal is not None or self.adjoint is not None) and not (
                solver.periodic and solver.control == "force_field"):
            raise ValueError("warm-start networks serve periodic force-field controls only")

    def _primal_weights(self, solver, F):
        """(entries, weights) of the primal combination, or the newest entry alone."""
        entries = self.hist_f[-self.history:]
        kind = solver.control
        while len(entries) > 1:
            if kind == "young_scalar":
                a = float(F[0])
                x = 1.0 / (a * a) if a != 0.0 else math.inf
                xs = [e[1] for e in entries]
                if len(set(xs)) < len(xs) or not math.isfinite(x):
                    entries = entries[1:]
                    continue
                w = lagrange_weights(xs, x)
            elif kind in ("force_field", "force_basis2"):
                G = L.warm_dots([e[0] for e in entries] + [F.reshape(-1)])
                w = affine_fit_weights(G)
            else:
                break
            if np.all(np.isfinite(w)) and np.abs(w).max() <= self.max_weight:
                return entries, w
            entries = entries[1:]
        return entries[-1:], np.ones(1)

    def before_primal(self, solver, F):
        self._check(solver)
        import torch
        have_prev = self.reuse and bool(self.hist_f)
        if self.primal is None and not have_prev:
            return
        if have_prev:
            entries, w = self._primal_weights(solver, F)
            f0 = torch.empty_like(entries[-1][2])
            L.warm_combine(w, [e[2] for e in entries], f0)
            if self.primal is not None and getattr(self.primal, "net_on_change", True):
                ref = torch.empty_like(F.reshape(-1))
                L.warm_combine(w, [e[0] for e in entries], ref)
                self.primal.predict(F, f0, nx_fine=solver.nx, dx_fine=solver.dx, ref=ref,
                                    accumulate=True)
        elif isinstance(self.primal, PlateWarmStartNet):
            # per-node modulus fields only: for a uniform modulus the network's start is
            # not mirror-symmetric like the plate's state, and the iteration then has to
            # remove antisymmetric components that a start from rest never has (measured:
            # 7.5x more sweeps at N_x = 512), so those solves start from rest
            if solver.control != "young_field":
                return
            f0 = torch.empty(8 * solver.N, dtype=torch.float64, device="cuda")
            self.primal.predict(F.reshape(-1), f0, Nx_fine=solver.nx - 1)
        else:
            f0 = torch.empty(8 * solver.N, dtype=torch.float64, device="cuda")
            self.primal.predict(F, f0, nx_fine=solver.nx, dx_fine=solver.dx)
        solver.set_populations(0, f0)

    def after_primal(self, solver, F):
        if self.reuse:
            a = F.detach().reshape(-1).clone()
            feat = 1.0 / float(a[0]) ** 2 if solver.control == "young_scalar" else None
            self.hist_f.append((a, feat, solver.get_populations(0).clone()))
            del self.hist_f[:-self.history]

    def before_adjoint(self, solver):
        import torch
        have_prev = self.reuse and bool(self.hist_p)
        if self.adjoint is None and not have_prev:
            return
        self._r = solver.adjoint_source()
        if have_prev:
            entries = self.hist_p[-self.history:]
            if self.adjoint is not None and self.adjoint_change:
                p0 = entries[-1][1].clone()
                self.adjoint.predict(self._r, p0, nx_fine=solver.nx, dx_fine=solver.dx,
                                     ref=entries[-1][0], accumulate=True)
            else:
                p0 = torch.empty_like(entries[-1][1])
                if len(entries) == 1 and self.history == 1:
                    w = np.ones(1)
                else:
                    while True:
                        G = L.warm_dots([e[0] for e in entries] + [self._r])
                        w = source_fit_weights(G)
                        if len(entries) == 1 or (np.all(np.isfinite(w)) and
                                                 np.abs(w).max() <= self.max_weight):
                            break
                        entries = entries[1:]
                    if not np.all(np.isfinite(w)) or fit_residual(G, w) > self.max_residual:
                        if self.adjoint is None:
                            return  # from rest
                        w = np.zeros(len(entries))
                L.warm_combine(w, [e[1] for e in entries], p0)
        else:
            p0 = torch.empty(8 * solver.N, dtype=torch.float64, device="cuda")
            self.adjoint.predict(self._r, p0, nx_fine=solver.nx, dx_fine=solver.dx)
        solver.set_populations(2, p0)

    def after_adjoint(self, solver):
        if self.reuse:
            r = self._r if self._r is not None else solver.adjoint_source()
            self.hist_p.append((r, solver.get_populations(2).clone()))
            del self.hist_p[:-self.history]
        self._r = None
