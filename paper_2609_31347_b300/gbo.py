"""Gradient-based optimisation on top of the CUDA solver (host orchestration).

- ``LBMObjective``: a ``torch.autograd.Function`` whose forward runs the primal solve
  and the objective (Algorithm 2, its primal step) and whose backward runs the adjoint solve and
  the gradient (Algorithm 1, Eq. optimality).  A control at which the primal iteration
  diverges (no steady state, e.g. a modulus that makes the boundary collision singular)
  gets J = +inf, so that the line search steps back.  Only the steady primal state f_S is kept
  for the backward pass (the adjoint of a steady problem needs no trajectory); it is
  restored into the handle if another forward ran in between.
- ``lbfgs``: limited-memory BFGS (two-loop recursion) with a line search satisfying the
  strong Wolfe conditions, and the termination rules of Algorithm 2: gradient norm
  below eps, relative control change below eps_alpha for every component, or m_max
  steps.  Parameters mirror Tables 2-4 (l, lambda0, k_max, m_max, eps, eps_alpha).

All vectors stay on the GPU as float64 tensors; the per-iteration host work is a few
dot products.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import torch

from .lbm import LBM_ERR_DIVERGED


@dataclass
class SolveOpts:
    """Stopping rule used for the primal and adjoint solves of every evaluation."""
    max_steps: int = 2_000_000
    tol: float = 1e-10
    criterion: int = 1          # 1 residual rule, 0 CV window of Eq. convergence_crit
    window: int = 100
    check_every: int = 64
    fixed_steps: bool = False

    def kw(self):
        return dict(max_steps=self.max_steps, tol=self.tol, criterion=self.criterion,
                    window=self.window, check_every=self.check_every,
                    fixed_steps=self.fixed_steps, allow_not_converged=True)


class LBMObjective(torch.autograd.Function):
    """J(alpha) with dJ/dalpha from the discrete adjoint."""

    @staticmethod
    def forward(ctx, alpha, solver, primal: SolveOpts, adjoint: SolveOpts, project: bool,
                warm=None):
        a = alpha.detach().contiguous()
        solver.set_control(a)
        if warm is not None:
            warm.before_primal(solver, a)
        info = solver.primal_solve(**primal.kw())
        ctx.solver, ctx.adjoint, ctx.project, ctx.warm = solver, adjoint, project, warm
        ctx.failed = info.status == LBM_ERR_DIVERGED  # no steady state at this control
        if ctx.failed:
            # J = +inf makes the line search step back; the gradient is not used
            ctx.alpha = alpha.detach().clone()
            return alpha.new_tensor(float("inf"))
        J = solver.objective()
        if not math.isfinite(J):
            ctx.failed = True
            ctx.alpha = alpha.detach().clone()
            return alpha.new_tensor(float("inf"))
        if warm is not None:
            warm.after_primal(solver, a)
        ctx.fS = solver.get_populations(0).clone()  # steady-state checkpoint
        ctx.alpha = alpha.detach().clone()
        solver._state_token = id(ctx)
        ctx.token = id(ctx)
        return alpha.new_tensor(J)

    @staticmethod
    def backward(ctx, gJ):
        if ctx.failed:
            return torch.zeros_like(ctx.alpha), None, None, None, None, None
        s = ctx.solver
        if getattr(s, "_state_token", None) != ctx.token:
            # another evaluation overwrote the handle: restore control and steady state
            s.set_control(ctx.alpha)
            s.set_populations(0, ctx.fS)
            s.primal_solve(1, fixed_steps=True)
            s._state_token = ctx.token
        if ctx.warm is not None:
            ctx.warm.before_adjoint(s)
        info = s.adjoint_solve(**ctx.adjoint.kw())
        if info.status == LBM_ERR_DIVERGED:
            raise RuntimeError("adjoint solve diverged at a control whose primal converged")
        if ctx.warm is not None:
            ctx.warm.after_adjoint(s)
        g = s.gradient(project_zero_mean=ctx.project)
        return gJ * g.view_as(ctx.alpha), None, None, None, None, None


def objective(alpha, solver, primal: Optional[SolveOpts] = None,
              adjoint: Optional[SolveOpts] = None, project: bool = False, warm=None):
    """J(alpha) as a differentiable torch scalar.  warm: optional initial-state supplier
    (``warmstart.WarmStarter``) for the primal and adjoint solves."""
    return LBMObjective.apply(alpha, solver, primal or SolveOpts(), adjoint or SolveOpts(),
                              project, warm)


@dataclass
class LBFGSResult:
    alpha: torch.Tensor
    J: float
    grad_norm: float
    steps: int
    reason: str
    history: List[dict] = field(default_factory=list)


def _dot(a, b):
    return float(torch.dot(a.reshape(-1), b.reshape(-1)))


def _cubic_min(a0, f0, g0, a1, f1, g1):
    """Minimiser of the cubic through (a0, f0, g0), (a1, f1, g1) (Nocedal & Wright 3.59);
    None if it does not exist."""
    if a0 == a1:
        return None
    d1 = g0 + g1 - 3.0 * (f0 - f1) / (a0 - a1)
    disc = d1 * d1 - g0 * g1
    if disc < 0:
        return None
    d2 = (1.0 if a1 > a0 else -1.0) * disc ** 0.5
    den = g1 - g0 + 2.0 * d2
    if den == 0:
        return None
    return a1 - (a1 - a0) * (g1 + d2 - d1) / den


def _zoom(fg, x, d, f0, g0d, lo, hi, c1, c2, kmax, evals):
    # Zoom phase of the strong-Wolfe line search: lo, hi = [a, f(a), f'(a)], the
    # interval containing steps that satisfy the conditions (Nocedal & Wright Alg. 3.6).
    while evals[0] < kmax:
        width = hi[0] - lo[0]
        a = _cubic_min(lo[0], lo[1], lo[2], hi[0], hi[1], hi[2])
        lo_b, hi_b = min(lo[0], hi[0]), max(lo[0], hi[0])
        if a is None or not (lo_b + 0.1 * abs(width) <= a <= hi_b - 0.1 * abs(width)):
            a = 0.5 * (lo[0] + hi[0])
        fa, ga = fg(x + a * d)
        evals[0] += 1
        gad = _dot(ga, d)
        if fa > f0 + c1 * a * g0d or fa >= lo[1]:
            hi[:] = [a, fa, gad]
        else:
            if abs(gad) <= -c2 * g0d:
                return a, fa, ga
            if gad * (hi[0] - lo[0]) >= 0:
                hi[:] = list(lo)
            lo[:] = [a, fa, gad]
        if abs(hi[0] - lo[0]) <= 1e-16 * max(1.0, abs(lo[0])):
            break
    return None


def strong_wolfe(fg, x, f0, g0, d, lam0=1.0, c1=1e-4, c2=0.9, kmax=100):
    """Step length satisfying the strong Wolfe conditions (bracketing with cubic
    extrapolation, then zoom; Nocedal & Wright Alg. 3.5)."""
    g0d = _dot(g0, d)
    if g0d >= 0:
        return None
    evals = [0]
    prev = [0.0, f0, g0d]
    a = lam0
    while evals[0] < kmax:
        fa, ga = fg(x + a * d)
        evals[0] += 1
        gad = _dot(ga, d)
        cur = [a, fa, gad]
        if fa > f0 + c1 * a * g0d or (evals[0] > 1 and fa >= prev[1]):
            return _zoom(fg, x, d, f0, g0d, prev, cur, c1, c2, kmax, evals)
        if abs(gad) <= -c2 * g0d:
            return a, fa, ga
        if gad >= 0:
            return _zoom(fg, x, d, f0, g0d, cur, prev, c1, c2, kmax, evals)
        # still descending: extrapolate (cubic minimiser clipped to [2a, 10a])
        t = _cubic_min(prev[0], prev[1], prev[2], a, fa, gad)
        prev = cur
        a = min(max(t if t is not None else 4.0 * a, 2.0 * a), 10.0 * a)
    return None


def lbfgs(fg: Callable, alpha0: torch.Tensor, m_max: int = 50, eps: float = 1e-10,
          eps_alpha: float = 2.2e-16, history: int = 20, lam0: float = 1.0,
          gamma0: Optional[float] = None, k_max: int = 100,
          norm: Optional[Callable] = None, f_target: Optional[float] = None) -> LBFGSResult:
    """Minimise J with L-BFGS (Algorithm 2).  fg(alpha) -> (J, dJ/dalpha).

    f_target (optional, not part of Algorithm 2): also stop once J <= f_target, to compare
    runs by the work they need to reach the same objective.

    gamma0 scales the first step's direction (H0 = gamma0 I before any curvature pair;
    None: 1 / |g|_1); later steps use the usual s'y / y'y scaling.  norm(g) is the
    gradient norm of the termination test (Euclidean by default; the distributed control
    uses the L2 norm).
    """
    norm = norm or (lambda g: float(torch.linalg.vector_norm(g)))
    x = alpha0.detach().clone()
    f, g = fg(x)
    S, Y, R = [], [], []
    hist = [{"J": f, "grad_norm": norm(g)}]
    for m in range(m_max):
        gn = norm(g)
        if gn < eps:
            return LBFGSResult(x, f, gn, m, "gradient", hist)
        if f_target is not None and f <= f_target:
            return LBFGSResult(x, f, gn, m, "target", hist)
        # two-loop recursion: d = -H g
        q = g.clone()
        al = []
        for s_, y_, r_ in reversed(list(zip(S, Y, R))):
            a_ = r_ * _dot(s_, q)
            al.append(a_)
            q -= a_ * y_
        if S:
            q *= _dot(S[-1], Y[-1]) / _dot(Y[-1], Y[-1])
        else:
            q *= gamma0 if gamma0 is not None else 1.0 / max(float(g.abs().sum()), 1e-300)
        for (s_, y_, r_), a_ in zip(zip(S, Y, R), reversed(al)):
            b_ = r_ * _dot(y_, q)
            q += (a_ - b_) * s_
        d = -q
        ls = strong_wolfe(fg, x, f, g, d, lam0=lam0, kmax=k_max)
        if ls is None:
            return LBFGSResult(x, f, gn, m, "line search", hist)
        a, fn, gnew = ls
        s_ = a * d
        xn = x + s_
        y_ = gnew - g
        sy = _dot(s_, y_)
        if sy > 1e-300:
            S.append(s_)
            Y.append(y_)
            R.append(1.0 / sy)
            if len(S) > history:
                S.pop(0), Y.pop(0), R.pop(0)
        rel = torch.abs(2.0 * s_ / (xn + x))
        x, f, g = xn, fn, gnew
        hist.append({"J": f, "grad_norm": norm(g), "step": a})
        if bool(torch.all(rel < eps_alpha)):
            return LBFGSResult(x, f, norm(g), m + 1, "control change", hist)
    if f_target is not None and f <= f_target:
        return LBFGSResult(x, f, norm(g), m_max, "target", hist)
    return LBFGSResult(x, f, norm(g), m_max, "m_max", hist)


def make_fg(solver, primal: Optional[SolveOpts] = None, adjoint: Optional[SolveOpts] = None,
            project: bool = False, warm=None):
    """(J, grad) closure for lbfgs through the autograd function."""
    def fg(a):
        a = a.detach().clone().requires_grad_(True)
        J = objective(a, solver, primal, adjoint, project, warm)
        J.backward()
        return float(J.detach()), a.grad.detach().clone()
    return fg
