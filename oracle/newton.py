"""Newton's method with backtracking line search, time stepping (oracle; test infrastructure).

Follows the solver of Sec. 2 and Sec. 3.1:

* each Newton step solves J(x^k) dx = -F(x^k) (Eq. 4) with a matrix-free
  Krylov method whose operator is the AD JVP (Eq. 9; here the complex step,
  which returns the same derivative) or the FD JVP (Eq. 7, step of Eq. 8 or
  the scaled rule);
* the iteration stops when ||F(x^k)|| / ||F(x*)|| < tol_Newton (Eq. 5), x*
  being the previous converged state (or the initial guess);
* after each Krylov solve a backtracking line search replaces x + dx by
  x + alpha dx, alpha halved until sufficient decrease. The paper does not fix
  the test; this oracle uses the Armijo condition on the residual norm,
  ||F(x + alpha dx)|| <= (1 - c1 alpha) ||F(x)|| with c1 = 1e-4, and accepts
  the smallest trial alpha_min = 2^-10 when no trial passes (counted as a
  line-search failure);
* the outer continuation (Sec. 3.1) is implicit time stepping for the
  initial-boundary-value problems (previous state as initial guess) and, for
  the Maxwell problem, a Born start: the linear problem at chi3 = 0 solved once
  from zero.
"""
from __future__ import annotations

import copy
from dataclasses import dataclass, field

import numpy as np

from . import jvp as _jvp
from . import krylov as _kr
from . import pdes as _pdes


@dataclass
class Options:
    lin: str = "ad"            # "ad" | "fd"
    krylov: str = "gmres"      # "gmres" | "bicgstab" | "cg"
    ortho: str = "cgs2"        # GMRES Arnoldi: "cgs2" | "dcgs2" (second pass delayed one step)
    restart: int = 30
    max_cycles: int = 100      # GMRES restart cycles; iteration cap for BiCGSTAB / CG
    max_newton: int = 15
    tol_newton: float = 1e-6
    tol_krylov: float = 1e-8
    fd_rule: str = "scaled"    # "scaled" (sqrt(eps)(1+|x|)/|v|) | "paper" (Eq. 8)
    fd_eps: float = 0.0        # > 0: fixed step, overrides the rule
    ls_c1: float = 1e-4
    ls_min_alpha: float = 2.0 ** -10
    precond: str = "none"      # GMRES right preconditioner: "none" | "cslp" (Maxwell, App. A)
    precond_damping: float = 0.5


@dataclass
class Report:
    status: str = "running"    # converged | max_newton | breakdown | nonfinite
    newton_its: int = 0
    krylov_its: int = 0
    jvp_calls: int = 0
    ls_backtracks: int = 0
    ls_failures: int = 0
    krylov_failures: int = 0
    res0: float = 0.0
    res_final: float = 0.0
    history: list = field(default_factory=list)
    alphas: list = field(default_factory=list)   # accepted line-search step of each Newton iteration


def _operator(problem, b, x, Fx, opt: Options, rep: Report):
    """Matrix-free v -> J(x) v with the chosen linearisation."""
    Fres = lambda z: problem.residual(z, b)
    if opt.lin == "ad":
        def A(v):
            rep.jvp_calls += 1
            return _jvp.jvp_complex_step(Fres, x, v)[1]
        return A
    if opt.fd_eps > 0.0:
        eps_fixed = opt.fd_eps
    elif opt.fd_rule == "paper":
        eps_fixed = _jvp.fd_eps_paper(x)
    else:
        eps_fixed = None

    def A(v):
        rep.jvp_calls += 1
        eps = eps_fixed if eps_fixed is not None else _jvp.fd_eps_scaled(x, v)
        return _jvp.jvp_fd(Fres, x, v, eps, Fx)
    return A


def _right_preconditioned(problem, x, A, opt: Options):
    """(operator v -> J M^-1 v, map y -> M^-1 y) of the right preconditioner at x, or (A, None)."""
    if opt.precond == "none":
        return A, None
    if opt.precond != "cslp":
        raise ValueError(opt.precond)
    minv = 1.0 / problem.cslp_diag(x, opt.precond_damping)
    apply = getattr(problem, "apply_diag", None) or _pdes.apply_cell_complex
    P = lambda y: apply(minv, y)
    return (lambda v: A(P(v))), P


def _solve_step(problem, x, A, rhs, opt: Options):
    """Krylov solve of J d = rhs, right-preconditioned when opt.precond says so: d = M^-1 y, J M^-1 y = rhs."""
    Ap, P = _right_preconditioned(problem, x, A, opt)
    kr = _krylov(Ap, rhs, opt)
    if P is not None:
        kr.x = P(kr.x)
    return kr


def _krylov(A, rhs, opt: Options):
    if opt.krylov == "gmres":
        if opt.ortho == "dcgs2":
            return _kr.gmres_dcgs2(A, rhs, opt.restart, opt.tol_krylov, opt.max_cycles)
        return _kr.gmres(A, rhs, opt.restart, opt.tol_krylov, opt.max_cycles)
    if opt.krylov == "bicgstab":
        return _kr.bicgstab(A, rhs, opt.tol_krylov, opt.max_cycles)
    if opt.krylov == "cg":
        return _kr.cg(A, rhs, opt.tol_krylov, opt.max_cycles)
    raise ValueError(opt.krylov)


def newton(problem, b, x0: np.ndarray, opt: Options, denom: float | None = None):
    """Solve F(x; b) = 0 from x0; returns (x, Report). denom defaults to ||F(x0)||."""
    rep = Report()
    x = x0.astype(np.float64).copy()
    F = problem.residual(x, b)
    fnorm = float(np.linalg.norm(F))
    f0 = fnorm if denom is None else denom
    rep.res0 = f0
    rep.history.append(fnorm)
    for k in range(opt.max_newton + 1):
        if not np.isfinite(fnorm):
            rep.status = "nonfinite"
            break
        if f0 == 0.0 or fnorm / f0 < opt.tol_newton:
            rep.status = "converged"
            break
        if k == opt.max_newton:
            rep.status = "max_newton"
            break
        A = _operator(problem, b, x, F, opt, rep)
        kr = _solve_step(problem, x, A, -F, opt)
        rep.krylov_its += kr.iterations
        if kr.breakdown:
            rep.status = "breakdown"
            break
        if not kr.converged:
            rep.krylov_failures += 1
        dx = kr.x
        alpha = 1.0
        while True:
            xt = x + alpha * dx
            Ft = problem.residual(xt, b)
            ft = float(np.linalg.norm(Ft))
            if np.isfinite(ft) and ft <= (1.0 - opt.ls_c1 * alpha) * fnorm:
                break
            if alpha * 0.5 < opt.ls_min_alpha:
                rep.ls_failures += 1
                break
            alpha *= 0.5
            rep.ls_backtracks += 1
        x, F, fnorm = xt, Ft, ft
        rep.alphas.append(alpha)
        rep.newton_its += 1
        rep.history.append(fnorm)
    rep.res_final = fnorm
    return x, rep


def time_steps(problem, xn: np.ndarray, steps: int, opt: Options):
    """Advance ``steps`` implicit steps; each Newton solve starts from the previous state."""
    reports = []
    x = xn.astype(np.float64).copy()
    for _ in range(steps):
        b = problem.rhs(x)
        x_new, rep = newton(problem, b, x, opt)
        reports.append(rep)
        if rep.status in ("nonfinite", "breakdown"):
            return x_new, reports
        x = x_new
    return x, reports


def born_start(problem, opt: Options):
    """Initial guess for the Maxwell problem: the chi3 = 0 linear problem solved from zero.

    Returns (x_born, Report of that linear solve)."""
    if hasattr(problem, "born"):
        lin = problem.born()
    else:
        lin = copy.copy(problem)
        lin.chi3 = 0.0
    x0 = np.zeros(problem.n_unknowns)
    F0 = lin.residual(x0, None)
    rep = Report(res0=float(np.linalg.norm(F0)))
    A = _operator(lin, None, x0, F0, opt, rep)
    kr = _solve_step(lin, x0, A, -F0, opt)
    rep.krylov_its = kr.iterations
    rep.status = "converged" if kr.converged else ("breakdown" if kr.breakdown else "max_newton")
    rep.res_final = float(np.linalg.norm(lin.residual(kr.x, None)))
    return kr.x, rep


def bvp_solve(problem, opt: Options):
    """Born start, then Newton on the full problem with ||F(x_born)|| as the Eq. 5 denominator."""
    xb, brep = born_start(problem, opt)
    x, rep = newton(problem, None, xb, opt)
    return x, rep, brep


def run_failed(reports, tol_newton: float) -> bool:
    """Failure rule of Sec. 3.4 for a time-dependent run.

    Failed when any step ended on non-finite values or a breakdown, or when
    more than 20% of the steps missed 100 x tol_Newton.
    """
    if any(r.status in ("nonfinite", "breakdown") for r in reports):
        return True
    missed = sum(1 for r in reports
                 if not (r.res0 == 0.0 or r.res_final / r.res0 < 100.0 * tol_newton))
    return missed > 0.2 * len(reports)
