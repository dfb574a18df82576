"""Pins of the oracle's Newton solver, line search and time stepping (CPU only).

* Quadratic convergence near the root with a tight Krylov tolerance, and the
  same iterates as a textbook Newton with a dense LU solve of the complex-step
  Jacobian (numpy.linalg.solve).
* The backtracking line search rescues Newton on arctan from x0 = 10, where
  full steps diverge (a classic case), and the Armijo decrease holds.
* Conservation after a solve: periodic Burgers keeps sum(u) up to ||F||; the
  radiation energy changes by dt times the theta-weighted Marshak flux.
* The Maxwell problem at chi3 = 0 is linear: Newton ends after one step.
* AD and FD (Eq. 7, FP64) reach the same solution of a benign step.
"""
from dataclasses import dataclass

import numpy as np
import pytest

import synthetic_inputs as si
from oracle import jvp, newton as nw, pdes


def test_quadratic_convergence_and_dense_newton_sequence():
    p = pdes.Burgers1D(N=64, nu=1e-2, dt=4e-3)
    u0 = si.burgers_ic(64, 0)
    b = p.rhs(u0)
    opt = nw.Options(restart=64, tol_krylov=1e-14, tol_newton=1e-15, max_newton=6)
    x, rep = nw.newton(p, b, u0, opt)
    h = rep.history
    assert rep.ls_backtracks == 0
    # ||F_{k+1}|| <= C ||F_k||^2 once in the quadratic regime
    ratios = [h[i + 1] / h[i] ** 2 for i in range(len(h) - 1) if h[i + 1] > 1e-13 * h[0]]
    assert len(ratios) >= 2 and max(ratios[1:]) < 10.0 * max(ratios[0], 1.0)
    assert h[-1] < 1e-12 * h[0]
    # textbook Newton with a dense LU solve gives the same iterates
    F = lambda z: p.residual(z, b)
    xd = u0.copy()
    for k in range(3):
        xd = xd - np.linalg.solve(jvp.dense_jacobian(F, xd), F(xd))
        assert np.linalg.norm(F(xd)) == pytest.approx(h[k + 1], rel=1e-6, abs=1e-13)


@dataclass
class _Arctan:
    """F(x) = arctan(x) elementwise: full Newton steps diverge for |x0| > 1.39."""
    n: int = 3
    bvp = True

    @property
    def n_unknowns(self):
        return self.n

    def residual(self, x, b):
        return np.arctan(x)


def test_line_search_rescues_newton_on_arctan():
    x0 = np.array([10.0, -3.0, 0.5])
    opt = nw.Options(restart=3, max_newton=40, tol_newton=1e-12, tol_krylov=1e-13)
    x, rep = nw.newton(_Arctan(), None, x0, opt)
    assert rep.status == "converged"
    assert np.abs(x).max() < 1e-10
    assert rep.ls_backtracks > 0
    assert all(rep.history[i + 1] <= rep.history[i] for i in range(len(rep.history) - 1))
    # without the line search (every trial accepted) the iteration blows up
    bad = nw.Options(restart=3, max_newton=6, tol_newton=1e-12, tol_krylov=1e-13, ls_min_alpha=1.0, ls_c1=-1e30)
    xb, rb = nw.newton(_Arctan(), None, x0, bad)
    assert rb.status != "converged" and np.abs(xb).max() > 1e3


def test_burgers_step_conserves_sum():
    p = pdes.Burgers1D(N=256, nu=1e-2, dt=1e-3)
    u0 = si.burgers_ic(256, 0)
    x, reps = nw.time_steps(p, u0, 2, nw.Options(restart=30, tol_newton=1e-10, tol_krylov=1e-10))
    assert all(r.status == "converged" for r in reps)
    assert abs(x.sum() - u0.sum()) <= np.sqrt(256) * 1e-10 * reps[-1].res0 * 10


def test_su_olson_step_energy_balance():
    nx = ny = 16
    dt, th = 1e-3, 0.5
    p = pdes.SuOlson2D(nx=nx, ny=ny, dt=dt, theta=th)
    x0 = si.su_olson_ic(nx, ny)
    x1, reps = nw.time_steps(p, x0, 1, nw.Options(restart=30, tol_newton=1e-12, tol_krylov=1e-12))
    assert reps[0].status == "converged"
    n = nx * ny
    e0 = (p.M(x0)[:n] + p.M(x0)[n:]).sum() / n
    e1 = (p.M(x1)[:n] + p.M(x1)[n:]).sum() / n
    hy = 1.0 / ny
    flux = lambda x: p.marshak_flux(x[:n].reshape(ny, nx)[:, 0]).sum() * hy
    expect = dt * (th * flux(x1) + (1 - th) * flux(x0))
    assert e1 - e0 == pytest.approx(expect, rel=1e-8)
    assert e1 > e0        # the hot wall heats the cold slab


def test_maxwell_linear_case_one_newton_step():
    n = 12
    p = pdes.MaxwellTE2D(nx=n, ny=n, k=3.0, chi3=0.0, eps_r=si.maxwell_medium(n, n, 0),
                         f=si.maxwell_point_source(n, n))
    opt = nw.Options(restart=60, max_cycles=50, tol_krylov=1e-12, tol_newton=1e-9, max_newton=50)
    x, rep = nw.newton(p, None, np.zeros(2 * n * n), opt)
    assert rep.status == "converged" and rep.newton_its == 1
    # the Born start is that same solve
    xb, brep = nw.born_start(p, opt)
    assert np.allclose(xb, x, rtol=1e-9, atol=1e-12)


def test_ad_and_fd_fp64_reach_same_solution():
    p = pdes.AllenCahn2D(nx=32, ny=32)
    u0 = si.allen_cahn_ic(32, 32, 1)
    xa, ra = nw.time_steps(p, u0, 1, nw.Options(lin="ad", restart=40, tol_newton=1e-10, tol_krylov=1e-10))
    xf, rf = nw.time_steps(p, u0, 1, nw.Options(lin="fd", restart=40, tol_newton=1e-10, tol_krylov=1e-10))
    assert ra[0].status == rf[0].status == "converged"
    assert np.abs(xa - xf).max() <= 1e-9 * np.abs(xa).max()


def test_failure_rule():
    ok = nw.Report(status="converged", res0=1.0, res_final=1e-9)
    near = nw.Report(status="max_newton", res0=1.0, res_final=5e-5)    # within 100 x 1e-6
    far = nw.Report(status="max_newton", res0=1.0, res_final=1e-2)
    assert not nw.run_failed([ok] * 4 + [near], 1e-6)
    assert not nw.run_failed([ok] * 4 + [far], 1e-6)                   # 20% is not "more than 20%"
    assert nw.run_failed([ok] * 3 + [far] * 2, 1e-6)
    assert nw.run_failed([ok, nw.Report(status="breakdown")], 1e-6)
