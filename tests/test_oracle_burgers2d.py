"""Pins of the oracle's 2D viscous Burgers problem (CPU only).

App. A, Burgers' Equation: central advection u D_x U + v D_y U, 5-point
diffusion, Crank-Nicolson in time, the adaptive CFL time step, and the TGV,
DSL and 4VC initial conditions on the periodic square [0, 2 pi)^2.

* Manufactured solution: the discrete G converges to -(U.grad)U + nu lap U,
  written with sympy from the PDE, at order 2 (the paper's second-order
  central differences).
* The dense Jacobian of the Crank-Nicolson residual equals the Jacobian
  assembled by hand from Kronecker products of 1D difference matrices.
* CFL rule: closed-form time steps on the node grid where max|u| = 1 exactly,
  and the adaptive step taken inside the oracle's time stepping.
* Symmetry: the Taylor-Green vortex is odd/even under the reflections
  x -> -x and y -> -y; the discrete scheme and the whole Newton-Krylov step
  keep that to round-off.
* Spatial convergence of whole time steps: successive grid differences at
  the shared nodes fall by about 4 per refinement.
"""
import math

import numpy as np
import pytest
import sympy as sp

import synthetic_inputs as si
from oracle import jvp, newton as onw, pdes

X, Y = sp.symbols("x y", real=True)


def _nodes(n, L=2 * math.pi):
    return np.arange(n) * (L / n)


def test_burgers2d_mms_order_two():
    nu = 0.07
    u = sp.sin(X) * sp.cos(2 * Y) + sp.Rational(3, 10)
    v = sp.cos(X + Y) - sp.Rational(1, 5) * sp.sin(Y)
    Gu = -(u * sp.diff(u, X) + v * sp.diff(u, Y)) + nu * (sp.diff(u, X, 2) + sp.diff(u, Y, 2))
    Gv = -(u * sp.diff(v, X) + v * sp.diff(v, Y)) + nu * (sp.diff(v, X, 2) + sp.diff(v, Y, 2))
    ev = lambda e, XX, YY: np.broadcast_to(sp.lambdify((X, Y), e, "numpy")(XX, YY), XX.shape).reshape(-1)
    errs, ns = [], [32, 64, 128, 256]
    for n in ns:
        XX, YY = np.meshgrid(_nodes(n), _nodes(n))
        p = pdes.Burgers2D(nx=n, ny=n, nu=nu)
        g = p.G(np.concatenate([ev(u, XX, YY), ev(v, XX, YY)]))
        errs.append(np.abs(g - np.concatenate([ev(Gu, XX, YY), ev(Gv, XX, YY)])).max())
    orders = [math.log(errs[i] / errs[i + 1]) / math.log(2.0) for i in range(len(errs) - 1)]
    assert all(1.9 < o < 2.1 for o in orders), orders


def _d1(n, h):
    E = np.roll(np.eye(n), 1, axis=1)          # (E u)_i = u_{i+1}
    return (E - E.T) / (2.0 * h)


def _l1(n, h):
    E = np.roll(np.eye(n), 1, axis=1)
    return (E + E.T - 2.0 * np.eye(n)) / (h * h)


def test_burgers2d_jacobian_by_hand(rng):
    nx, ny, nu, dt = 6, 5, 0.03, 0.2
    L = 2 * math.pi
    p = pdes.Burgers2D(nx=nx, ny=ny, nu=nu, dt=dt, theta=0.5)
    x = rng.uniform(-1, 1, 2 * nx * ny)
    J = jvp.dense_jacobian(lambda z: p.residual(z, p.rhs(0.9 * x)), x)
    hx, hy = L / nx, L / ny
    Ix, Iy = np.eye(nx), np.eye(ny)
    Dx, Dy = np.kron(Iy, _d1(nx, hx)), np.kron(_d1(ny, hy), Ix)
    Lap = np.kron(Iy, _l1(nx, hx)) + np.kron(_l1(ny, hy), Ix)
    n = nx * ny
    u, v = x[:n], x[n:]
    conv = np.diag(u) @ Dx + np.diag(v) @ Dy
    dG = np.block([[-(np.diag(Dx @ u) + conv) + nu * Lap, -np.diag(Dy @ u)],
                   [-np.diag(Dx @ v), -(conv + np.diag(Dy @ v)) + nu * Lap]])
    J_hand = np.eye(2 * n) - 0.5 * dt * dG
    assert np.allclose(J, J_hand, rtol=1e-12, atol=1e-12 * np.abs(J_hand).max())
    # nonsymmetric, as the paper notes for the advective problem
    assert not np.allclose(J, J.T, atol=1e-3)


def test_burgers2d_crank_nicolson_residual_vanishes_at_steady_state():
    """A constant field is a steady state of Burgers: F(U; U) = 0 for any dt."""
    p = pdes.Burgers2D(nx=8, ny=6, nu=0.05, dt=0.3)
    x = np.concatenate([np.full(48, 0.7), np.full(48, -0.2)])
    assert np.abs(p.residual(x, p.rhs(x))).max() < 1e-15


@pytest.mark.parametrize("nu,expect", [(0.05, "diffusive"), (0.01, "advective")])
def test_burgers2d_cfl_closed_form(nu, expect):
    n = 64
    h = 2 * math.pi / n
    x = si.burgers2d_ic(n, n, "tgv")
    # the node grid holds x = pi/2 and y = 0, so max|u| = max|v| = 1 exactly
    assert np.abs(x[: n * n]).max() == 1.0 and np.abs(x[n * n:]).max() == 1.0
    p = pdes.Burgers2D(nx=n, ny=n, nu=nu, courant=1.0)
    dt_diff = 1.0 / (2 * nu * (2 / h ** 2))
    want = dt_diff if expect == "diffusive" else h
    assert min(h, dt_diff) == want
    assert p.cfl_dt(x) == pytest.approx(want, rel=1e-15)
    q = pdes.Burgers2D(nx=n, ny=n, nu=nu, courant=0.5)
    assert q.cfl_dt(x) == pytest.approx(0.5 * want, rel=1e-15)
    # a field at rest in one component drops that term
    z = x.copy()
    z[n * n:] = 0.0
    assert p.cfl_dt(z) == pytest.approx(want, rel=1e-15)


def test_burgers2d_adaptive_step_follows_the_state():
    n = 16
    p = pdes.Burgers2D(nx=n, ny=n, nu=0.01, courant=1.0, dt=123.0)
    x0 = si.burgers2d_ic(n, n, "4vc")
    b = p.rhs(x0)
    assert p.dt == pytest.approx(p.cfl_dt(x0), rel=1e-15)
    assert np.allclose(b, x0 + 0.5 * p.dt * p.G(x0), rtol=1e-14, atol=1e-14)
    opts = onw.Options(lin="ad", krylov="gmres", restart=30, tol_newton=1e-10, tol_krylov=1e-10)
    x1, reps = onw.time_steps(p, x0, 2, opts)
    assert all(r.status == "converged" for r in reps)
    # the second step's dt was taken from the first step's result
    x_first, _ = onw.time_steps(pdes.Burgers2D(nx=n, ny=n, nu=0.01, courant=1.0), x0, 1, opts)
    assert p.dt == pytest.approx(p.cfl_dt(x_first), rel=1e-12)


@pytest.mark.parametrize("kind", si.BURGERS2D_KINDS)
def test_burgers2d_initial_conditions(kind):
    n = 32
    x = si.burgers2d_ic(n, n, kind)
    assert x.shape == (2 * n * n,) and np.all(np.isfinite(x))
    u, v = x[: n * n].reshape(n, n), x[n * n:].reshape(n, n)
    xs = _nodes(n)
    if kind == "tgv":
        assert u[0, 8] == pytest.approx(1.0) and v[8, 0] == pytest.approx(-1.0)
    elif kind == "dsl":
        assert np.abs(u).max() <= 1.0 and u[0, 0] == pytest.approx(math.tanh(-30 * math.pi / 2))
        assert np.allclose(v, 0.05 * np.sin(xs)[None, :])
    else:
        # four vortices of alternating sign: the vorticity at the centres alternates
        dvdx = (np.roll(v, -1, 1) - np.roll(v, 1, 1)) / (2 * xs[1])
        dudy = (np.roll(u, -1, 0) - np.roll(u, 1, 0)) / (2 * xs[1])
        w = dvdx - dudy
        assert abs(u[0, 0]) < 1e-10 and abs(v[0, 0]) < 1e-10      # Gaussians vanish at the periodic edge
        idx = [int(round((math.pi + sx) / xs[1])) for sx in (-1.0, 1.0)]
        signs = [np.sign(w[idx[j], idx[i]]) for (i, j) in ((0, 0), (1, 0), (1, 1), (0, 1))]
        assert signs == [1.0, -1.0, 1.0, -1.0]


def test_burgers2d_tgv_reflection_symmetry_survives_newton_steps():
    n = 24
    p = pdes.Burgers2D(nx=n, ny=n, nu=0.05, courant=1.0)
    x0 = si.burgers2d_ic(n, n, "tgv")
    opts = onw.Options(lin="ad", krylov="gmres", restart=30, tol_newton=1e-11, tol_krylov=1e-12)
    x, reps = onw.time_steps(p, x0, 3, opts)
    assert all(r.status == "converged" for r in reps)
    u, v = x[: n * n].reshape(n, n), x[n * n:].reshape(n, n)
    rx = lambda a: np.roll(a[:, ::-1], 1, axis=1)     # a(-x, y) on the periodic node grid
    ry = lambda a: np.roll(a[::-1, :], 1, axis=0)     # a(x, -y)
    s = np.abs(x).max()
    assert np.abs(rx(u) + u).max() < 1e-9 * s and np.abs(rx(v) - v).max() < 1e-9 * s
    assert np.abs(ry(u) - u).max() < 1e-9 * s and np.abs(ry(v) + v).max() < 1e-9 * s
    # the flow has moved, so the symmetry is not the initial state's alone
    assert np.abs(x - x0).max() > 1e-3


def test_burgers2d_spatial_convergence_of_time_steps():
    """Same dt on every grid, so grid differences at shared nodes isolate the O(h^2) spatial error."""
    nu, dt, steps = 0.1, 0.02, 5
    opts = onw.Options(lin="ad", krylov="gmres", restart=40, tol_newton=1e-12, tol_krylov=1e-12)
    sols = {}
    for n in (16, 32, 64):
        p = pdes.Burgers2D(nx=n, ny=n, nu=nu, dt=dt)
        x, reps = onw.time_steps(p, si.burgers2d_ic(n, n, "tgv"), steps, opts)
        assert all(r.status == "converged" for r in reps)
        sols[n] = x[: n * n].reshape(n, n)
    d16 = np.abs(sols[16] - sols[32][::2, ::2]).max()
    d32 = np.abs(sols[32] - sols[64][::2, ::2])[::2, ::2].max()
    assert 3.6 < d16 / d32 < 4.4, d16 / d32
