"""Pins of the oracle's reaction-diffusion problem with the paper's Dirichlet walls (CPU only).

App. A, Nonlinear Reaction-Diffusion: u_t = D lap u - u^3 on [-1/2, 1/2]^2 with
u = 0 on the boundary, Crank-Nicolson, SPD Jacobian, Gaussian / multi-Gaussian
/ sinusoidal initial data and the step dt = C dx^2 / D.

* Manufactured solution vanishing on the walls: the discrete G converges to
  D lap u - u^3 (sympy) at order 2.
* The dense Jacobian equals the paper's J = I - (dt/2) D L + (3 dt/2) diag(u^2)
  with L assembled from 1D Dirichlet second-difference matrices, and is SPD.
* D = 0 decouples the nodes: one Crank-Nicolson step solves the scalar cubic
  (dt/2) u^3 + u = u_n - (dt/2) u_n^3 at every node, whose real root numpy's
  polynomial solver gives.
* CG and GMRES solve the same implicit step to the same state.
"""
import math

import numpy as np
import pytest
import sympy as sp

import synthetic_inputs as si
from oracle import jvp, newton as onw, pdes

X, Y = sp.symbols("x y", real=True)


def _nodes(n):
    return -0.5 + np.arange(1, n + 1) / (n + 1)


def test_dirichlet_mms_order_two():
    D = 0.03
    u = sp.sin(sp.pi * (X + sp.Rational(1, 2))) * sp.sin(2 * sp.pi * (Y + sp.Rational(1, 2)))
    G = D * (sp.diff(u, X, 2) + sp.diff(u, Y, 2)) - u ** 3
    f, g = sp.lambdify((X, Y), u, "numpy"), sp.lambdify((X, Y), G, "numpy")
    errs, ns = [], [31, 63, 127, 255]
    for n in ns:
        XX, YY = np.meshgrid(_nodes(n), _nodes(n))
        p = pdes.AllenCahn2D(nx=n, ny=n, D=D, linear_coef=0.0, dirichlet=True)
        errs.append(np.abs(p.G(f(XX, YY).reshape(-1)) - g(XX, YY).reshape(-1)).max())
    orders = [math.log(errs[i] / errs[i + 1]) / math.log((ns[i + 1] + 1) / (ns[i] + 1)) for i in range(len(ns) - 1)]
    assert all(1.9 < o < 2.1 for o in orders), orders


def _t1(n):
    h = 1.0 / (n + 1)
    return (np.diag(np.full(n - 1, 1.0), 1) + np.diag(np.full(n - 1, 1.0), -1) - 2.0 * np.eye(n)) / (h * h)


def test_dirichlet_jacobian_is_the_papers_and_spd(rng):
    nx, ny, D, dt = 7, 5, 0.02, 0.3
    p = pdes.AllenCahn2D(nx=nx, ny=ny, D=D, dt=dt, theta=0.5, linear_coef=0.0, dirichlet=True)
    u = rng.uniform(-1, 1, nx * ny)
    J = jvp.dense_jacobian(lambda z: p.residual(z, p.rhs(u)), u)
    L = np.kron(np.eye(ny), _t1(nx)) + np.kron(_t1(ny), np.eye(nx))
    J_paper = np.eye(nx * ny) - 0.5 * dt * D * L + 1.5 * dt * np.diag(u * u)
    assert np.allclose(J, J_paper, rtol=1e-12, atol=1e-12 * np.abs(J_paper).max())
    assert np.allclose(J, J.T, atol=1e-12 * np.abs(J).max())
    assert np.linalg.eigvalsh(0.5 * (J + J.T)).min() > 0.0
    # the walls differ from the periodic form: a wrapped neighbour would appear in the corner entries
    Jp = jvp.dense_jacobian(lambda z: pdes.AllenCahn2D(nx=nx, ny=ny, D=D, dt=dt, linear_coef=0.0).residual(z, 0 * z), u)
    assert Jp[0, nx - 1] != 0.0 and J[0, nx - 1] == 0.0


def test_pure_sink_step_solves_the_nodal_cubic(rng):
    n, dt = 9, 0.4
    un = rng.uniform(-1.5, 1.5, n * n)
    p = pdes.AllenCahn2D(nx=n, ny=n, D=0.0, dt=dt, theta=0.5, linear_coef=0.0, dirichlet=True)
    x, reps = onw.time_steps(p, un, 1, onw.Options(lin="ad", krylov="gmres", restart=30, tol_newton=1e-13,
                                                   tol_krylov=1e-13))
    assert reps[0].status == "converged"
    for i in range(0, n * n, 7):
        roots = np.roots([0.5 * dt, 0.0, 1.0, -(un[i] - 0.5 * dt * un[i] ** 3)])
        real = roots[np.abs(roots.imag) < 1e-9].real
        assert real.size == 1 and abs(x[i] - real[0]) < 1e-11


@pytest.mark.parametrize("kind", si.RD_KINDS)
def test_cg_and_gmres_agree_on_the_dirichlet_step(kind):
    n, D = 24, 0.01
    h = 1.0 / (n + 1)
    u0 = si.rd_ic(n, n, kind)
    p = pdes.AllenCahn2D(nx=n, ny=n, D=D, dt=h * h / D, theta=0.5, linear_coef=0.0, dirichlet=True)
    opt = dict(lin="ad", restart=40, tol_newton=1e-12, tol_krylov=1e-12, max_cycles=400)
    xg, rg = onw.time_steps(p, u0, 2, onw.Options(krylov="gmres", **opt))
    xc, rc = onw.time_steps(p, u0, 2, onw.Options(krylov="cg", **opt))
    assert all(r.status == "converged" for r in rg + rc)
    assert np.abs(xg - xc).max() <= 1e-10 * np.abs(xg).max()
    assert u0.max() <= 1.0 and u0.min() >= 0.0
