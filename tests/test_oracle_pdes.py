"""Pins of the oracle's discrete residuals (CPU only).

* Manufactured solutions: the discrete operators converge to the continuous
  ones (written with sympy from the PDEs, not from the discretisation) at
  order 2 in space (the paper's second-order central differences, Sec. 4.1)
  and order 1 for the first-order upwind convection of the 1D Burgers form.
* Conservation identities that hold exactly for the discrete operators:
  periodic Burgers and the Allen-Cahn Laplacian telescope to zero; the
  radiation problem's total energy changes only through the Marshak wall.
* Special case: with the flux limiter off and V = a T^4, the radiation
  residual is the paper's linear Su-Olson Crank-Nicolson residual with
  xi = 1 (App. A, Su-Olson).
"""
import math

import numpy as np
import pytest
import sympy as sp

import synthetic_inputs as si
from oracle import pdes

X, Y = sp.symbols("x y", real=True)


def _eval(expr, xs, ys):
    f = sp.lambdify((X, Y), expr, "numpy")
    XX, YY = np.meshgrid(xs, ys)
    return np.broadcast_to(f(XX, YY), XX.shape)


def _order(errs, ns):
    return [math.log(errs[i] / errs[i + 1]) / math.log(ns[i + 1] / ns[i]) for i in range(len(errs) - 1)]


def test_allen_cahn_mms_order_two():
    D = 3e-2
    u = sp.sin(2 * sp.pi * X) * sp.cos(4 * sp.pi * Y) + sp.Rational(3, 10)
    G = D * (sp.diff(u, X, 2) + sp.diff(u, Y, 2)) + u - u ** 3
    errs, ns = [], [32, 64, 128, 256]
    for n in ns:
        p = pdes.AllenCahn2D(nx=n, ny=n, D=D)
        c = (np.arange(n) + 0.5) / n
        uh = _eval(u, c, c).reshape(-1)
        errs.append(np.abs(p.G(uh) - _eval(G, c, c).reshape(-1)).max())
    assert all(1.9 < o < 2.1 for o in _order(errs, ns)), _order(errs, ns)


def test_burgers_mms_order_one():
    nu = 1e-2
    u = sp.Rational(1, 2) + sp.Rational(3, 10) * sp.sin(2 * sp.pi * X)      # u > 0: left-state flux everywhere
    G = -u * sp.diff(u, X) + nu * sp.diff(u, X, 2)
    f, g = sp.lambdify(X, u), sp.lambdify(X, G)
    errs, ns = [], [64, 128, 256, 512]
    for N in ns:
        x = np.arange(N) / N
        errs.append(np.abs(pdes.Burgers1D(N=N, nu=nu).G(f(x)) - g(x)).max())
    assert all(0.9 < o < 1.1 for o in _order(errs, ns)), _order(errs, ns)


def test_maxwell_mms_order_two_interior():
    k, chi = 6.0, 0.2
    a = sp.sin(3 * X) * sp.cos(2 * Y)
    b = sp.cos(X + Y)
    eps = 1.5
    m2 = a ** 2 + b ** 2
    Gr = sp.diff(a, X, 2) + sp.diff(a, Y, 2) + k ** 2 * (eps + chi * m2) * a
    Gi = sp.diff(b, X, 2) + sp.diff(b, Y, 2) + k ** 2 * (eps + chi * m2) * b
    errs, ns = [], [32, 64, 128, 256]
    for n in ns:
        c = (np.arange(n) + 0.5) / n
        p = pdes.MaxwellTE2D(nx=n, ny=n, k=k, chi3=chi, eps_r=np.full(n * n, eps), f=np.zeros(2 * n * n))
        x = np.concatenate([_eval(a, c, c).reshape(-1), _eval(b, c, c).reshape(-1)])
        g = p.G(x)
        er = (g[: n * n].reshape(n, n) - _eval(Gr, c, c))[1:-1, 1:-1]
        ei = (g[n * n:].reshape(n, n) - _eval(Gi, c, c))[1:-1, 1:-1]
        errs.append(max(np.abs(er).max(), np.abs(ei).max()))
    assert all(1.9 < o < 2.1 for o in _order(errs, ns)), _order(errs, ns)


def test_su_olson_flux_limited_diffusion_mms_order_two_interior():
    sigma, rho = 1.0, 1e-6
    # |grad E| / E is not smooth where grad E = 0, so the field has no critical point
    E = 2 + X + Y / 2 + sp.sin(sp.pi * X) * sp.cos(sp.pi * Y) / 10
    gx, gy = sp.diff(E, X), sp.diff(E, Y)
    Dc = 1 / (3 * sigma + sp.sqrt((gx ** 2 + gy ** 2) / E ** 2 + rho ** 2))
    divDg = sp.diff(Dc * gx, X) + sp.diff(Dc * gy, Y)
    errs, ns = [], [32, 64, 128, 256]
    for n in ns:
        c = (np.arange(n) + 0.5) / n
        p = pdes.SuOlson2D(nx=n, ny=n, sigma=sigma, rho=rho)
        d = p.diffusion(_eval(E, c, c).copy())
        errs.append(np.abs((d - _eval(divDg, c, c))[2:-2, 2:-2]).max())
    assert all(1.85 < o < 2.15 for o in _order(errs, ns)), _order(errs, ns)


def test_burgers_sum_telescopes(rng):
    u = rng.standard_normal(128)
    g = pdes.Burgers1D(N=128).G(u)
    assert abs(g.sum()) <= 1e-12 * np.abs(g).sum()


def test_allen_cahn_laplacian_sums_to_zero(rng):
    p = pdes.AllenCahn2D(nx=20, ny=12, D=0.7)
    u = rng.standard_normal(240)
    assert abs(p.G(u).sum() - (u - u ** 3).sum()) <= 1e-11 * np.abs(p.G(u)).sum()


@pytest.mark.parametrize("limiter", [True, False])
def test_su_olson_energy_changes_only_through_marshak_wall(rng, limiter):
    nx, ny = 10, 7
    p = pdes.SuOlson2D(nx=nx, ny=ny, limiter=limiter)
    x = np.concatenate([rng.uniform(0.1, 2.0, nx * ny), rng.uniform(0.2, 1.2, nx * ny)])
    g = p.G(x)
    E = x[: nx * ny].reshape(ny, nx)
    hx, hy = 1.0 / nx, 1.0 / ny
    # sum over cells of (G_E + G_T) h^2 = total inward flux through the left wall
    total = (g[: nx * ny] + g[nx * ny:]).sum() * hx * hy
    wall = p.marshak_flux(E[:, 0]).sum() * hy
    assert total == pytest.approx(wall, rel=1e-12, abs=1e-13)
    # Marshak flux at equilibrium E_0 = a T_b^4 is zero; cold wall E_0 = 0 gives 2 D_b a T_b^4 / (h + 4 D_b)
    assert p.marshak_flux(np.array([p.a * p.Tb ** 4]))[0] == pytest.approx(0.0, abs=1e-15)
    Db = 1.0 / 3.0
    assert p.marshak_flux(np.array([0.0]))[0] == pytest.approx(2 * Db / (hx + 4 * Db), rel=1e-15)


def test_su_olson_linear_case_is_papers_crank_nicolson(rng):
    """Limiter off, sigma = a = 1, theta = 1/2: F_E, F_T equal the paper's F_U, F_V with xi = 1, Q = 0."""
    nx = ny = 9
    dt = 0.05
    p = pdes.SuOlson2D(nx=nx, ny=ny, sigma=1.0, a=1.0, limiter=False, dt=dt, theta=0.5)
    n = nx * ny
    Un, Uk = rng.uniform(0.5, 1, n), rng.uniform(0.5, 1, n)
    Vn, Vk = rng.uniform(0.5, 1, n), rng.uniform(0.5, 1, n)
    xn = np.concatenate([Un, Vn ** 0.25])
    xk = np.concatenate([Uk, Vk ** 0.25])
    F = p.residual(xk, p.rhs(xn))

    def lap(U):
        U = U.reshape(ny, nx)
        return (np.roll(U, -1, 1) - 2 * U + np.roll(U, 1, 1)) * nx ** 2 + (np.roll(U, -1, 0) - 2 * U + np.roll(U, 1, 0)) * ny ** 2

    FU = (Uk - Un).reshape(ny, nx) - 0.5 * dt * (lap(Uk + Un) / 3 - (Uk + Un - Vk - Vn).reshape(ny, nx))
    FV = Vk - Vn - 0.5 * dt * 1.0 * ((Uk + Un) - (Vk + Vn))
    inner = (slice(1, -1), slice(1, -1))   # the paper's Laplacian and ours agree away from the walls
    assert np.allclose(F[:n].reshape(ny, nx)[inner], FU[inner], rtol=1e-12, atol=1e-13)
    assert np.allclose(F[n:], FV, rtol=1e-12, atol=1e-13)


def test_theta_method_constant_part():
    """F(x^n; b(x^n)) = -dt G(x^n) for any theta: the Eq. 5 denominator is dt ||G(x^n)||."""
    p = pdes.AllenCahn2D(nx=8, ny=8, dt=0.3, theta=0.5)
    u = si.allen_cahn_ic(8, 8, 4)
    assert np.allclose(p.residual(u, p.rhs(u)), -0.3 * p.G(u), rtol=1e-13, atol=1e-15)


def test_maxwell_ghost_coefficient_is_unit_modulus_outgoing():
    p = pdes.MaxwellTE2D(nx=8, ny=8, k=5.0)
    cr, ci = p.ghost_coef(0.1)
    assert cr * cr + ci * ci == pytest.approx(1.0, rel=1e-15)
    # (E_g - E_0)/h = i k (E_g + E_0)/2  (first-order outgoing condition dE/dn = i k E at the wall)
    E0 = 0.3 - 0.7j
    Eg = (cr + 1j * ci) * E0
    assert (Eg - E0) / 0.1 == pytest.approx(1j * 5.0 * (Eg + E0) / 2, rel=1e-14)
