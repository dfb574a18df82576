"""Pins of the oracle's vector TE Maxwell problem (CPU only).

App. A, Time-Harmonic Maxwell's Equations in Kerr media: curl curl E -
w^2 eps(E) E = i w J with eps(E) = (1 - 0.05 i)(1 + chi |E|), perfectly
conducting walls, the Born start and the block-diagonal CSLP preconditioner.

* Manufactured field with the image symmetries of a conductor (tangential
  components odd, normal components even across the walls): the discrete
  residual converges to the continuous one (sympy) at order 2 on every row
  that is not a PEC row, including the normal components on the walls, and
  the PEC rows vanish.
* At chi = 0 the map is affine: J v = F(v) - F(0). The Kerr term adds
  -w^2 chi [ (dm) (1 - 0.05 i) E + m (1 - 0.05 i) v ] with m = |E|, node by node.
* PEC rows of the Jacobian are rows of the identity.
* Undamped and at chi = 0 the CSLP diagonal is the complex diagonal of the
  Jacobian's interior rows; the right-preconditioned Newton-GMRES solve
  reaches the same field as the plain one.
"""
import math

import numpy as np
import pytest
import sympy as sp

from oracle import jvp, newton as onw, pdes

X, Y = sp.symbols("x y", real=True)


def _field():
    ex = (1 + sp.Rational(1, 2) * sp.I) * sp.cos(sp.pi * X) * sp.sin(sp.pi * Y)
    ey = (sp.Rational(3, 10) - sp.Rational(7, 10) * sp.I) * sp.sin(sp.pi * X) * sp.cos(2 * sp.pi * Y)
    return ex, ey


def _eval_planes(n, exprs):
    xs = np.linspace(0.0, 1.0, n)
    XX, YY = np.meshgrid(xs, xs)
    out = []
    for e in exprs:
        f = sp.lambdify((X, Y), e, "numpy")
        out.append(np.broadcast_to(f(XX, YY), XX.shape).astype(complex))
    return out


def test_mms_order_two_and_pec_rows():
    w, chi = 3.0, 0.2
    ex, ey = _field()
    ccx = sp.diff(ey, X, Y) - sp.diff(ex, Y, 2)
    ccy = sp.diff(ex, X, Y) - sp.diff(ey, X, 2)
    m = sp.sqrt(sp.re(ex) ** 2 + sp.im(ex) ** 2 + sp.re(ey) ** 2 + sp.im(ey) ** 2)
    eps = (1 - sp.Rational(1, 20) * sp.I) * (1 + chi * m)
    Fx, Fy = ccx - w ** 2 * eps * ex, ccy - w ** 2 * eps * ey
    errs, ns = [], [17, 33, 65, 129]
    for n in ns:
        exn, eyn, fxn, fyn = _eval_planes(n, [ex, ey, Fx, Fy])
        x = np.concatenate([exn.real.ravel(), exn.imag.ravel(), eyn.real.ravel(), eyn.imag.ravel()])
        p = pdes.MaxwellVecTE2D(nx=n, ny=n, omega=w, chi=chi)
        F = p.residual(x, None)
        N = n * n
        fa, fb, fc, fd = (F[k * N:(k + 1) * N].reshape(n, n) for k in range(4))
        # PEC rows: Ex on the y walls, Ey on the x walls, which the field makes zero
        assert max(np.abs(fa[[0, -1], :]).max(), np.abs(fc[:, [0, -1]]).max()) < 1e-14
        mx = np.ones((n, n), bool)
        mx[[0, -1], :] = False
        my = np.ones((n, n), bool)
        my[:, [0, -1]] = False
        e = max(np.abs(fa - fxn.real)[mx].max(), np.abs(fb - fxn.imag)[mx].max(),
                np.abs(fc - fyn.real)[my].max(), np.abs(fd - fyn.imag)[my].max())
        errs.append(e)
    orders = [math.log(errs[i] / errs[i + 1]) / math.log((ns[i + 1] - 1) / (ns[i] - 1)) for i in range(len(ns) - 1)]
    assert all(1.9 < o < 2.1 for o in orders), orders


def test_affine_at_zero_kerr_and_kerr_derivative(rng):
    n, w = 9, 4.0
    J = rng.standard_normal(4 * n * n)
    lin = pdes.MaxwellVecTE2D(nx=n, ny=n, omega=w, chi=0.0, J=J)
    x, v = rng.standard_normal(4 * n * n), rng.standard_normal(4 * n * n)
    Jv0 = jvp.jvp_complex_step(lambda z: lin.residual(z, None), x, v)[1]
    Av = lin.residual(v, None) - lin.residual(np.zeros_like(v), None)
    assert np.allclose(Jv0, Av, rtol=1e-12, atol=1e-12 * np.abs(Av).max())
    chi = 0.37
    kerr = pdes.MaxwellVecTE2D(nx=n, ny=n, omega=w, chi=chi, J=J)
    Jk = jvp.jvp_complex_step(lambda z: kerr.residual(z, None), x, v)[1]
    N = n * n
    a, b, c, d = (x[k * N:(k + 1) * N] for k in range(4))
    da, db, dc, dd = (v[k * N:(k + 1) * N] for k in range(4))
    m = np.sqrt(a * a + b * b + c * c + d * d)
    dm = (a * da + b * db + c * dc + d * dd) / m
    lo = 1 - 0.05j
    ex, ey, vx, vy = a + 1j * b, c + 1j * d, da + 1j * db, dc + 1j * dd
    kx = -w * w * chi * lo * (dm * ex + m * vx)
    ky = -w * w * chi * lo * (dm * ey + m * vy)
    extra = np.concatenate([kx.real, kx.imag, ky.real, ky.imag]).reshape(4, n, n)
    # PEC rows carry no Kerr term
    extra[0][[0, -1], :] = 0.0
    extra[1][[0, -1], :] = 0.0
    extra[2][:, [0, -1]] = 0.0
    extra[3][:, [0, -1]] = 0.0
    assert np.allclose(Jk - Jv0, extra.reshape(-1), rtol=1e-11, atol=1e-11 * np.abs(extra).max())


def test_pec_rows_identity_and_cslp_is_the_interior_diagonal(rng):
    n, w = 7, 2.5
    p = pdes.MaxwellVecTE2D(nx=n, ny=n, omega=w, chi=0.0)
    x = rng.standard_normal(4 * n * n)
    Jd = jvp.dense_jacobian(lambda z: p.residual(z, None), x)
    N = n * n
    rows_a = [j * n + i for j in (0, n - 1) for i in range(n)]
    rows_c = [2 * N + j * n + i for j in range(n) for i in (0, n - 1)]
    for r in rows_a + rows_c:
        e = np.zeros(4 * N)
        e[r] = 1.0
        assert np.array_equal(Jd[r], e)
    M = p.cslp_diag(x, damping=0.0)
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            q = j * n + i
            mx, my = M[q], M[N + q]
            assert Jd[q, q] == pytest.approx(mx.real) and Jd[N + q, q] == pytest.approx(mx.imag)
            assert Jd[q, N + q] == pytest.approx(-mx.imag)
            assert Jd[2 * N + q, 2 * N + q] == pytest.approx(my.real)
            assert Jd[3 * N + q, 2 * N + q] == pytest.approx(my.imag)


def test_preconditioned_solve_reaches_the_same_field():
    """Full GMRES (restart = the unknowns) on a 9^2 grid: Born start, then Newton to 1e-10, with and
    without the CSLP right preconditioner, reaches the same field with the same Newton count."""
    n, w = 9, 3.0
    xs = np.linspace(0.0, 1.0, n)
    XX, YY = np.meshgrid(xs, xs)
    J = np.zeros((4, n, n))
    J[0] = np.exp(-((XX - 0.5) ** 2 + (YY - 0.5) ** 2) / (2 * 0.15 ** 2))
    p = pdes.MaxwellVecTE2D(nx=n, ny=n, omega=w, chi=0.05, J=J.reshape(-1))
    o = dict(lin="ad", krylov="gmres", restart=4 * n * n, tol_newton=1e-10, tol_krylov=1e-12, max_newton=30,
             max_cycles=20)
    x1, r1, _ = onw.bvp_solve(p, onw.Options(**o))
    x2, r2, _ = onw.bvp_solve(p, onw.Options(precond="cslp", **o))
    assert r1.status == r2.status == "converged"
    assert r1.newton_its == r2.newton_its
    assert np.abs(x1 - x2).max() <= 1e-8 * np.abs(x1).max()
    # the field is nonzero and satisfies the PEC rows
    assert np.abs(x1).max() > 1e-3
