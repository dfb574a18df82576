"""Pins of the oracle's JVPs against what the mathematics fixes (CPU only).

* Taylor remainder: ||F(x + t v) - F(x) - t Jv|| = O(t^2) for every PDE, so a
  dropped or wrong derivative term (which leaves an O(t) remainder) fails.
* Closed-form Jacobians: the reaction-diffusion Jacobian the paper prints
  (App. A, Nonlinear Reaction-Diffusion), and the upwind Burgers Jacobian
  derived by hand.
* Structure: SPD Jacobian for the paper's reaction-diffusion form; the
  Maxwell map is affine at chi3 = 0 and its Kerr derivative is pointwise.
* FD quotient (Eq. 7): the truncation / round-off U-curve in FP64 and FP32,
  with its minimum near sqrt(eps_mach) (Eq. 8), and the two step rules.
"""
import math

import numpy as np
import pytest

import synthetic_inputs as si
from oracle import jvp, pdes


def _problems(rng):
    n = 12
    out = []
    b = pdes.Burgers1D(N=32, nu=1e-2, dt=1e-3)
    x = 0.6 + 0.3 * np.sin(2 * np.pi * np.arange(32) / 32)      # face speeds well away from 0
    out.append(("burgers", b, x, b.rhs(x + 0.01)))
    a = pdes.AllenCahn2D(nx=n, ny=n + 2, D=1e-3, dt=0.1)
    x = rng.uniform(-1, 1, a.n_unknowns)
    out.append(("allen_cahn", a, x, a.rhs(x * 0.9)))
    s = pdes.SuOlson2D(nx=n, ny=n + 2, dt=1e-2)
    x = np.concatenate([rng.uniform(0.2, 1.0, n * (n + 2)), rng.uniform(0.3, 1.0, n * (n + 2))])
    out.append(("su_olson", s, x, s.rhs(x * 0.95)))
    m = pdes.MaxwellTE2D(nx=n, ny=n + 2, k=7.0, chi3=0.3, eps_r=si.maxwell_medium(n, n + 2, 1),
                         f=si.maxwell_point_source(n, n + 2))
    x = rng.standard_normal(m.n_unknowns)
    out.append(("maxwell", m, x, None))
    g = pdes.Burgers2D(nx=n, ny=n + 2, nu=0.05, dt=0.05)
    x = rng.uniform(-1, 1, g.n_unknowns)
    out.append(("burgers2d", g, x, g.rhs(x * 0.9)))
    mv = pdes.MaxwellVecTE2D(nx=n, ny=n + 2, omega=4.0, chi=0.3, J=rng.standard_normal(4 * n * (n + 2)))
    out.append(("maxwell_vec", mv, rng.standard_normal(mv.n_unknowns), None))
    return out


@pytest.mark.parametrize("idx", range(6))
def test_taylor_remainder_is_second_order(rng, idx):
    name, p, x, b = _problems(rng)[idx]
    v = rng.standard_normal(x.size)
    if name == "su_olson":
        v *= 0.1
    F = lambda z: p.residual(z, b)
    F0, Jv = jvp.jvp_complex_step(F, x, v)
    assert np.allclose(F0, F(x), rtol=1e-14, atol=1e-14 * np.abs(F0).max())
    ts = [1e-2 * 2.0 ** -i for i in range(6)]
    rem = [np.linalg.norm(F(x + t * v) - F0 - t * Jv) for t in ts]
    ratios = [rem[i] / rem[i + 1] for i in range(len(ts) - 1)]
    # a correct derivative leaves an O(t^2) remainder: each halving divides it by 4
    assert all(3.6 < r < 4.4 for r in ratios), (name, ratios)
    # a derivative with one term dropped leaves O(t): check the test would see it
    bad = Jv.copy()
    bad[bad.size // 2] += 1e-3 * np.abs(Jv).max() + 1e-3
    rem_bad = [np.linalg.norm(F(x + t * v) - F0 - t * bad) for t in ts]
    assert rem_bad[-2] / rem_bad[-1] < 2.5


def test_reaction_diffusion_jacobian_closed_form(rng):
    """The paper's RD Jacobian J = I - (dt/2) D L + (3 dt / 2) diag(u^2) (theta = 1/2, no +u term)."""
    nx, ny, D, dt = 7, 5, 0.03, 0.2
    p = pdes.AllenCahn2D(nx=nx, ny=ny, D=D, dt=dt, theta=0.5, linear_coef=0.0)
    u = rng.uniform(-1, 1, nx * ny)
    J = jvp.dense_jacobian(lambda z: p.residual(z, p.rhs(u)), u)

    def lap1(n, h):
        L = -2.0 * np.eye(n) + np.roll(np.eye(n), 1, axis=1) + np.roll(np.eye(n), -1, axis=1)
        return L / (h * h)
    L = np.kron(np.eye(ny), lap1(nx, 1.0 / nx)) + np.kron(lap1(ny, 1.0 / ny), np.eye(nx))
    J_paper = np.eye(nx * ny) - 0.5 * dt * D * L + 1.5 * dt * np.diag(u * u)
    assert np.allclose(J, J_paper, rtol=1e-12, atol=1e-12 * np.abs(J_paper).max())
    # symmetric positive definite, as the paper states for this problem
    assert np.allclose(J, J.T, atol=1e-12 * np.abs(J).max())
    assert np.linalg.eigvalsh(0.5 * (J + J.T)).min() > 0.0
    # the Allen-Cahn variant adds -theta dt I from the +u term
    q = pdes.AllenCahn2D(nx=nx, ny=ny, D=D, dt=dt, theta=0.5, linear_coef=1.0)
    Jq = jvp.dense_jacobian(lambda z: q.residual(z, q.rhs(u)), u)
    assert np.allclose(Jq, J_paper - 0.5 * dt * np.eye(nx * ny), rtol=1e-12, atol=1e-12 * np.abs(J).max())


def test_burgers_upwind_jacobian_by_hand(rng):
    N, nu, dt = 16, 0.02, 0.01
    p = pdes.Burgers1D(N=N, nu=nu, dt=dt)
    u = rng.uniform(-1, 1, N)
    J = jvp.dense_jacobian(lambda z: p.residual(z, p.rhs(u)), u)
    h = 1.0 / N
    # dPhi_{i+1/2}/du: u_i on the left state when u_i + u_{i+1} >= 0, else u_{i+1} on the right
    dG = np.zeros((N, N))
    for i in range(N):
        for face, sgn in ((i, -1.0), ((i - 1) % N, +1.0)):       # +Phi_{i-1/2}, -Phi_{i+1/2}
            l, r = face, (face + 1) % N
            upw = l if u[l] + u[r] >= 0 else r
            dG[i, upw] += sgn * u[upw] / h
        dG[i, i] += -2.0 * nu / h ** 2
        dG[i, (i + 1) % N] += nu / h ** 2
        dG[i, (i - 1) % N] += nu / h ** 2
    assert np.allclose(J, np.eye(N) - dt * dG, rtol=1e-12, atol=1e-12)


def test_maxwell_affine_at_zero_kerr_and_kerr_derivative(rng):
    n = 9
    eps = si.maxwell_medium(n, n, 3)
    f = si.maxwell_point_source(n, n)
    lin = pdes.MaxwellTE2D(nx=n, ny=n, k=11.0, chi3=0.0, eps_r=eps, f=f)
    x = rng.standard_normal(2 * n * n)
    v = rng.standard_normal(2 * n * n)
    F = lambda z: lin.residual(z, None)
    Jv = jvp.jvp_complex_step(F, x, v)[1]
    # G(x) = A x - f is affine: J v = G(v) - G(0)
    Av = F(v) - F(np.zeros_like(v))
    assert np.allclose(Jv, Av, rtol=1e-12, atol=1e-12 * np.abs(Av).max())
    # the Kerr term k^2 chi3 |E|^2 E adds k^2 chi3 [ |E|^2 dE + 2 E (a da + b db) ] per cell
    chi = 0.37
    kerr = pdes.MaxwellTE2D(nx=n, ny=n, k=11.0, chi3=chi, eps_r=eps, f=f)
    Jk = jvp.jvp_complex_step(lambda z: kerr.residual(z, None), x, v)[1]
    a, b = x[: n * n], x[n * n:]
    da, db = v[: n * n], v[n * n:]
    m2 = a * a + b * b
    dot = a * da + b * db
    extra = 11.0 ** 2 * chi * np.concatenate([m2 * da + 2 * a * dot, m2 * db + 2 * b * dot])
    assert np.allclose(Jk - Jv, extra, rtol=1e-11, atol=1e-11 * np.abs(extra).max())


def test_fd_error_u_curve_fp64_and_fp32(rng):
    """FD error vs eps: O(eps) truncation on the right, O(eps_mach / eps) round-off on the left."""
    p = pdes.AllenCahn2D(nx=16, ny=16, D=1e-3, dt=0.1)
    x = rng.uniform(-1, 1, 256)
    v = rng.standard_normal(256)
    b = p.rhs(0.9 * x)
    Jv = jvp.jvp_complex_step(lambda z: p.residual(z, b), x, v)[1]
    for dtype in (np.float64, np.float32):
        xd, vd, bd = x.astype(dtype), v.astype(dtype), b.astype(dtype)
        F = lambda z: p.residual(z, bd)
        assert F(xd).dtype == dtype
        epss = 10.0 ** np.arange(-13 if dtype == np.float64 else -6, 0.0, 1.0)
        err = np.array([np.linalg.norm(jvp.jvp_fd(F, xd, vd, e).astype(np.float64) - Jv)
                        for e in epss]) / np.linalg.norm(Jv)
        em = np.finfo(dtype).eps
        # truncation branch: slope +1 over the two largest steps
        assert 0.8 < math.log10(err[-1] / err[-2]) < 1.2
        # round-off branch: the smallest step is much worse than the best one
        assert err[0] > 30.0 * err.min()
        # the best step sits within a decade or two of sqrt(eps_mach) and gives ~sqrt(eps_mach)
        best = epss[int(np.argmin(err))]
        assert 1e-2 * math.sqrt(em) <= best <= 1e2 * math.sqrt(em)
        assert err.min() < 30.0 * math.sqrt(em)


def test_fd_step_rules():
    x = np.array([3.0, 4.0])          # ||x|| = 5
    v = np.array([0.0, 2.0])          # ||v|| = 2
    em = np.finfo(np.float64).eps
    assert jvp.fd_eps_paper(x) == pytest.approx(math.sqrt(em) * 5.0, rel=1e-15)
    assert jvp.fd_eps_paper(0.1 * x) == pytest.approx(math.sqrt(em), rel=1e-15)   # max(1, .)
    assert jvp.fd_eps_scaled(x, v) == pytest.approx(math.sqrt(em) * 6.0 / 2.0, rel=1e-15)
    e32 = np.finfo(np.float32).eps
    assert jvp.fd_eps_scaled(x, v, e32) == pytest.approx(math.sqrt(2.0 ** -23) * 3.0, rel=1e-15)
    with pytest.raises(ValueError):
        jvp.fd_eps_scaled(x, np.zeros(2))


def test_fd_is_linear_in_v_under_scaled_rule(rng):
    """With eps ~ 1/||v|| the perturbed state x + eps v does not depend on ||v||, so FD(c v) = c FD(v)."""
    p = pdes.AllenCahn2D(nx=8, ny=8)
    x = rng.uniform(-1, 1, 64)
    v = rng.standard_normal(64)
    F = lambda z: p.residual(z, p.rhs(x))
    e1 = jvp.fd_eps_scaled(x, v)
    e2 = jvp.fd_eps_scaled(x, 4.0 * v)
    assert np.allclose(jvp.jvp_fd(F, x, 4.0 * v, e2), 4.0 * jvp.jvp_fd(F, x, v, e1), rtol=1e-12, atol=1e-12)
