"""Pins of the oracle's Krylov solvers against library routines (CPU only).

* GMRES without restart on an N <= 32 system reaches numpy.linalg.solve.
* After k Arnoldi steps GMRES returns the minimum-residual point of the
  Krylov space K_k of Eq. 10 (computed here by numpy.linalg.lstsq on an
  explicit power basis), which pins the Givens least squares.
* Restarted GMRES, BiCGSTAB and CG meet their relative tolerance on the true
  residual; CG on an SPD system and BiCGSTAB agree with numpy's solve.
* A circulant Allen-Cahn Jacobian (linearised at a constant state) is
  inverted exactly by FFT; GMRES with the complex-step JVP matches it.
* A forced BiCGSTAB breakdown (r_hat . A r0 = 0) is reported, not hidden.
"""
import numpy as np
import pytest

from oracle import jvp, krylov, pdes


def _nonsym(rng, n, shift=4.0):
    return rng.standard_normal((n, n)) / np.sqrt(n) + shift * np.eye(n)


def test_gmres_full_equals_dense_solve(rng):
    n = 32
    A = _nonsym(rng, n, 1.0)
    b = rng.standard_normal(n)
    r = krylov.gmres(lambda v: A @ v, b, m=n, tol=1e-14, max_cycles=1)
    assert r.converged
    assert np.allclose(r.x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_gmres_is_minimum_residual_over_krylov_space(rng, k):
    n = 24
    A = _nonsym(rng, n, 0.5)
    b = rng.standard_normal(n)
    r = krylov.gmres(lambda v: A @ v, b, m=k, tol=0.0, max_cycles=1)
    assert r.iterations == k
    # explicit basis of K_k = span{b, Ab, ..., A^{k-1} b}, orthonormalised by QR
    K = np.empty((n, k))
    K[:, 0] = b
    for i in range(1, k):
        K[:, i] = A @ K[:, i - 1]
    Q, _ = np.linalg.qr(K)
    c = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
    x_min = Q @ c
    assert np.allclose(r.x, x_min, rtol=1e-8, atol=1e-10)
    assert abs(r.resid_est - np.linalg.norm(b - A @ r.x)) <= 1e-9 * np.linalg.norm(b)


def test_givens_rotation():
    for f, g in [(3.0, 4.0), (-2.0, 0.5), (0.0, -1.0), (-1.0, 0.0), (0.0, 0.0)]:
        c, s = krylov.givens(f, g)
        assert c * c + s * s == pytest.approx(1.0)
        assert -s * f + c * g == pytest.approx(0.0, abs=1e-15)
        assert c * f + s * g == pytest.approx(np.hypot(f, g))


def test_restarted_gmres_meets_tolerance(rng):
    n = 200
    A = _nonsym(rng, n, 2.0)
    b = rng.standard_normal(n)
    r = krylov.gmres(lambda v: A @ v, b, m=10, tol=1e-10, max_cycles=200)
    assert r.converged
    assert np.linalg.norm(b - A @ r.x) <= 1.01e-10 * np.linalg.norm(b)
    assert r.matvecs == r.iterations + (r.iterations - 1) // 10   # one true-residual product per restart


def test_bicgstab_and_cg_against_solve(rng):
    n = 60
    A = _nonsym(rng, n, 3.0)
    b = rng.standard_normal(n)
    r = krylov.bicgstab(lambda v: A @ v, b, tol=1e-12, maxiter=500)
    assert r.converged and not r.breakdown
    assert np.allclose(r.x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-10)
    B = rng.standard_normal((n, n))
    S = B @ B.T / n + np.eye(n)
    r = krylov.cg(lambda v: S @ v, b, tol=1e-12, maxiter=500)
    assert r.converged
    assert np.allclose(r.x, np.linalg.solve(S, b), rtol=1e-9, atol=1e-10)


def test_bicgstab_breakdown_is_reported():
    A = np.array([[0.0, -1.0], [1.0, 0.0]])   # rotation by 90 degrees: b . A b = 0
    r = krylov.bicgstab(lambda v: A @ v, np.array([1.0, 0.0]), tol=1e-12, maxiter=10)
    assert r.breakdown and not r.converged


def test_zero_rhs_returns_zero():
    for solve in (lambda A, b: krylov.gmres(A, b, 5, 1e-8, 3), lambda A, b: krylov.bicgstab(A, b, 1e-8, 3),
                  lambda A, b: krylov.cg(A, b, 1e-8, 3)):
        r = solve(lambda v: 2.0 * v, np.zeros(7))
        assert r.converged and r.iterations == 0 and not r.x.any()


def test_gmres_on_circulant_allen_cahn_matches_fft():
    """Linearised at u = c the Allen-Cahn Jacobian is circulant: J^{-1} b by FFT is exact."""
    n, D, dt, th, c = 32, 1e-3, 0.1, 0.5, 0.4
    p = pdes.AllenCahn2D(nx=n, ny=n, D=D, dt=dt, theta=th)
    u = np.full(n * n, c)
    b = np.random.default_rng(7).standard_normal(n * n)
    F = lambda z: p.residual(z, p.rhs(u))
    r = krylov.gmres(lambda v: jvp.jvp_complex_step(F, u, v)[1], b, m=40, tol=1e-12, max_cycles=50)
    assert r.converged
    k = np.fft.fftfreq(n, d=1.0 / n)
    sym1 = (2 * np.cos(2 * np.pi * k / n) - 2) * n * n              # eigenvalues of the periodic 1D second difference
    lam = 1.0 - th * dt * (D * (sym1[None, :] + sym1[:, None]) + 1.0 - 3.0 * c * c)
    x_fft = np.real(np.fft.ifft2(np.fft.fft2(b.reshape(n, n)) / lam)).reshape(-1)
    assert np.allclose(r.x, x_fft, rtol=1e-9, atol=1e-10 * np.abs(x_fft).max())


# ---------------------------------------------------------------------------
# delayed CGS2 (the second Gram-Schmidt pass one Arnoldi step late)
# ---------------------------------------------------------------------------
def test_dcgs2_gmres_full_equals_dense_solve(rng):
    n = 32
    A = _nonsym(rng, n, 1.0)
    b = rng.standard_normal(n)
    r = krylov.gmres_dcgs2(lambda v: A @ v, b, m=n, tol=1e-14, max_cycles=1)
    assert r.converged
    assert np.allclose(r.x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_dcgs2_gmres_is_minimum_residual_over_krylov_space(rng, k):
    """After k completed columns the iterate is the minimum-residual point of K_k (lstsq on a power basis)."""
    n = 24
    A = _nonsym(rng, n, 0.5)
    b = rng.standard_normal(n)
    r = krylov.gmres_dcgs2(lambda v: A @ v, b, m=k, tol=0.0, max_cycles=1)
    assert r.iterations == k
    assert r.matvecs == k                       # the last column is completed without a product
    K = np.empty((n, k))
    K[:, 0] = b
    for i in range(1, k):
        K[:, i] = A @ K[:, i - 1]
    Q, _ = np.linalg.qr(K)
    c = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
    assert np.allclose(r.x, Q @ c, rtol=1e-8, atol=1e-10)
    assert abs(r.resid_est - np.linalg.norm(b - A @ r.x)) <= 1e-9 * np.linalg.norm(b)


@pytest.mark.parametrize("m", [3, 8, 20])
def test_dcgs2_iterates_equal_cgs2(rng, m):
    """Same Krylov spaces, so the same restarted iteration: counts equal, iterates equal to rounding;
    a cycle that converges before its last column costs one operator product more (the candidate after
    the last completed column)."""
    n = 60
    A = _nonsym(rng, n, 2.0)
    b = rng.standard_normal(n)
    r1 = krylov.gmres(lambda v: A @ v, b, m=m, tol=1e-10, max_cycles=100)
    r2 = krylov.gmres_dcgs2(lambda v: A @ v, b, m=m, tol=1e-10, max_cycles=100)
    assert r1.converged and r2.converged
    assert r2.iterations == r1.iterations
    last = r1.iterations - m * ((r1.iterations - 1) // m)     # columns of the converged cycle
    assert r2.matvecs == r1.matvecs + (1 if last < m else 0)
    assert np.abs(r2.x - r1.x).max() <= 1e-9 * np.abs(r1.x).max()
    assert np.linalg.norm(b - A @ r2.x) <= 1e-10 * np.linalg.norm(b) * 1.0001


def test_dcgs2_keeps_orthogonality_where_one_pass_loses_it():
    """A matrix with singular values spread over 1e-10..1: one classical Gram-Schmidt pass loses
    orthogonality here, the delayed second pass must not; GMRES(n) then still reaches the dense solve."""
    n = 40
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    W, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = U @ np.diag(np.logspace(0, -10, n)) @ W.T
    b = A @ rng.standard_normal(n)
    r = krylov.gmres_dcgs2(lambda v: A @ v, b, m=n, tol=1e-12, max_cycles=1)
    r_ref = krylov.gmres(lambda v: A @ v, b, m=n, tol=1e-12, max_cycles=1)
    assert np.linalg.norm(b - A @ r.x) <= 1e-10 * np.linalg.norm(b)
    assert abs(r.iterations - r_ref.iterations) <= 1


def test_dcgs2_newton_step_equals_cgs2():
    """A Crank-Nicolson Allen-Cahn step solved with either Arnoldi form: same Newton and Krylov counts,
    same state to rounding."""
    from oracle import newton
    import synthetic_inputs as si
    n = 24
    p = pdes.AllenCahn2D(nx=n, ny=n, D=1e-3, dt=0.1, theta=0.5)
    u0 = si.allen_cahn_ic(n, n, 1)
    o1 = newton.Options(restart=10, tol_newton=1e-10, tol_krylov=1e-10)
    o2 = newton.Options(restart=10, tol_newton=1e-10, tol_krylov=1e-10, ortho="dcgs2")
    x1, r1 = newton.time_steps(p, u0, 1, o1)
    x2, r2 = newton.time_steps(p, u0, 1, o2)
    assert [r.newton_its for r in r1] == [r.newton_its for r in r2]
    assert abs(sum(r.krylov_its for r in r1) - sum(r.krylov_its for r in r2)) <= 1
    assert np.abs(x1 - x2).max() <= 1e-12 * np.abs(x1).max()


# ---------------------------------------------------------------------------
# diagonal complex-shifted-Laplacian preconditioner of the Maxwell problem
# ---------------------------------------------------------------------------
def test_cslp_diagonal_is_the_shifted_operator_diagonal():
    """Undamped and at chi3 = 0 the preconditioner is the diagonal of the dense (complex-step) Jacobian at
    interior cells (the walls add the absorbing ghost, which the paper's form leaves out); damping shifts it
    by -i d k^2 eps."""
    import synthetic_inputs as si
    n = 8
    p = pdes.MaxwellTE2D(nx=n, ny=n, k=4.0, chi3=0.0, eps_r=si.maxwell_medium(n, n, 1),
                         f=si.maxwell_point_source(n, n))
    x = np.random.default_rng(2).standard_normal(2 * n * n)
    Jd = jvp.dense_jacobian(lambda z: p.residual(z, None), x)
    m0 = p.cslp_diag(x, 0.0)
    nc = n * n
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            c = j * n + i
            assert Jd[c, c] == pytest.approx(m0[c].real, rel=1e-12)
            assert Jd[nc + c, nc + c] == pytest.approx(m0[c].real, rel=1e-12)
            assert abs(Jd[c, nc + c]) <= 1e-12 * abs(m0[c].real)
    m5 = p.cslp_diag(x, 0.5)
    assert np.allclose(m5, m0 - 0.5j * p.k ** 2 * p.eps_r, rtol=1e-14, atol=0)
    v = np.random.default_rng(3).standard_normal(2 * nc)
    assert np.allclose(pdes.apply_cell_complex(1.0 / m5, pdes.apply_cell_complex(m5, v)), v, rtol=1e-12, atol=1e-14)


def test_right_preconditioning_solves_the_same_system():
    """Newton on the linear (chi3 = 0) problem with full GMRES, with and without the preconditioner: both reach
    the dense solve of J x = f in one step."""
    import synthetic_inputs as si
    from oracle import newton
    n = 6
    p = pdes.MaxwellTE2D(nx=n, ny=n, k=3.0, chi3=0.0, eps_r=si.maxwell_medium(n, n, 0),
                         f=si.maxwell_point_source(n, n))
    Jd = jvp.dense_jacobian(lambda z: p.residual(z, None), np.zeros(2 * n * n))
    x_ref = np.linalg.solve(Jd, -p.residual(np.zeros(2 * n * n), None))
    for pc in ("none", "cslp"):
        o = newton.Options(restart=2 * n * n, tol_newton=1e-10, tol_krylov=1e-13, max_cycles=1, precond=pc)
        x, rep, _ = newton.bvp_solve(p, o)
        assert np.abs(x - x_ref).max() <= 1e-9 * np.abs(x_ref).max(), pc
