"""Parity of the CUDA residual and JVP kernels with the CPU oracle (GPU).

Every case calls the library through its C ABI on seeded inputs and compares
element by element with the oracle:

* AD JVP, FP64: against the complex-step derivative (the exact derivative of
  the same residual), relative to max |Jv|, tolerance 1e-12 (the JVP
  accuracy the method targets); F(x) returned by the same sweep, 1e-12.
* AD JVP, FP32: inputs rounded to FP32 and the oracle evaluated in FP64 on
  those values (so that branch decisions coincide); tolerance 5e-5 of
  max |Jv| (about 400 FP32 ulps: some twenty roundings of stencil terms
  that, with dt/h^2 scaling, reach a few times max |Jv|).
* FD JVP: FP64 with the same step as the oracle, tolerance 1e-6 of max |Jv|
  (the quotient amplifies residual rounding by 1/eps). FP32 is not unique to
  rounding (the quotient amplifies FP32 noise by 1/eps ~ 1e3), so it is
  checked by a property: its error against the exact JVP is within 10x the
  error of the oracle's own FP32 quotient at the same step.

Grids span several 32 x 8 thread tiles with ragged tails in both directions.
"""
import math

import numpy as np
import pytest

import synthetic_inputs as si
from oracle import jvp as ojvp, pdes as opdes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def J():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13378_gb300 import build
    build.build()
    from paper_2605_13378_gb300 import jfnk
    return jfnk


@pytest.fixture
def ctx(J):
    c = J.jfnk_create(0)
    yield c
    J.jfnk_destroy(c)


def _case(name, nx, ny, seed=0):
    """(oracle problem, library problem, x, v, b) for a PDE on an nx x ny grid."""
    rng = np.random.default_rng(seed)
    from paper_2605_13378_gb300 import jfnk as J
    if name == "burgers":
        p = opdes.Burgers1D(N=nx, nu=1e-2, dt=1e-3, theta=1.0)
        x = si.burgers_ic(nx, seed)
        lp = J.make_problem("burgers1d", nx, 1, 1e-3, 1.0, (1e-2,))
        extra = None
    elif name == "allen_cahn":
        p = opdes.AllenCahn2D(nx=nx, ny=ny, D=1e-3, dt=0.1, theta=0.5)
        x = rng.uniform(-1.0, 1.0, nx * ny)
        lp = J.make_problem("allen_cahn", nx, ny, 0.1, 0.5, (1e-3, 1.0))
        extra = None
    elif name == "su_olson":
        p = opdes.SuOlson2D(nx=nx, ny=ny, dt=1e-2, theta=0.5)
        x = np.concatenate([rng.uniform(0.05, 1.0, nx * ny), rng.uniform(0.2, 1.0, nx * ny)])
        lp = J.make_problem("su_olson", nx, ny, 1e-2, 0.5, (1.0, 1.0, 1.0, 1e-6, 1.0))
        extra = None
    elif name == "rd_dirichlet":
        p = opdes.AllenCahn2D(nx=nx, ny=ny, D=1e-2, dt=0.05, theta=0.5, linear_coef=0.0, dirichlet=True)
        x = rng.uniform(-1.0, 1.0, nx * ny)
        lp = J.make_problem("allen_cahn", nx, ny, 0.05, 0.5, (1e-2, 0.0, 1.0))
        extra = None
    elif name == "burgers2d":
        p = opdes.Burgers2D(nx=nx, ny=ny, nu=0.02, dt=0.05, theta=0.5)
        x = rng.uniform(-1.0, 1.0, 2 * nx * ny)
        lp = J.make_problem("burgers2d", nx, ny, 0.05, 0.5, (0.02, 0.0, 0.0))
        extra = None
    else:
        eps = si.maxwell_medium(nx, ny, seed)
        f = si.maxwell_point_source(nx, ny)
        k = 9.0
        p = opdes.MaxwellTE2D(nx=nx, ny=ny, k=k, chi3=0.2, eps_r=eps, f=f)
        x = rng.standard_normal(2 * nx * ny)
        extra = (eps, f)
        lp = J.make_problem("maxwell", nx, ny, 0.0, 1.0, (k, 0.2), eps_r=eps, source=f)
    v = rng.standard_normal(x.size)
    b = None if p.bvp else p.rhs(x * 0.97)
    return p, lp, x, v, b, extra


# odd row lengths take the gather launch form, multiples of 4 the march form (16-byte row vectors)
CASES = [("burgers", 1000, 1), ("allen_cahn", 70, 45), ("su_olson", 67, 41), ("maxwell", 66, 37),
         ("burgers", 996, 1), ("allen_cahn", 68, 44), ("su_olson", 72, 40), ("maxwell", 64, 37),
         ("su_olson", 40, 40), ("maxwell", 96, 9), ("burgers2d", 70, 45), ("burgers2d", 64, 37),
         ("rd_dirichlet", 70, 45), ("rd_dirichlet", 64, 37)]


def _dev(a, dtype=torch.float64):
    return None if a is None else torch.tensor(a, dtype=dtype, device="cuda")


@pytest.mark.parametrize("name,nx,ny", CASES)
def test_ad_jvp_fp64_matches_complex_step(J, ctx, name, nx, ny):
    p, lp, x, v, b, _ = _case(name, nx, ny)
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    xt, vt, bt = _dev(x), _dev(v), _dev(b)
    F = torch.empty_like(xt)
    Jv = torch.empty_like(xt)
    J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_AD, J.JFNK_FP64, xt, vt, bt, F, Jv, 0.0), "jvp")
    torch.cuda.synchronize()
    F_ref, Jv_ref = ojvp.jvp_complex_step(lambda z: p.residual(z, b), x, v)
    assert np.abs(Jv.cpu().numpy() - Jv_ref).max() <= 1e-12 * np.abs(Jv_ref).max()
    assert np.abs(F.cpu().numpy() - F_ref).max() <= 1e-12 * np.abs(F_ref).max()
    # the plain residual kernel agrees with the F of the dual sweep
    F2 = torch.empty_like(xt)
    J.check(ctx, J.jfnk_residual(ctx, J.JFNK_FP64, xt, bt, F2), "residual")
    torch.cuda.synchronize()
    assert np.abs(F2.cpu().numpy() - F_ref).max() <= 1e-12 * np.abs(F_ref).max()


@pytest.mark.parametrize("name,nx,ny", CASES)
def test_ad_jvp_fp32_matches_oracle_on_rounded_inputs(J, ctx, name, nx, ny):
    p, lp, x, v, b, _ = _case(name, nx, ny)
    x = x.astype(np.float32).astype(np.float64)
    v = v.astype(np.float32).astype(np.float64)
    b = None if b is None else b.astype(np.float32).astype(np.float64)
    if name == "maxwell":   # the kernel reads eps_r and the source in FP32 as well
        p.eps_r = p.eps_r.astype(np.float32).astype(np.float64)
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    xt, vt, bt = _dev(x, torch.float32), _dev(v, torch.float32), _dev(b, torch.float32)
    F = torch.empty_like(xt)
    Jv = torch.empty_like(xt)
    J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_AD, J.JFNK_FP32, xt, vt, bt, F, Jv, 0.0), "jvp")
    torch.cuda.synchronize()
    F_ref, Jv_ref = ojvp.jvp_complex_step(lambda z: p.residual(z, b), x, v)
    assert np.abs(Jv.cpu().numpy() - Jv_ref).max() <= 5e-5 * np.abs(Jv_ref).max()


@pytest.mark.parametrize("name,nx,ny", CASES)
def test_fd_jvp_fp64_matches_oracle_quotient(J, ctx, name, nx, ny):
    p, lp, x, v, b, _ = _case(name, nx, ny)
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    eps = ojvp.fd_eps_scaled(x, v)
    F = lambda z: p.residual(z, b)
    ref = ojvp.jvp_fd(F, x, v, eps)
    Jv_exact = ojvp.jvp_complex_step(F, x, v)[1]
    xt, vt, bt = _dev(x), _dev(v), _dev(b)
    out = torch.empty_like(xt)
    # library-side rule: the same step sqrt(eps)(1 + ||x||)/||v|| from device norms
    J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_FD, J.JFNK_FP64, xt, vt, bt, None, out, 0.0), "jvp")
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-6 * np.abs(Jv_exact).max()
    # explicit step
    J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_FD, J.JFNK_FP64, xt, vt, bt, None, out, 1e-5), "jvp")
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ojvp.jvp_fd(F, x, v, 1e-5)).max() <= 1e-6 * np.abs(Jv_exact).max()


@pytest.mark.parametrize("name,nx,ny", CASES)
def test_fd_jvp_fp32_within_fd_error_bound(J, ctx, name, nx, ny):
    p, lp, x, v, b, _ = _case(name, nx, ny)
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    Jv_exact = ojvp.jvp_complex_step(lambda z: p.residual(z, b), x, v)[1]
    x32, v32 = x.astype(np.float32), v.astype(np.float32)
    b32 = None if b is None else b.astype(np.float32)
    eps = ojvp.fd_eps_scaled(x32.astype(np.float64), v32.astype(np.float64), np.finfo(np.float32).eps)
    if name == "maxwell":
        p.eps_r = p.eps_r.astype(np.float32)
        p.f = p.f.astype(np.float32)
    ref32 = ojvp.jvp_fd(lambda z: p.residual(z, b32), x32, v32, eps).astype(np.float64)
    err_ref = np.abs(ref32 - Jv_exact).max()
    xt, vt, bt = _dev(x, torch.float32), _dev(v, torch.float32), _dev(b, torch.float32)
    out = torch.empty_like(xt)
    J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_FD, J.JFNK_FP32, xt, vt, bt, None, out, 0.0), "jvp")
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all()
    err = np.abs(got - Jv_exact).max()
    assert err <= 10.0 * err_ref + 1e-5 * np.abs(Jv_exact).max(), (err, err_ref)


def test_ad_jvp_full_size_allen_cahn_2048(J, ctx):
    """The benchmark grid (2048^2, the launch configuration the benchmark times): full comparison."""
    n = 2048
    p = opdes.AllenCahn2D(nx=n, ny=n, D=1e-3, dt=0.1, theta=0.5)
    x = si.allen_cahn_ic(n, n, 0)
    v = np.random.default_rng(3).standard_normal(n * n)
    b = p.rhs(x)
    J.check(ctx, J.jfnk_set_problem(ctx, J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))), "set")
    xt, vt, bt = _dev(x), _dev(v), _dev(b)
    F = torch.empty_like(xt)
    Jv = torch.empty_like(xt)
    J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_AD, J.JFNK_FP64, xt, vt, bt, F, Jv, 0.0), "jvp")
    torch.cuda.synchronize()
    F_ref, Jv_ref = ojvp.jvp_complex_step(lambda z: p.residual(z, b), x, v)
    assert np.abs(Jv.cpu().numpy() - Jv_ref).max() <= 1e-12 * np.abs(Jv_ref).max()
    assert np.abs(F.cpu().numpy() - F_ref).max() <= 1e-12 * np.abs(F_ref).max()


def test_zero_direction_and_minimal_grid(J, ctx):
    n = 3
    p = opdes.AllenCahn2D(nx=n, ny=n, D=0.3, dt=0.1)
    x = np.linspace(-1, 1, 9)
    J.check(ctx, J.jfnk_set_problem(ctx, J.make_problem("allen_cahn", n, n, 0.1, 0.5, (0.3, 1.0))), "set")
    xt = _dev(x)
    Jv = torch.full_like(xt, 7.0)
    J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_AD, J.JFNK_FP64, xt, torch.zeros_like(xt), None, None, Jv, 0.0), "jvp")
    torch.cuda.synchronize()
    assert (Jv.cpu().numpy() == 0.0).all()
    v = np.arange(9.0)
    J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_AD, J.JFNK_FP64, xt, _dev(v), None, None, Jv, 0.0), "jvp")
    torch.cuda.synchronize()
    ref = ojvp.jvp_complex_step(lambda z: p.residual(z, np.zeros(9)), x, v)[1]
    assert np.abs(Jv.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_invalid_problems_are_rejected(J, ctx):
    assert J.jfnk_set_problem(ctx, J.make_problem("burgers1d", 2, 1, 1e-3, 1.0, (0.01,))) == J.JFNK_E_INVALID
    assert J.jfnk_set_problem(ctx, J.make_problem("allen_cahn", 16, 2, 0.1, 0.5, (1e-3, 1.0))) == J.JFNK_E_INVALID
    assert J.jfnk_set_problem(ctx, J.make_problem("allen_cahn", 16, 16, -0.1, 0.5, (1e-3, 1.0))) == J.JFNK_E_INVALID
    assert "dt" in J.jfnk_last_error(ctx)
    assert J.jfnk_set_problem(ctx, J.make_problem("maxwell", 16, 16, 0.0, 1.0, (0.0, 0.1))) == J.JFNK_E_INVALID
    assert J.jfnk_set_problem(ctx, J.make_problem("burgers2d", 16, 16, 0.1, 0.5, (-0.1, 0.0, 0.0))) == J.JFNK_E_INVALID
    assert "nu" in J.jfnk_last_error(ctx)
    assert J.jfnk_set_problem(ctx, J.make_problem("burgers2d", 16, 16, 0.0, 0.5, (0.1, 0.0, 0.0))) == J.JFNK_E_INVALID
    # with a Courant number the step is adaptive and dt is not needed
    assert J.jfnk_set_problem(ctx, J.make_problem("burgers2d", 16, 16, 0.0, 0.5, (0.1, 0.0, 1.0))) == J.JFNK_OK


# The plain Krylov product (no F output, no addend) on 2D grids with rows of at least 1024 FP32 or 512
# FP64 cells and at least 64 rows runs the staged form: rows of x and v copied into shared memory by bulk
# copies, one CTA per (strip, band) unit. These cases give ragged last strips (1028 = 1024 + 4 columns;
# 3 strips of 512 + 4 in FP64), ragged last bands, both wall policies (wrap: Allen-Cahn, 2D Burgers;
# clamp: radiation, Maxwell, Dirichlet walls) and, at 5120 x 368 (5 strips x 92 bands of 4 rows, 460 units on 456
# CTAs at three per SM), CTAs that take a second unit.
STAGED = [("allen_cahn", 1028, 70), ("su_olson", 1024, 66), ("maxwell", 1028, 64), ("burgers2d", 1024, 65),
          ("rd_dirichlet", 1028, 67), ("allen_cahn", 5120, 368)]


@pytest.mark.parametrize("name,nx,ny", STAGED)
def test_staged_ad_jvp_fp64_matches_complex_step(J, ctx, name, nx, ny):
    p, lp, x, v, b, _ = _case(name, nx, ny)
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    xt, vt, bt = _dev(x), _dev(v), _dev(b)
    Jv = torch.full_like(xt, float("nan"))
    J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_AD, J.JFNK_FP64, xt, vt, bt, None, Jv, 0.0), "jvp")
    torch.cuda.synchronize()
    _, Jv_ref = ojvp.jvp_complex_step(lambda z: p.residual(z, b), x, v)
    assert np.abs(Jv.cpu().numpy() - Jv_ref).max() <= 1e-12 * np.abs(Jv_ref).max()


@pytest.mark.parametrize("name,nx,ny", STAGED)
def test_staged_ad_jvp_fp32_matches_oracle_on_rounded_inputs(J, ctx, name, nx, ny):
    p, lp, x, v, b, _ = _case(name, nx, ny)
    x = x.astype(np.float32).astype(np.float64)
    v = v.astype(np.float32).astype(np.float64)
    b = None if b is None else b.astype(np.float32).astype(np.float64)
    if name == "maxwell":
        p.eps_r = p.eps_r.astype(np.float32).astype(np.float64)
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    xt, vt, bt = _dev(x, torch.float32), _dev(v, torch.float32), _dev(b, torch.float32)
    Jv = torch.full_like(xt, float("nan"))
    J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_AD, J.JFNK_FP32, xt, vt, bt, None, Jv, 0.0), "jvp")
    torch.cuda.synchronize()
    _, Jv_ref = ojvp.jvp_complex_step(lambda z: p.residual(z, b), x, v)
    assert np.abs(Jv.cpu().numpy() - Jv_ref).max() <= 5e-5 * np.abs(Jv_ref).max()


@pytest.mark.parametrize("name,nx,ny", STAGED[:3])
def test_staged_fd_jvp_fp64_matches_oracle_quotient(J, ctx, name, nx, ny):
    p, lp, x, v, b, _ = _case(name, nx, ny)
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    F = lambda z: p.residual(z, b)
    ref = ojvp.jvp_fd(F, x, v, ojvp.fd_eps_scaled(x, v))
    scale = np.abs(ojvp.jvp_complex_step(F, x, v)[1]).max()
    xt, vt, bt = _dev(x), _dev(v), _dev(b)
    out = torch.full_like(xt, float("nan"))
    J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_FD, J.JFNK_FP64, xt, vt, bt, None, out, 0.0), "jvp")
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-6 * scale


def test_staged_ad_jvp_fp32_full_size_allen_cahn_2048(J, ctx):
    """The product the benchmark's Krylov loop applies: FP32 AD, plain output, 2048^2 grid."""
    n = 2048
    p = opdes.AllenCahn2D(nx=n, ny=n, D=1e-3, dt=0.1, theta=0.5)
    x = si.allen_cahn_ic(n, n, 0).astype(np.float32).astype(np.float64)
    v = np.random.default_rng(4).standard_normal(n * n).astype(np.float32).astype(np.float64)
    b = p.rhs(x).astype(np.float32).astype(np.float64)
    J.check(ctx, J.jfnk_set_problem(ctx, J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))), "set")
    xt, vt, bt = _dev(x, torch.float32), _dev(v, torch.float32), _dev(b, torch.float32)
    Jv = torch.full_like(xt, float("nan"))
    for _ in range(2):   # the second launch reuses the ring's barriers from a fresh launch
        J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_AD, J.JFNK_FP32, xt, vt, bt, None, Jv, 0.0), "jvp")
    torch.cuda.synchronize()
    _, Jv_ref = ojvp.jvp_complex_step(lambda z: p.residual(z, b), x, v)
    assert np.abs(Jv.cpu().numpy() - Jv_ref).max() <= 5e-5 * np.abs(Jv_ref).max()
