"""The paper's 2D viscous Burgers problem through jfnk_solve against the oracle (GPU).

App. A, Burgers' Equation: central advection, 5-point diffusion,
Crank-Nicolson, the adaptive CFL step and the TGV, DSL and 4VC initial
velocities on the periodic square [0, 2 pi)^2. Each case runs through the C
ABI on the same seeded input as the oracle (oracle.newton.time_steps with
oracle.pdes.Burgers2D). Parity bar as for the other PDEs: solution to 1e-10
relative in FP64 (1e-5 in reduced precision), equal Newton counts in FP64,
Krylov counts within 2 per Newton step; the adaptive time step the library
reports equals the oracle's CFL step to 1e-13 relative (both evaluate the
same rule in FP64 from maxima of states that agree to 1e-10). Edge cases: a
ragged grid, BiCGSTAB, delayed CGS2, the undefined rule (nu = 0 at rest) and
a non-finite state.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import newton as onw, pdes as opdes

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


def _opts(J, prec, lin="ad", krylov="gmres", restart=30, tol_n=1e-10, tol_k=1e-10, max_newton=15,
          max_krylov=100, ortho=None):
    o = J.jfnk_default_opts(prec)
    o.lin = J.JFNK_AD if lin == "ad" else J.JFNK_FD
    o.krylov = {"gmres": J.JFNK_GMRES, "bicgstab": J.JFNK_BICGSTAB}[krylov]
    o.restart, o.tol_newton, o.tol_krylov = restart, tol_n, tol_k
    o.max_newton, o.max_krylov = max_newton, max_krylov
    o.ortho = J.JFNK_CGS2 if ortho is None else ortho
    return o


def _oopts(lin="ad", krylov="gmres", restart=30, tol_n=1e-10, tol_k=1e-10, max_newton=15, max_krylov=100):
    return onw.Options(lin=lin, krylov=krylov, restart=restart, tol_newton=tol_n, tol_krylov=tol_k,
                       max_newton=max_newton, max_cycles=max_krylov)


def _run(J, ctx, lp, opts, x0, steps):
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    x = torch.tensor(x0, device="cuda")
    rep = J.jfnk_report()
    s = J.jfnk_solve(ctx, opts, None, x, steps, rep)
    torch.cuda.synchronize()
    return s, x.cpu().numpy(), rep


def _compare(x, x_ref, rep, reps, tol_x, exact=True):
    err = np.abs(x - x_ref).max() / np.abs(x_ref).max()
    assert err <= tol_x, err
    if exact:
        nn = sum(r.newton_its for r in reps)
        assert rep.newton_its == nn, (rep.newton_its, nn)
        kk = sum(r.krylov_its for r in reps)
        assert abs(rep.krylov_its - kk) <= 2 * max(nn, 1), (rep.krylov_its, kk)


def _lp(J, n, ny, nu, C, dt=0.0):
    return J.make_problem("burgers2d", n, ny, dt, 0.5, (nu, 0.0, C))


@pytest.mark.parametrize("kind", si.BURGERS2D_KINDS)
@pytest.mark.parametrize("lin", ["ad", "fd"])
def test_adaptive_cfl_steps_fp64(J, ctx, kind, lin):
    n, nu, steps = 48, 0.05, 3
    x0 = si.burgers2d_ic(n, n, kind)
    p = opdes.Burgers2D(nx=n, ny=n, nu=nu, courant=1.0)
    s, x, rep = _run(J, ctx, _lp(J, n, n, nu, 1.0), _opts(J, J.JFNK_FP64, lin), x0, steps)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    x_ref, reps = onw.time_steps(p, x0, steps, _oopts(lin))
    _compare(x, x_ref, rep, reps, 1e-10)
    assert rep.steps_done == steps and rep.steps_failed == 0
    assert rep.dt_last == pytest.approx(p.dt, rel=1e-13)


def test_fixed_step_ragged_grid_and_dcgs2(J, ctx):
    nx, ny, nu, dt = 37, 29, 0.02, 0.04          # 2 * 37 * 29 unknowns: not a multiple of 8
    x0 = si.burgers2d_ic(nx, ny, "tgv")
    p = opdes.Burgers2D(nx=nx, ny=ny, nu=nu, dt=dt)
    s, x, rep = _run(J, ctx, _lp(J, nx, ny, nu, 0.0, dt), _opts(J, J.JFNK_FP64), x0, 2)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    x_ref, reps = onw.time_steps(p, x0, 2, _oopts())
    _compare(x, x_ref, rep, reps, 1e-10)
    assert rep.dt_last == dt
    # delayed CGS2 on a grid whose unknowns are a multiple of 8, against the CGS2 solve
    n = 40
    x0 = si.burgers2d_ic(n, n, "dsl")
    lp = _lp(J, n, n, nu, 1.0)
    s1, x1, r1 = _run(J, ctx, lp, _opts(J, J.JFNK_FP64), x0, 2)
    s2, x2, r2 = _run(J, ctx, lp, _opts(J, J.JFNK_FP64, ortho=J.JFNK_DCGS2), x0, 2)
    assert s1 == s2 == J.JFNK_OK
    assert np.abs(x1 - x2).max() <= 1e-10 * np.abs(x1).max()
    assert r1.newton_its == r2.newton_its


def test_bicgstab_fp64(J, ctx):
    n, nu = 40, 0.01
    x0 = si.burgers2d_ic(n, n, "4vc")
    p = opdes.Burgers2D(nx=n, ny=n, nu=nu, courant=1.0)
    s, x, rep = _run(J, ctx, _lp(J, n, n, nu, 1.0), _opts(J, J.JFNK_FP64, krylov="bicgstab", max_krylov=400),
                     x0, 2)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    x_ref, reps = onw.time_steps(p, x0, 2, _oopts(krylov="bicgstab", max_krylov=400))
    _compare(x, x_ref, rep, reps, 1e-9, exact=False)
    assert rep.newton_its == sum(r.newton_its for r in reps)


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_reduced_precision(J, ctx, prec):
    n, nu = 64, 0.01
    x0 = si.burgers2d_ic(n, n, "tgv")
    p = opdes.Burgers2D(nx=n, ny=n, nu=nu, courant=1.0)
    code = J.JFNK_MIXED_FP32 if prec == "mixed" else J.JFNK_FP32
    tol_n = 1e-9 if prec == "mixed" else 1e-5
    o = _opts(J, code, "ad", restart=30, tol_n=tol_n, tol_k=1e-6, max_newton=30)
    s, x, rep = _run(J, ctx, _lp(J, n, n, nu, 1.0), o, x0, 2)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    x_ref, reps = onw.time_steps(p, x0, 2, _oopts("ad", restart=30, tol_n=1e-12, tol_k=1e-12))
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-5
    assert rep.dt_last == pytest.approx(p.dt, rel=1e-5)


def test_paper_gpu_grid_512_tgv(J, ctx):
    """The paper's larger GPU grid (512 x 512, C = 1): two steps against the oracle at every node."""
    n, nu = 512, 0.01
    x0 = si.burgers2d_ic(n, n, "tgv")
    p = opdes.Burgers2D(nx=n, ny=n, nu=nu, courant=1.0)
    o = _opts(J, J.JFNK_FP64, "ad", restart=30, tol_n=1e-8, tol_k=1e-8)
    s, x, rep = _run(J, ctx, _lp(J, n, n, nu, 1.0), o, x0, 2)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    x_ref, reps = onw.time_steps(p, x0, 2, _oopts("ad", restart=30, tol_n=1e-8, tol_k=1e-8))
    _compare(x, x_ref, rep, reps, 1e-8)
    assert rep.dt_last == pytest.approx(p.dt, rel=1e-12)


def test_undefined_rule_and_nonfinite_state(J, ctx):
    n = 16
    # nu = 0 and the fluid at rest: no term of the CFL rule is defined
    s, _, _ = _run(J, ctx, _lp(J, n, n, 0.0, 1.0), _opts(J, J.JFNK_FP64), np.zeros(2 * n * n), 1)
    assert s == J.JFNK_E_INVALID and "CFL" in J.jfnk_last_error(ctx)
    # nu = 0 with motion is fine: the advective terms define the step
    x0 = si.burgers2d_ic(n, n, "tgv")
    s, _, rep = _run(J, ctx, _lp(J, n, n, 0.0, 0.5), _opts(J, J.JFNK_FP64), x0, 1)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    assert rep.dt_last == pytest.approx(0.5 * 2 * np.pi / n, rel=1e-14)
    bad = x0.copy()
    bad[5] = np.nan
    s, _, rep = _run(J, ctx, _lp(J, n, n, 0.05, 1.0), _opts(J, J.JFNK_FP64), bad, 2)
    assert s == J.JFNK_E_NONFINITE
    assert rep.steps_failed == 1 and rep.steps_done == 0 and np.isnan(rep.dt_last)


def test_jvp_and_residual_refuse_an_adaptive_step(J, ctx):
    """With the CFL rule (C > 0) the time step exists only inside jfnk_solve: the standalone JVP and
    residual entry points refuse such a problem instead of using dt = 0; with C = 0 and a step they run."""
    n = 16
    x = torch.tensor(si.burgers2d_ic(n, n, "tgv"), device="cuda")
    out = torch.zeros_like(x)
    J.check(ctx, J.jfnk_set_problem(ctx, _lp(J, n, n, 0.05, 1.0)), "set_problem")
    for lin in (J.JFNK_AD, J.JFNK_FD):
        assert J.jfnk_jvp(ctx, lin, J.JFNK_FP64, x, x, None, None, out, 0.0) == J.JFNK_E_INVALID
        assert "adaptive" in J.jfnk_last_error(ctx)
    assert J.jfnk_residual(ctx, J.JFNK_FP64, x, None, out) == J.JFNK_E_INVALID
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
    J.check(ctx, J.jfnk_set_problem(ctx, J.make_problem("burgers2d", n, n, 1e-3, 0.5, (0.05, 0.0, 0.0))), "set")
    assert J.jfnk_jvp(ctx, J.JFNK_AD, J.JFNK_FP64, x, x, None, None, out, 0.0) == J.JFNK_OK
    torch.cuda.synchronize()
    p = opdes.Burgers2D(nx=n, ny=n, nu=0.05, dt=1e-3)
    from oracle import jvp as ojvp
    xh = x.cpu().numpy()
    _, Jv = ojvp.jvp_complex_step(lambda z: p.residual(z, np.zeros_like(z)), xh, xh)
    assert np.abs(out.cpu().numpy() - Jv).max() <= 1e-12 * np.abs(Jv).max()
