"""Newton's backtracking line search, decided on the device, against the oracle (GPU).

The implicit Allen-Cahn step u - u^n - (dt/2)(D lap u + u - u^3 + G(u^n)) = 0
with dt = 1.96 and D = 1e-5 sits near the edge where the cell map
u (1 - dt/2) + (dt/2) u^3 stops being monotone: at u^n ~ U[-0.1, 0.1] its
Jacobian is close to (1 - dt/2) I = 0.02 I, so Newton's full step overshoots
by orders of magnitude and the line search of Sec. 2 (Armijo on ||F||,
alpha halved) has to backtrack before quadratic convergence sets in. Every
Armijo decision of this case is far from its threshold (the accepted trials
have ||F(x + alpha d)|| / ((1 - c1 alpha)||F(x)||) <= 0.54 and the rejected
ones >= 1.9 in the oracle), so the GPU must take exactly the oracle's steps:
the same accepted alpha at every Newton iteration, the same backtrack and
failure counts, the same Newton count, and the solution within the FP64
solution tolerance 1e-10 (1e-5 for the mixed form). With alpha_min = 1/2 the
first iteration finds no passing trial and takes alpha_min, counted as a
line-search failure.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import newton as onw, pdes as opdes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D, DT, SEED = 1e-5, 1.96, 3


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


def _solve(J, ctx, nx, ny, prec, lin, min_alpha, tol_k):
    lp = J.make_problem("allen_cahn", nx, ny, DT, 0.5, (D, 1.0))
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    o = J.jfnk_default_opts(prec)
    o.lin = J.JFNK_AD if lin == "ad" else J.JFNK_FD
    o.restart, o.tol_newton, o.tol_krylov, o.max_newton = 40, 1e-10, tol_k, 40
    o.ls_min_alpha = min_alpha
    x = torch.tensor(si.allen_cahn_ic(nx, ny, SEED), device="cuda")
    rep = J.jfnk_report()
    J.jfnk_reset_stats(ctx)
    J.jfnk_set_timing(ctx, True)
    s = J.jfnk_solve(ctx, o, None, x, 1, rep)
    J.jfnk_set_timing(ctx, False)
    torch.cuda.synchronize()
    return s, x.cpu().numpy(), rep, J.jfnk_kernel_stats(ctx)


def _oracle(nx, ny, lin, min_alpha):
    p = opdes.AllenCahn2D(nx=nx, ny=ny, D=D, dt=DT, theta=0.5)
    u0 = si.allen_cahn_ic(nx, ny, SEED)
    o = onw.Options(lin=lin, restart=40, tol_newton=1e-10, tol_krylov=1e-12, max_newton=40, ls_min_alpha=min_alpha)
    x, reps = onw.time_steps(p, u0, 1, o)
    return p, u0, x, reps[0]


@pytest.mark.parametrize("nx,ny", [(24, 24), (25, 23)])   # march form; gather form (odd rows)
@pytest.mark.parametrize("lin", ["ad", "fd"])
@pytest.mark.parametrize("min_alpha", [2.0 ** -10, 0.5])
def test_backtracking_matches_the_oracle_fp64(J, ctx, nx, ny, lin, min_alpha):
    s, x, rep, st = _solve(J, ctx, nx, ny, J.JFNK_FP64, lin, min_alpha, 1e-12)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    p, u0, x_ref, r = _oracle(nx, ny, lin, min_alpha)
    assert r.ls_backtracks > 0
    assert rep.ls_backtracks == r.ls_backtracks, (rep.ls_backtracks, r.ls_backtracks)
    assert rep.ls_failures == r.ls_failures, (rep.ls_failures, r.ls_failures)
    assert rep.newton_its == r.newton_its, (rep.newton_its, r.newton_its)
    assert list(rep.ls_alpha[:rep.newton_its]) == r.alphas, (list(rep.ls_alpha[:rep.newton_its]), r.alphas)
    assert all(a == 0.0 for a in rep.ls_alpha[rep.newton_its:])
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-10
    assert np.linalg.norm(p.residual(x, p.rhs(u0))) <= 1e-10 * r.res0
    # AD: Krylov counts within 2 per Newton step (reduction order). FD: the FP64 quotient carries ~1e-8
    # relative rounding noise (eps_mach / step), so GMRES driven to 1e-12 iterates in that noise and its
    # count is not unique: within 10%
    if lin == "ad":
        assert abs(rep.krylov_its - r.krylov_its) <= 2 * r.newton_its
    else:
        assert abs(rep.krylov_its - r.krylov_its) <= 0.1 * r.krylov_its
    # only the trials up to the accepted one did work: one residual of the start
    # plus one per trial, although every trial down to alpha_min was queued
    assert st["residual"]["launches"] == 1 + rep.newton_its + rep.ls_backtracks


def test_backtracking_mixed_precision(J, ctx):
    """FP32 JVP and basis, FP64 residual and merit: the line search takes the oracle's
    first steps and the solution meets the FP32 solution tolerance."""
    s, x, rep, _ = _solve(J, ctx, 24, 24, J.JFNK_MIXED_FP32, "ad", 2.0 ** -10, 1e-6)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    p, u0, x_ref, r = _oracle(24, 24, "ad", 2.0 ** -10)
    assert list(rep.ls_alpha[:2]) == r.alphas[:2] == [0.125, 0.5]
    assert rep.ls_backtracks == r.ls_backtracks
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-5
    assert np.linalg.norm(p.residual(x, p.rhs(u0))) <= 1e-10 * r.res0


def test_full_steps_leave_no_backtrack(J, ctx):
    """The benchmark-like step (dt = 0.1) accepts alpha = 1 at every Newton iteration."""
    lp = J.make_problem("allen_cahn", 32, 32, 0.1, 0.5, (1e-3, 1.0))
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    o = J.jfnk_default_opts(J.JFNK_FP64)
    o.restart, o.tol_newton, o.tol_krylov = 40, 1e-10, 1e-10
    x = torch.tensor(si.allen_cahn_ic(32, 32, 0), device="cuda")
    rep = J.jfnk_report()
    assert J.jfnk_solve(ctx, o, None, x, 1, rep) == J.JFNK_OK
    assert rep.ls_backtracks == 0 and rep.ls_failures == 0
    assert list(rep.ls_alpha[:rep.newton_its]) == [1.0] * rep.newton_its
