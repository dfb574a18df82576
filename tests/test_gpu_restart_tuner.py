"""The GMRES restart autotuner of jfnk_solve (opts.restart = 0) (GPU).

The first Newton system of a problem class is solved once per candidate restart length, each to the
requested Krylov tolerance; the fastest candidate is kept for the class on the context and its step is
used. The choice is made at equal tolerance, so the result is held to the same solution tolerances
against the oracle as a fixed restart length (1e-10 FP64 against a tightly solved reference, 1e-5 mixed),
and a second solve of the same class reuses the choice without timing the candidates again.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import newton as onw, pdes as opdes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CANDIDATES = (10, 20, 30, 40, 60)


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


def _solve(J, ctx, lp, prec, ortho, x0, steps, tol_n, tol_k):
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    o = J.jfnk_default_opts(prec)
    o.restart, o.tol_newton, o.tol_krylov, o.max_newton = 0, tol_n, tol_k, 30
    o.ortho = ortho
    x = torch.tensor(x0, device="cuda")
    rep = J.jfnk_report()
    s = J.jfnk_solve(ctx, o, None, x, steps, rep)
    torch.cuda.synchronize()
    return s, x.cpu().numpy(), rep


@pytest.mark.parametrize("prec,ortho", [("fp64", "cgs2"), ("mixed", "dcgs2")])
def test_tuned_restart_meets_the_solution_tolerance(J, ctx, prec, ortho):
    n = 128
    u0 = si.allen_cahn_ic(n, n, 2)
    p = opdes.AllenCahn2D(nx=n, ny=n, D=1e-3, dt=0.1, theta=0.5)
    lp = J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))
    code = J.JFNK_FP64 if prec == "fp64" else J.JFNK_MIXED_FP32
    oc = J.JFNK_DCGS2 if ortho == "dcgs2" else J.JFNK_CGS2
    tol_n, tol_k, tol_x = (1e-12, 1e-12, 1e-10) if prec == "fp64" else (1e-9, 1e-6, 1e-5)
    s, x, rep = _solve(J, ctx, lp, code, oc, u0, 1, tol_n, tol_k)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    assert rep.restart_used in CANDIDATES
    x_ref, reps = onw.time_steps(p, u0, 1, onw.Options(restart=40, tol_newton=1e-13, tol_krylov=1e-12))
    assert np.abs(x - x_ref).max() <= tol_x * np.abs(x_ref).max()
    assert np.linalg.norm(p.residual(x, p.rhs(u0))) <= max(tol_n, 1e-12) * reps[0].res0 * 1.0001
    # the same class again: the chosen length, no candidates timed (fewer Krylov steps than the first call)
    s2, x2, rep2 = _solve(J, ctx, lp, code, oc, u0, 1, tol_n, tol_k)
    assert s2 == J.JFNK_OK
    assert rep2.restart_used == rep.restart_used
    assert rep2.krylov_its < rep.krylov_its
    assert np.abs(x2 - x_ref).max() <= tol_x * np.abs(x_ref).max()


def test_batched_entry_points_need_a_restart_length(J, ctx):
    lp = J.make_problem("allen_cahn", 64, 64, 0.1, 0.5, (1e-3, 1.0))
    o = J.jfnk_default_opts(J.JFNK_FP64)
    o.restart = 0
    x = torch.tensor(si.allen_cahn_ic(64, 64, 0), device="cuda")
    s, _, _ = J.jfnk_solve_batch(ctx, [lp], o, None, [x], 1)
    assert s == J.JFNK_E_INVALID
    o.restart = -1
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    assert J.jfnk_solve(ctx, o, None, x, 1, None) == J.JFNK_E_INVALID
