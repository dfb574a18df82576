"""Batched solves with delayed CGS2 Arnoldi (jfnk_solve_batch, opts.ortho = JFNK_DCGS2) (GPU).

The batch engine runs the delayed-CGS2 form of GMRES (Sec. 3: the second
Gram-Schmidt pass of each Arnoldi vector one step late) as two phases per step,
the dots q_i . u_j, q_i . w and the update forming q_j and u_{j+1}, with the
coefficient step on the CTA that finishes the dots. Each problem of a mixed
batch is held to the single-solve bars against oracle.krylov.gmres_dcgs2 on the
same seeded input (solution 1e-10 in FP64, 1e-5 in reduced precision; Newton
counts equal and Krylov counts within 2 per Newton step in FP64), and a
problem's result is bitwise the same alone and in the mix at two forced tile
sizes. Short restart lengths run the last dots pass of a cycle (no w) often.
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


def _opts(J, prec, lin="ad", restart=30, tol_n=1e-10, tol_k=1e-10, max_newton=15, max_krylov=100):
    o = J.jfnk_default_opts(prec)
    o.lin = J.JFNK_AD if lin == "ad" else J.JFNK_FD
    o.restart, o.tol_newton, o.tol_krylov = restart, tol_n, tol_k
    o.max_newton, o.max_krylov = max_newton, max_krylov
    o.ortho = J.JFNK_DCGS2
    return o


def _oopts(lin="ad", restart=30, tol_n=1e-10, tol_k=1e-10, max_newton=15, max_krylov=100):
    return onw.Options(lin=lin, krylov="gmres", restart=restart, tol_newton=tol_n, tol_krylov=tol_k,
                       max_newton=max_newton, max_cycles=max_krylov, ortho="dcgs2")


def _cases(J):
    """(name, problem, opts, x0, steps, oracle() -> (x_ref, [reports]), tol_x, exact_counts)."""
    c = []
    N = 1024
    u0 = si.burgers_ic(N, 1)
    pb = opdes.Burgers1D(N=N, nu=1e-2, dt=1e-3)
    c.append(("burgers_ad", J.make_problem("burgers1d", N, 1, 1e-3, 1.0, (1e-2,)), _opts(J, J.JFNK_FP64), u0, 1,
              lambda: onw.time_steps(pb, u0, 1, _oopts()), 1e-10, True))
    n = 72
    a0 = si.allen_cahn_ic(n, n, 4)
    pa = opdes.AllenCahn2D(nx=n, ny=n, D=1e-3, dt=0.1, theta=0.5)
    c.append(("allen_cahn_fd", J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0)),
              _opts(J, J.JFNK_FP64, "fd", 40), a0, 2,
              lambda: onw.time_steps(pa, a0, 2, _oopts("fd", 40)), 1e-10, True))
    # restart 5: the cycle's last dots pass (no w) and the restart JVP every five steps
    c.append(("allen_cahn_m5", J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0)),
              _opts(J, J.JFNK_FP64, "ad", 5), a0, 1,
              lambda: onw.time_steps(pa, a0, 1, _oopts("ad", 5)), 1e-10, True))
    m0 = si.allen_cahn_ic(n, n, 6)
    for prec, lin in (("mixed", "ad"), ("mixed", "fd"), ("fp32", "ad")):
        code = J.JFNK_MIXED_FP32 if prec == "mixed" else J.JFNK_FP32
        tol_n = 1e-4 if prec == "fp32" else 1e-9
        c.append((f"allen_cahn_{prec}_{lin}", J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0)),
                  _opts(J, code, lin, 40, tol_n, 1e-5, max_newton=30), m0, 1,
                  lambda: onw.time_steps(pa, m0, 1, _oopts("ad", 40, 1e-12, 1e-12)), 1e-5, False))
    nm, k, chi = 16, 3.0, 0.1
    eps, f = si.maxwell_medium(nm, nm, 1), si.maxwell_point_source(nm, nm)
    pm = opdes.MaxwellTE2D(nx=nm, ny=nm, k=k, chi3=chi, eps_r=eps, f=f)

    def mx_oracle():
        x_ref, rep, born = onw.bvp_solve(pm, _oopts("ad", 60, 1e-8, 1e-8, 50, 30))
        return x_ref, [rep]
    c.append(("maxwell_born", J.make_problem("maxwell", nm, nm, 0.0, 1.0, (k, chi), eps_r=eps, source=f),
              _opts(J, J.JFNK_FP64, "ad", 60, 1e-8, 1e-8, 50, 30), np.zeros(2 * nm * nm), 1, mx_oracle, 1e-8,
              False))
    nb = 40
    v0 = si.burgers2d_ic(nb, nb, "4vc")
    b2 = opdes.Burgers2D(nx=nb, ny=nb, nu=0.05, dt=0.05, theta=0.5, courant=1.0)
    c.append(("burgers2d_4vc_cfl_mixed", J.make_problem("burgers2d", nb, nb, 0.0, 0.5, (0.05, 0.0, 1.0)),
              _opts(J, J.JFNK_MIXED_FP32, "ad", 30, 1e-9, 1e-5, max_newton=30), v0, 2,
              lambda: onw.time_steps(b2, v0, 2, _oopts("ad", 30, 1e-12, 1e-12)), 1e-5, False))
    return c


def _batch(J, cases, tile=None):
    ctx = J.jfnk_create(0)
    try:
        if tile is not None:
            assert J.jfnk_tune(ctx, J.JFNK_TUNE_BATCH_TILE, tile) == J.JFNK_OK
        xs = [torch.tensor(cs[3], device="cuda") for cs in cases]
        s, reps, sts = J.jfnk_solve_batch(ctx, [cs[1] for cs in cases], [cs[2] for cs in cases], None, xs,
                                          [cs[4] for cs in cases])
        torch.cuda.synchronize()
        return s, [x.cpu().numpy() for x in xs], reps, sts, J.jfnk_last_error(ctx)
    finally:
        J.jfnk_destroy(ctx)


def test_dcgs2_batch_matches_oracle(J):
    cases = _cases(J)
    s, xs, reps, sts, err = _batch(J, cases)
    assert s == J.JFNK_OK, (err, sts)
    for (name, _, _, x0, steps, oracle, tol_x, exact), x, rep in zip(cases, xs, reps):
        x_ref, oreps = oracle()
        e = np.abs(x - x_ref).max() / np.abs(x_ref).max()
        assert e <= tol_x, (name, e)
        nn = sum(r.newton_its for r in oreps)
        kk = sum(r.krylov_its for r in oreps)
        if exact:
            assert rep.newton_its == nn, (name, rep.newton_its, nn)
            assert abs(rep.krylov_its - kk) <= 2 * max(nn, 1), (name, rep.krylov_its, kk)
        assert rep.steps_done == steps and rep.steps_failed == 0, name
        assert rep.jvp_calls >= rep.krylov_its > 0, name


def test_dcgs2_result_independent_of_mix_and_tile_size(J):
    cases = _cases(J)
    s, xs_mix, reps_mix, _, err = _batch(J, cases, tile=2048)
    assert s == J.JFNK_OK, err
    for i, cs in enumerate(cases):
        s1, xs1, reps1, _, err1 = _batch(J, [cs], tile=256)
        assert s1 == J.JFNK_OK, (cs[0], err1)
        assert np.array_equal(xs1[0], xs_mix[i]), cs[0]
        assert (reps1[0].newton_its, reps1[0].krylov_its, reps1[0].jvp_calls) == \
            (reps_mix[i].newton_its, reps_mix[i].krylov_its, reps_mix[i].jvp_calls), cs[0]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dcgs2_batch_agrees_with_single_solve(J, prec):
    """The same delayed-CGS2 iteration as jfnk_solve; only the reduction order differs."""
    n = 64
    u0 = si.allen_cahn_ic(n, n, 11)
    lp = J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))
    code = J.JFNK_FP64 if prec == "fp64" else J.JFNK_MIXED_FP32
    tol_n, tol_k, tol_x = (1e-10, 1e-10, 1e-10) if prec == "fp64" else (1e-9, 1e-6, 1e-5)
    o = _opts(J, code, "ad", 40, tol_n, tol_k, max_newton=30)
    ctx = J.jfnk_create(0)
    try:
        J.check(ctx, J.jfnk_set_problem(ctx, lp), "set")
        xs = u0.copy()
        rs = J.jfnk_report()
        J.check(ctx, J.jfnk_solve(ctx, o, None, xs, 3, rs), "solve")
        xb = u0.copy()
        s, reps, sts = J.jfnk_solve_batch(ctx, [lp], o, None, [xb], 3)
        assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    finally:
        J.jfnk_destroy(ctx)
    assert np.abs(xb - xs).max() <= tol_x * np.abs(xs).max()
    assert reps[0].steps_done == 3 and reps[0].steps_failed == 0
    if prec == "fp64":
        assert reps[0].newton_its == rs.newton_its
        assert abs(reps[0].krylov_its - rs.krylov_its) <= 2 * rs.newton_its


def test_fused_form_is_refused_in_batches(J):
    lp = J.make_problem("allen_cahn", 64, 64, 0.1, 0.5, (1e-3, 1.0))
    o = _opts(J, J.JFNK_MIXED_FP32)
    o.ortho = J.JFNK_DCGS2_FUSED
    ctx = J.jfnk_create(0)
    try:
        x = torch.tensor(si.allen_cahn_ic(64, 64, 0), device="cuda")
        s, _, _ = J.jfnk_solve_batch(ctx, [lp], o, None, [x], 1)
        assert s == J.JFNK_E_INVALID
    finally:
        J.jfnk_destroy(ctx)
