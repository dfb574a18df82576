"""Batched solves (jfnk_solve_batch) against the CPU oracle and against themselves (GPU).

jfnk_solve_batch advances many independent Newton-GMRES solves together, one
phase of each per kernel launch, with every solve's control state on the
device. Its parity bar is the single-solve one: each problem of a mixed batch
(five PDEs, FP64 / FP32 / mixed FP32, AD and FD, fixed and adaptive CFL steps) is compared with the oracle
on the same seeded input (solution to 1e-10 in FP64, 1e-5 in reduced
precision; Newton counts equal in FP64; Krylov counts within 2 per Newton
step, or inside the oracle's own perturbation band for the radiation problem).
Reductions are summed per 256-cell unit in a fixed order, so a problem's
result must be bitwise the same in a batch of one and in the mix, whatever
tile size the autotuner chose; that is checked with two forced tile sizes.
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
    return o


def _oopts(lin="ad", restart=30, tol_n=1e-10, tol_k=1e-10, max_newton=15, max_krylov=100):
    return onw.Options(lin=lin, krylov="gmres", restart=restart, tol_newton=tol_n, tol_krylov=tol_k,
                       max_newton=max_newton, max_cycles=max_krylov)


def _cases(J):
    """(name, problem, opts, x0, steps, oracle() -> (x_ref, [reports]), tol_x, exact_newton, band())."""
    c = []
    N = 1024
    u0 = si.burgers_ic(N, 0)
    pb = opdes.Burgers1D(N=N, nu=1e-2, dt=1e-3)
    for lin in ("ad", "fd"):
        c.append((f"burgers_{lin}", J.make_problem("burgers1d", N, 1, 1e-3, 1.0, (1e-2,)),
                  _opts(J, J.JFNK_FP64, lin), u0, 1,
                  lambda lin=lin: onw.time_steps(pb, u0, 1, _oopts(lin)), 1e-10, True, None))
    n = 72
    a0 = si.allen_cahn_ic(n, n, 3)
    pa = opdes.AllenCahn2D(nx=n, ny=n, D=1e-3, dt=0.1, theta=0.5)
    for lin in ("ad", "fd"):
        c.append((f"allen_cahn_{lin}", J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0)),
                  _opts(J, J.JFNK_FP64, lin, 40), a0, 2,
                  lambda lin=lin: onw.time_steps(pa, a0, 2, _oopts(lin, 40)), 1e-10, True, None))
    m0 = si.allen_cahn_ic(n, n, 5)
    for prec, lin in (("mixed", "ad"), ("mixed", "fd"), ("fp32", "ad")):
        code = J.JFNK_MIXED_FP32 if prec == "mixed" else J.JFNK_FP32
        tol_n = 1e-4 if prec == "fp32" else 1e-9
        c.append((f"allen_cahn_{prec}_{lin}", J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0)),
                  _opts(J, code, lin, 40, tol_n, 1e-5, max_newton=30), m0, 1,
                  lambda: onw.time_steps(pa, m0, 1, _oopts("ad", 40, 1e-12, 1e-12)), 1e-5, False, None))
    ns = 32
    s0 = si.su_olson_ic(ns, ns)
    ps = opdes.SuOlson2D(nx=ns, ny=ns, dt=1e-3, theta=0.5)
    so_run = lambda xs: onw.time_steps(ps, xs, 2, _oopts("ad", 30, 1e-9, 1e-10))
    c.append(("su_olson", J.make_problem("su_olson", ns, ns, 1e-3, 0.5, (1.0, 1.0, 1.0, 1e-6, 1.0)),
              _opts(J, J.JFNK_FP64, "ad", 30, 1e-9, 1e-10), s0, 2, lambda: so_run(s0), 1e-10, True,
              lambda: _band(lambda xs: so_run(xs)[1], s0)))
    nm, k, chi = 16, 3.0, 0.1
    eps, f = si.maxwell_medium(nm, nm, 0), si.maxwell_point_source(nm, nm)
    pm = opdes.MaxwellTE2D(nx=nm, ny=nm, k=k, chi3=chi, eps_r=eps, f=f)

    def mx_oracle():
        x_ref, rep, born = onw.bvp_solve(pm, _oopts("ad", 60, 1e-8, 1e-8, 50, 30))
        return x_ref, [rep]
    c.append(("maxwell_born", J.make_problem("maxwell", nm, nm, 0.0, 1.0, (k, chi), eps_r=eps, source=f),
              _opts(J, J.JFNK_FP64, "ad", 60, 1e-8, 1e-8, 50, 30), np.zeros(2 * nm * nm), 1, mx_oracle, 1e-8,
              True, "no_krylov"))
    # 2D Burgers: fixed step (TGV), adaptive CFL step (DSL, FD), adaptive mixed precision (4VC)
    nb = 40
    t0, d0, v0 = (si.burgers2d_ic(nb, nb, k) for k in ("tgv", "dsl", "4vc"))
    b2 = lambda C, dt=0.05: opdes.Burgers2D(nx=nb, ny=nb, nu=0.05, dt=dt, theta=0.5, courant=C)
    c.append(("burgers2d_tgv", J.make_problem("burgers2d", nb, nb, 0.05, 0.5, (0.05, 0.0, 0.0)),
              _opts(J, J.JFNK_FP64, "ad"), t0, 3,
              lambda: onw.time_steps(b2(0.0), t0, 3, _oopts("ad")), 1e-10, True, None))
    c.append(("burgers2d_dsl_cfl_fd", J.make_problem("burgers2d", nb, nb, 0.0, 0.5, (0.05, 0.0, 1.0)),
              _opts(J, J.JFNK_FP64, "fd"), d0, 3,
              lambda: onw.time_steps(b2(1.0), d0, 3, _oopts("fd")), 1e-10, True, None))
    c.append(("burgers2d_4vc_cfl_mixed", J.make_problem("burgers2d", nb, nb, 0.0, 0.5, (0.05, 0.0, 1.0)),
              _opts(J, J.JFNK_MIXED_FP32, "ad", 30, 1e-9, 1e-5, max_newton=30), v0, 2,
              lambda: onw.time_steps(b2(1.0), v0, 2, _oopts("ad", 30, 1e-12, 1e-12)), 1e-5, False, None))
    return c


def _band(run, x0, n_pert=4):
    counts = []
    for seed in range(n_pert + 1):
        xp = x0 if seed == 0 else x0 * (1 + 1e-15 * np.random.default_rng(seed).standard_normal(x0.size))
        counts.append(sum(r.krylov_its for r in run(xp)))
    return min(counts), max(counts)


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


def test_mixed_batch_matches_oracle(J):
    cases = _cases(J)
    s, xs, reps, sts, err = _batch(J, cases)
    assert s == J.JFNK_OK, (err, sts)
    for (name, _, _, x0, steps, oracle, tol_x, exact_newton, band), x, rep in zip(cases, xs, reps):
        x_ref, oreps = oracle()
        e = np.abs(x - x_ref).max() / np.abs(x_ref).max()
        assert e <= tol_x, (name, e)
        nn = sum(r.newton_its for r in oreps)
        if exact_newton:
            assert rep.newton_its == nn, (name, rep.newton_its, nn)
        if band == "no_krylov":
            continue
        kk = sum(r.krylov_its for r in oreps)
        if band is None:
            if exact_newton:
                assert abs(rep.krylov_its - kk) <= 2 * max(nn, 1), (name, rep.krylov_its, kk)
        else:
            lo, hi = band()
            assert 0.9 * lo - 2 * nn <= rep.krylov_its <= 1.1 * hi + 2 * nn, (name, rep.krylov_its, (lo, hi))
        assert rep.steps_done == steps and rep.steps_failed == 0, name
        assert rep.jvp_calls >= rep.krylov_its > 0, name


def test_result_independent_of_mix_and_tile_size(J):
    cases = _cases(J)
    s, xs_mix, reps_mix, _, err = _batch(J, cases, tile=2048)
    assert s == J.JFNK_OK, err
    for i, cs in enumerate(cases):
        s1, xs1, reps1, _, err1 = _batch(J, [cs], tile=256)
        assert s1 == J.JFNK_OK, (cs[0], err1)
        assert np.array_equal(xs1[0], xs_mix[i]), cs[0]
        assert (reps1[0].newton_its, reps1[0].krylov_its, reps1[0].jvp_calls) == \
            (reps_mix[i].newton_its, reps_mix[i].krylov_its, reps_mix[i].jvp_calls), cs[0]


def test_batch_agrees_with_single_solve(J):
    """Same algorithm as jfnk_solve; only the reduction order differs."""
    n = 64
    u0 = si.allen_cahn_ic(n, n, 9)
    lp = J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))
    o = _opts(J, J.JFNK_FP64, "ad", 40, 1e-10, 1e-10)
    ctx = J.jfnk_create(0)
    try:
        J.check(ctx, J.jfnk_set_problem(ctx, lp), "set")
        xs = u0.copy()
        rs = J.jfnk_report()
        J.check(ctx, J.jfnk_solve(ctx, o, None, xs, 3, rs), "solve")
        xb = u0.copy()                               # host arrays through the batch call
        s, reps, sts = J.jfnk_solve_batch(ctx, [lp], o, None, [xb], 3)
        assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    finally:
        J.jfnk_destroy(ctx)
    assert np.abs(xb - xs).max() <= 1e-10 * np.abs(xs).max()
    assert reps[0].newton_its == rs.newton_its and reps[0].steps_done == 3
    assert abs(reps[0].krylov_its - rs.krylov_its) <= 2 * rs.newton_its


def test_many_small_solves_and_launch_count(J):
    """64 Allen-Cahn solves of 32^2 (seeds 0..63) in one batch: each equals its batch-of-one result, and the
    whole batch needs far fewer kernel launches than 64 separate batches."""
    n, cnt = 32, 64
    lp = J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))
    o = _opts(J, J.JFNK_MIXED_FP32, "ad", 30, 1e-9, 1e-6, max_newton=30)
    x0 = [si.allen_cahn_ic(n, n, s) for s in range(cnt)]
    ctx = J.jfnk_create(0)
    try:
        xs = [torch.tensor(a, device="cuda") for a in x0]
        s, reps, sts = J.jfnk_solve_batch(ctx, [lp] * cnt, o, None, xs, 2)
        assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
        launches_all, tile = J.jfnk_batch_stats(ctx, J.JFNK_ALLEN_CAHN2D, J.JFNK_MIXED_FP32, n, n)
        assert tile in (256, 512, 1024, 2048)
        single = []
        for i in (0, 17, 63):
            xi = torch.tensor(x0[i], device="cuda")
            before = J.jfnk_batch_stats(ctx)[0]
            s1, r1, _ = J.jfnk_solve_batch(ctx, [lp], o, None, [xi], 2)
            assert s1 == J.JFNK_OK
            single.append(J.jfnk_batch_stats(ctx)[0] - before)
            assert torch.equal(xi, xs[i]), i
            assert r1[0].krylov_its == reps[i].krylov_its
    finally:
        J.jfnk_destroy(ctx)
    assert all(r.steps_done == 2 and r.steps_failed == 0 for r in reps)
    assert launches_all < 0.25 * cnt * min(single), (launches_all, single)
    # every solve meets the FP64 nonlinear tolerance of its own problem
    p = opdes.AllenCahn2D(nx=n, ny=n, D=1e-3, dt=0.1, theta=0.5)
    for i in (0, 31, 63):
        x1, _ = onw.time_steps(p, x0[i], 2, _oopts("ad", 30, 1e-12, 1e-12))
        assert np.abs(xs[i].cpu().numpy() - x1).max() <= 1e-5 * np.abs(x1).max()


def test_invalid_and_budget(J):
    n = 32
    lp = J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))
    x = np.zeros(n * n)
    ctx = J.jfnk_create(0)
    try:
        o = _opts(J, J.JFNK_FP64)
        o.krylov = J.JFNK_BICGSTAB
        assert J.jfnk_solve_batch(ctx, [lp], o, None, [x], 1)[0] == J.JFNK_E_INVALID
        assert "GMRES" in J.jfnk_last_error(ctx)
        assert J.jfnk_solve_batch(ctx, [lp], _opts(J, J.JFNK_MIXED_BF16), None, [x], 1)[0] == J.JFNK_E_INVALID
        assert J.jfnk_solve_batch(ctx, [lp], _opts(J, J.JFNK_FP64, restart=65), None, [x], 1)[0] == J.JFNK_E_INVALID
        assert J.jfnk_solve_batch(ctx, [lp], _opts(J, J.JFNK_FP64), None, [x], 0)[0] == J.JFNK_E_INVALID
        assert J.jfnk_solve_batch(ctx, [], _opts(J, J.JFNK_FP64), None, [], [])[0] == J.JFNK_OK
        # u = 0 is a steady state: zero Newton iterations, state untouched
        s, reps, _ = J.jfnk_solve_batch(ctx, [lp], _opts(J, J.JFNK_FP64), None, [x], 3)
        assert s == J.JFNK_OK and reps[0].newton_its == 0 and reps[0].steps_done == 3 and (x == 0).all()
        # a non-finite input ends that solve with JFNK_E_NONFINITE, the other solve of the batch converges
        bad = si.allen_cahn_ic(n, n, 1)
        bad[7] = np.nan
        good = si.allen_cahn_ic(n, n, 2)
        s, reps, sts = J.jfnk_solve_batch(ctx, [lp, lp], _opts(J, J.JFNK_FP64), None, [bad, good], 1)
        assert sts == [J.JFNK_E_NONFINITE, J.JFNK_OK] and s == J.JFNK_E_NONFINITE
        assert reps[1].steps_done == 1 and reps[1].newton_its > 0
    finally:
        J.jfnk_destroy(ctx)
    c = J.jfnk_create(0, 1 << 20)
    try:
        big = J.make_problem("allen_cahn", 512, 512, 0.1, 0.5, (1e-3, 1.0))
        xb = np.zeros(512 * 512)
        assert J.jfnk_solve_batch(c, [big], _opts(J, J.JFNK_FP64), None, [xb], 1)[0] == J.JFNK_E_OOM
        assert "budget" in J.jfnk_last_error(c)
    finally:
        J.jfnk_destroy(c)
