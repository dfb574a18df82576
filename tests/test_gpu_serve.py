"""Serving: requests solved in a concurrent mix equal the same requests solved alone (GPU).

jfnk_submit queues a solve and returns a ticket; admitted requests run
concurrently on the device while later ones wait for budget. Requests the
batch engine supports (GMRES; FP64, FP32, mixed FP32) join the running batch
between replays of its launch graph; the others (here a BiCGSTAB request) run
on the single-solve worker through jfnk_solve, one at a time, beside the batch. Every reduction uses a partition that
depends only on the request's own size, so a request's result must be
bitwise the same alone and in the mix; it must also agree with jfnk_solve
(bitwise on the slot path, to 1e-9 in FP64 and 1e-6 in mixed precision on
the batch path, whose reductions are ordered differently). The test also
checks the reports, the budget refusal, unknown tickets and a request that
fails (non-finite input).
"""
import time

import numpy as np
import pytest

import synthetic_inputs as si

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


def _requests(J):
    reqs = []
    for n, seed, prec in [(64, 0, J.JFNK_MIXED_FP32), (96, 1, J.JFNK_FP64), (128, 2, J.JFNK_MIXED_FP32),
                          (72, 3, J.JFNK_FP64)]:
        p = J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))
        o = J.jfnk_default_opts(prec)
        o.restart, o.tol_newton, o.tol_krylov = 40, 1e-8, 1e-6 if prec != J.JFNK_FP64 else 1e-8
        reqs.append((p, o, si.allen_cahn_ic(n, n, seed), 3))
    p = J.make_problem("su_olson", 40, 40, 1e-3, 0.5, (1.0, 1.0, 1.0, 1e-6, 1.0))
    o = J.jfnk_default_opts(J.JFNK_FP64)
    o.tol_newton, o.tol_krylov = 1e-9, 1e-10
    reqs.append((p, o, si.su_olson_ic(40, 40), 2))
    p = J.make_problem("burgers1d", 1024, 1, 1e-3, 1.0, (1e-2,))
    o = J.jfnk_default_opts(J.JFNK_FP64)
    o.tol_newton, o.tol_krylov = 1e-10, 1e-10
    reqs.append((p, o, si.burgers_ic(1024, 0), 1))
    p = J.make_problem("allen_cahn", 80, 80, 0.1, 0.5, (1e-3, 1.0))
    o = J.jfnk_default_opts(J.JFNK_FP64)
    o.krylov, o.tol_newton, o.tol_krylov = J.JFNK_BICGSTAB, 1e-9, 1e-10
    reqs.append((p, o, si.allen_cahn_ic(80, 80, 4), 2))
    n = 16
    eps, f = si.maxwell_medium(n, n, 0), si.maxwell_point_source(n, n)
    p = J.make_problem("maxwell", n, n, 0.0, 1.0, (3.0, 0.1), eps_r=eps, source=f)
    o = J.jfnk_default_opts(J.JFNK_FP64)
    o.restart, o.max_newton, o.max_krylov, o.tol_newton = 60, 50, 30, 1e-8
    reqs.append((p, o, np.zeros(2 * n * n), 1, eps, f))
    return reqs


def _serve(J, reqs, check_tickets=False):
    ctx = J.jfnk_create(0)
    try:
        outs, tickets = [], []
        for r in reqs:
            p, o, x0, steps = r[:4]
            xo = np.zeros_like(x0)
            s, t = J.jfnk_submit(ctx, p, o, x0, xo, steps)
            assert s == J.JFNK_OK
            outs.append(xo)
            tickets.append(t)
        reps = [None] * len(reqs)
        deadline = time.time() + 300
        pending = set(range(len(reqs)))
        while pending and time.time() < deadline:
            for i in list(pending):
                rep = J.jfnk_report()
                s = J.jfnk_poll(ctx, tickets[i], rep)
                if s != J.JFNK_E_BUSY:
                    assert s == J.JFNK_OK, (i, J.jfnk_status_string(s))
                    reps[i] = rep
                    pending.discard(i)
            time.sleep(0.005)
        assert not pending
        if check_tickets:
            assert J.jfnk_poll(ctx, tickets[0], None) == J.JFNK_E_INVALID      # a finished ticket is gone
            assert J.jfnk_poll(ctx, 987654321, None) == J.JFNK_E_INVALID
        return outs, reps
    finally:
        J.jfnk_destroy(ctx)


def test_mix_equals_alone(J):
    reqs = _requests(J)
    outs, reps = _serve(J, reqs, check_tickets=True)
    for i, r in enumerate(reqs):
        p, o, x0, steps = r[:4]
        # alone through the server: the same executor, bitwise the same result and counts
        o1, r1 = _serve(J, [r])
        assert np.array_equal(o1[0], outs[i]), i
        assert (r1[0].newton_its, r1[0].krylov_its) == (reps[i].newton_its, reps[i].krylov_its), i
        assert reps[i].ms > 0
        # alone through jfnk_solve
        c1 = J.jfnk_create(0)
        try:
            J.check(c1, J.jfnk_set_problem(c1, p), "set")
            xa = x0.copy()
            ra = J.jfnk_report()
            J.check(c1, J.jfnk_solve(c1, o, None, xa, steps, ra), "solve")
        finally:
            J.jfnk_destroy(c1)
        if o.krylov == J.JFNK_BICGSTAB:
            assert np.array_equal(xa, outs[i]), i
            assert (ra.newton_its, ra.krylov_its) == (reps[i].newton_its, reps[i].krylov_its), i
        else:
            tol = 1e-9 if o.prec == J.JFNK_FP64 else 1e-6
            assert np.abs(xa - outs[i]).max() <= tol * np.abs(xa).max(), (i, np.abs(xa - outs[i]).max())
            assert ra.newton_its == reps[i].newton_its or o.prec != J.JFNK_FP64, i


def test_budget_refusal_and_failing_request(J):
    ctx = J.jfnk_create(0, 8 << 20)       # 8 MB: small requests fit, a 1024^2 one never can
    try:
        p = J.make_problem("allen_cahn", 1024, 1024, 0.1, 0.5, (1e-3, 1.0))
        o = J.jfnk_default_opts(J.JFNK_FP64)
        x0 = np.zeros(1024 * 1024)
        s, _ = J.jfnk_submit(ctx, p, o, x0, x0.copy(), 1)
        assert s == J.JFNK_E_OOM
        n = 32
        p = J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))
        bad = si.allen_cahn_ic(n, n, 0)
        bad[5] = np.nan
        xo = np.zeros_like(bad)
        s, t = J.jfnk_submit(ctx, p, o, bad, xo, 1)
        assert s == J.JFNK_OK
        rep = J.jfnk_report()
        for _ in range(10000):
            s = J.jfnk_poll(ctx, t, rep)
            if s != J.JFNK_E_BUSY:
                break
            time.sleep(0.005)
        assert s == J.JFNK_E_NONFINITE
    finally:
        J.jfnk_destroy(ctx)
