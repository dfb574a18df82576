"""The paper's reaction-diffusion problem with Dirichlet walls through the C ABI against the oracle (GPU).

App. A, Nonlinear Reaction-Diffusion: u_t = D lap u - u^3, u = 0 on the
boundary of [-1/2, 1/2]^2 (jfnk_problem p[2] = 1), Crank-Nicolson with
dt = C dx^2 / D at C = 1, Gaussian, multi-Gaussian and sinusoidal initial
data. The implicit-step Jacobian is SPD, so CG applies beside GMRES and
BiCGSTAB. Parity bar as for the other PDEs: solution to 1e-10 relative in
FP64 (1e-5 mixed), equal Newton counts, Krylov counts within 2 per Newton
step; also the batch engine, delayed CGS2 and its opt-in fused pass, and the
paper's 512^2 GPU grid.
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


KR = {"gmres": "JFNK_GMRES", "bicgstab": "JFNK_BICGSTAB", "cg": "JFNK_CG"}


def _opts(J, prec, lin="ad", krylov="gmres", restart=30, tol_n=1e-10, tol_k=1e-10, max_newton=15,
          max_krylov=200, ortho=None):
    o = J.jfnk_default_opts(prec)
    o.lin = J.JFNK_AD if lin == "ad" else J.JFNK_FD
    o.krylov = getattr(J, KR[krylov])
    o.restart, o.tol_newton, o.tol_krylov = restart, tol_n, tol_k
    o.max_newton, o.max_krylov = max_newton, max_krylov
    o.ortho = J.JFNK_CGS2 if ortho is None else ortho
    return o


def _oopts(lin="ad", krylov="gmres", restart=30, tol_n=1e-10, tol_k=1e-10, max_newton=15, max_krylov=200):
    return onw.Options(lin=lin, krylov=krylov, restart=restart, tol_newton=tol_n, tol_krylov=tol_k,
                       max_newton=max_newton, max_cycles=max_krylov)


def _problem(J, n, D):
    dt = (1.0 / (n + 1)) ** 2 / D
    return (opdes.AllenCahn2D(nx=n, ny=n, D=D, dt=dt, theta=0.5, linear_coef=0.0, dirichlet=True),
            J.make_problem("allen_cahn", n, n, dt, 0.5, (D, 0.0, 1.0)))


def _run(J, ctx, lp, opts, x0, steps):
    J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
    x = torch.tensor(x0, device="cuda")
    rep = J.jfnk_report()
    s = J.jfnk_solve(ctx, opts, None, x, steps, rep)
    torch.cuda.synchronize()
    return s, x.cpu().numpy(), rep


def _compare(x, x_ref, rep, reps, tol_x):
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= tol_x
    nn = sum(r.newton_its for r in reps)
    assert rep.newton_its == nn, (rep.newton_its, nn)
    kk = sum(r.krylov_its for r in reps)
    assert abs(rep.krylov_its - kk) <= 2 * max(nn, 1), (rep.krylov_its, kk)


@pytest.mark.parametrize("kind", si.RD_KINDS)
@pytest.mark.parametrize("krylov", ["cg", "gmres", "bicgstab"])
@pytest.mark.parametrize("lin", ["ad", "fd"])
def test_fp64_steps_against_oracle(J, ctx, kind, krylov, lin):
    n, D = 48, 0.01
    p, lp = _problem(J, n, D)
    u0 = si.rd_ic(n, n, kind)
    s, x, rep = _run(J, ctx, lp, _opts(J, J.JFNK_FP64, lin, krylov), u0, 2)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    x_ref, reps = onw.time_steps(p, u0, 2, _oopts(lin, krylov))
    _compare(x, x_ref, rep, reps, 1e-10)


@pytest.mark.parametrize("fused", [False, True])
def test_mixed_delayed_cgs2(J, ctx, fused):
    n, D = 64, 0.001
    p, lp = _problem(J, n, D)
    u0 = si.rd_ic(n, n, "multigauss")
    s, x, rep = _run(J, ctx, lp, _opts(J, J.JFNK_MIXED_FP32, "ad", "gmres", 40, 1e-9, 1e-5, max_newton=30,
                                       ortho=J.JFNK_DCGS2_FUSED if fused else J.JFNK_DCGS2), u0, 2)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    x_ref, reps = onw.time_steps(p, u0, 2, _oopts("ad", "gmres", 40, 1e-12, 1e-12))
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-5


def test_batch_engine(J, ctx):
    n, D = 40, 0.01
    p, lp = _problem(J, n, D)
    xs0 = [si.rd_ic(n, n, k) for k in si.RD_KINDS]
    xs = [torch.tensor(x0, device="cuda") for x0 in xs0]
    s, reps, sts = J.jfnk_solve_batch(ctx, [lp] * 3, _opts(J, J.JFNK_FP64), None, xs, 2)
    torch.cuda.synchronize()
    assert s == J.JFNK_OK, (J.jfnk_last_error(ctx), sts)
    for x0, x, rep in zip(xs0, xs, reps):
        x_ref, oreps = onw.time_steps(p, x0, 2, _oopts())
        _compare(x.cpu().numpy(), x_ref, rep, oreps, 1e-10)


def test_paper_gpu_grid_512(J, ctx):
    n, D = 512, 0.01
    p, lp = _problem(J, n, D)
    u0 = si.rd_ic(n, n, "sinusoidal")
    s, x, rep = _run(J, ctx, lp, _opts(J, J.JFNK_FP64, "ad", "cg", tol_n=1e-8, tol_k=1e-8), u0, 1)
    assert s == J.JFNK_OK, J.jfnk_last_error(ctx)
    x_ref, reps = onw.time_steps(p, u0, 1, _oopts("ad", "cg", tol_n=1e-8, tol_k=1e-8))
    _compare(x, x_ref, rep, reps, 1e-8)
