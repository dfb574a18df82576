"""jfnk_jvp_fd_noalloc against jfnk_jvp (GPU).

jfnk_jvp_fd_noalloc serves callers that cannot allocate device memory: it
needs no context and takes its workspace from one fixed device array. These
tests call it through the C ABI and check its output against the context
entry point jfnk_jvp (lin = FD) on the same inputs, on consecutive calls
(the array keeps the previous call's contents, so a second call must not see
stale state), with F(x) written to the caller's array and kept in the
library's array, and check that requests too large for that array are
refused before anything runs. Tolerances are those of the FD parity tests:
F(x) comes from the same residual sweep and must agree to rounding; the
quotient may differ by the rounding of the step's two norms (reduced in a
different order), amplified by 1/eps, so it is held to 1e-6 of max |Jv| in
FP64 and 1e-3 in FP32.

This file runs last in the suite (its name sorts last) and also passes alone.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import pdes as opdes

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


def _case(J, name, dtype):
    rng = np.random.default_rng(11)
    if name == "allen_cahn":
        nx, ny = 64, 48
        lp = J.make_problem("allen_cahn", nx, ny, 0.1, 0.5, (1e-3, 1.0))
        x = rng.uniform(-1, 1, nx * ny)
        b = opdes.AllenCahn2D(nx=nx, ny=ny, D=1e-3, dt=0.1).rhs(0.9 * x)
        keep = ()
    elif name == "burgers":
        lp = J.make_problem("burgers1d", 1024, 1, 1e-3, 1.0, (1e-2,))
        x = si.burgers_ic(1024, 0)
        b = opdes.Burgers1D(N=1024).rhs(x)
        keep = ()
    elif name == "burgers2d":
        nx, ny = 48, 40                       # fixed step (Courant number 0): the step is the caller's dt
        lp = J.make_problem("burgers2d", nx, ny, 2e-3, 0.5, (0.05, 0.0, 0.0))
        x = si.burgers2d_ic(nx, ny, "tgv") + 0.1 * rng.standard_normal(2 * nx * ny)
        b = opdes.Burgers2D(nx=nx, ny=ny, nu=0.05, dt=2e-3).rhs(x)
        keep = ()
    elif name == "su_olson":
        nx = ny = 40
        lp = J.make_problem("su_olson", nx, ny, 1e-2, 0.5, (1.0, 1.0, 1.0, 1e-6, 1.0))
        x = np.concatenate([rng.uniform(0.1, 1, nx * ny), rng.uniform(0.2, 1, nx * ny)])
        b = opdes.SuOlson2D(nx=nx, ny=ny, dt=1e-2).rhs(0.95 * x)
        keep = ()
    else:
        nx, ny = 32, 24
        eps = torch.tensor(si.maxwell_medium(nx, ny, 2), device="cuda")
        src = torch.tensor(si.maxwell_point_source(nx, ny), device="cuda")
        lp = J.make_problem("maxwell", nx, ny, 0.0, 1.0, (6.0, 0.2), eps_r=eps, source=src)
        x = rng.standard_normal(2 * nx * ny)
        b = None
        keep = (eps, src)      # device arrays used in place: keep them alive
    v = rng.standard_normal(x.size)
    t = lambda a: None if a is None else torch.tensor(a, dtype=dtype, device="cuda")
    return lp, t(x), t(v), t(b), keep


def _reference(J, lp, prec, x, v, b, fd_eps):
    ctx = J.jfnk_create(0)
    try:
        J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
        F = torch.empty_like(x)
        Jv = torch.empty_like(x)
        J.check(ctx, J.jfnk_jvp(ctx, J.JFNK_FD, prec, x, v, b, F, Jv, fd_eps), "jvp")
        torch.cuda.synchronize()
        return F, Jv
    finally:
        J.jfnk_destroy(ctx)


@pytest.mark.parametrize("name,prec", [("allen_cahn", "fp64"), ("burgers", "fp64"), ("su_olson", "fp64"),
                                       ("maxwell", "fp64"), ("burgers2d", "fp64"), ("allen_cahn", "fp32")])
def test_noalloc_fd_jvp_matches_context_entry_point(J, name, prec):
    dtype = torch.float64 if prec == "fp64" else torch.float32
    code = J.JFNK_FP64 if prec == "fp64" else J.JFNK_FP32
    tol = 1e-6 if prec == "fp64" else 1e-3
    lp, x, v, b, _keep = _case(J, name, dtype)
    F_ref, Jv_ref = _reference(J, lp, code, x, v, b, 0.0)
    scale = Jv_ref.abs().max().item()
    # two calls in a row: F(x) into the caller's array, then kept in the library's array
    for F_out in (torch.full_like(x, np.nan), None):
        Jv = torch.full_like(x, np.nan)
        s = J.jfnk_jvp_fd_noalloc(lp, code, x, v, b, F_out, Jv, 0.0)
        assert s == J.JFNK_OK, J.jfnk_status_string(s)
        torch.cuda.synchronize()
        assert torch.isfinite(Jv).all()
        assert (Jv - Jv_ref).abs().max().item() <= tol * scale
        if F_out is not None:
            assert torch.equal(F_out, F_ref)
    # a fixed step: the same sweeps, so the quotient agrees to rounding
    F_ref2, Jv_ref2 = _reference(J, lp, code, x, v, b, 1e-6)
    Jv = torch.empty_like(x)
    assert J.jfnk_jvp_fd_noalloc(lp, code, x, v, b, None, Jv, 1e-6) == J.JFNK_OK
    torch.cuda.synchronize()
    assert (Jv - Jv_ref2).abs().max().item() <= 1e-12 * Jv_ref2.abs().max().item() * (1 if prec == "fp64" else 1e6)


def test_noalloc_refuses_what_does_not_fit(J):
    n = 1024                                    # 8 MB of FP64 F(x) > JFNK_NOALLOC_MAX_FX_BYTES
    lp = J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))
    x = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    v = torch.ones_like(x)
    Jv = torch.empty_like(x)
    assert J.jfnk_jvp_fd_noalloc(lp, J.JFNK_FP64, x, v, None, None, Jv, 0.0) == J.JFNK_E_OOM
    # with the caller's F_out the same size works and matches the context entry point
    F = torch.empty_like(x)
    assert J.jfnk_jvp_fd_noalloc(lp, J.JFNK_FP64, x, v, None, F, Jv, 0.0) == J.JFNK_OK
    F_ref, Jv_ref = _reference(J, lp, J.JFNK_FP64, x, v, None, 0.0)
    assert (Jv - Jv_ref).abs().max().item() <= 1e-6 * Jv_ref.abs().max().item()
    # the Maxwell coefficients are FP64 device arrays: FP32 is refused
    lm = J.make_problem("maxwell", 16, 16, 0.0, 1.0, (3.0, 0.1))
    x32 = torch.zeros(2 * 256, dtype=torch.float32, device="cuda")
    assert J.jfnk_jvp_fd_noalloc(lm, J.JFNK_FP32, x32, x32, None, None, x32.clone(), 0.0) == J.JFNK_E_INVALID


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_zero_direction_gives_zero(J, prec):
    """J 0 = 0: with v = 0 the step rule takes ||v|| = 1, so the step stays finite and the quotient is
    (F(x) - F(x)) / eps, zero up to the rounding of F(x) between the two sweeps -- as in jfnk_jvp."""
    dtype = torch.float64 if prec == "fp64" else torch.float32
    code = J.JFNK_FP64 if prec == "fp64" else J.JFNK_FP32
    tol = 1e-6 if prec == "fp64" else 1e-3
    lp, x, _, b, _keep = _case(J, "allen_cahn", dtype)
    v = torch.zeros_like(x)
    F_ref, Jv_ref = _reference(J, lp, code, x, v, b, 0.0)
    bound = tol * F_ref.abs().max().item()
    assert torch.isfinite(Jv_ref).all() and Jv_ref.abs().max().item() <= bound
    for _ in range(2):
        Jv = torch.full_like(x, np.nan)
        assert J.jfnk_jvp_fd_noalloc(lp, code, x, v, b, None, Jv, 0.0) == J.JFNK_OK
        torch.cuda.synchronize()
        assert torch.isfinite(Jv).all() and Jv.abs().max().item() <= bound


def test_noalloc_refuses_an_adaptive_step(J):
    """A 2D Burgers problem whose step comes from the CFL rule has no step outside jfnk_solve."""
    nx, ny = 32, 32
    lp = J.make_problem("burgers2d", nx, ny, 0.0, 0.5, (0.05, 0.0, 1.0))
    x = torch.tensor(si.burgers2d_ic(nx, ny, "tgv"), device="cuda")
    Jv = torch.zeros_like(x)
    assert J.jfnk_jvp_fd_noalloc(lp, J.JFNK_FP64, x, x, None, None, Jv, 0.0) == J.JFNK_E_INVALID
    torch.cuda.synchronize()
    assert torch.count_nonzero(Jv).item() == 0
