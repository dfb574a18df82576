"""Python binding of libjfnk (argument marshalling only).

The functions below have the names and signatures of the C ABI declared in
include/jfnk.h; every step of the computation runs in the library's CUDA
kernels. Array arguments are raw addresses (``int``) or objects with a
``data_ptr()`` method (torch tensors), so callers keep device memory in
PyTorch and hand its pointers through. Importing this module loads the
in-tree ``libjfnk.so`` and raises ImportError when it has not been built;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libjfnk.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError("libjfnk.so is not built; run `python -m paper_2605_13378_gb300.build` "
                      "(or __graft_entry__.build()) first")
lib = C.CDLL(_LIB_PATH)

# enums (include/jfnk.h)
JFNK_OK, JFNK_E_INVALID, JFNK_E_OOM, JFNK_E_CUDA, JFNK_E_NOT_CONVERGED = 0, 1, 2, 3, 4
JFNK_E_BREAKDOWN, JFNK_E_NONFINITE, JFNK_E_LINESEARCH, JFNK_E_TIMEOUT, JFNK_E_BUSY = 5, 6, 7, 8, 9
JFNK_AD, JFNK_FD = 0, 1
JFNK_GMRES, JFNK_BICGSTAB, JFNK_CG = 0, 1, 2
JFNK_BURGERS1D, JFNK_ALLEN_CAHN2D, JFNK_SU_OLSON2D, JFNK_MAXWELL_TE2D, JFNK_BURGERS2D = 0, 1, 2, 3, 4
JFNK_MAXWELL_VEC2D = 5
JFNK_PRECOND_NONE, JFNK_PRECOND_CSLP = 0, 1
JFNK_FP64, JFNK_FP32, JFNK_MIXED_FP32, JFNK_MIXED_BF16 = 0, 1, 2, 3
JFNK_EPS_SCALED, JFNK_EPS_PAPER = 0, 1
JFNK_CGS2, JFNK_DCGS2, JFNK_DCGS2_FUSED = 0, 1, 2
JFNK_MAX_RESTART = 64
JFNK_ABI_VERSION = 3
JFNK_NOALLOC_MAX_FX_BYTES = 4194304
JFNK_NOALLOC_SCRATCH_BYTES = 4352 + JFNK_NOALLOC_MAX_FX_BYTES
JFNK_TUNE_BATCH_TILE, JFNK_TUNE_BULK_COPY = 0, 1

EXPORTED = ["jfnk_default_opts", "jfnk_create", "jfnk_set_problem", "jfnk_jvp", "jfnk_residual", "jfnk_solve",
            "jfnk_submit", "jfnk_poll", "jfnk_set_timing", "jfnk_kernel_stats", "jfnk_reset_stats",
            "jfnk_last_error", "jfnk_status_string", "jfnk_destroy", "jfnk_jvp_fd_noalloc", "jfnk_solve_batch",
            "jfnk_batch_stats", "jfnk_tune"]


class jfnk_problem(C.Structure):
    _fields_ = [("pde", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("dt", C.c_double), ("theta", C.c_double),
                ("p", C.c_double * 8), ("aux", C.c_void_p * 2)]


class jfnk_opts(C.Structure):
    _fields_ = [("lin", C.c_int), ("krylov", C.c_int), ("prec", C.c_int), ("restart", C.c_int),
                ("max_newton", C.c_int), ("max_krylov", C.c_int), ("tol_newton", C.c_double),
                ("tol_krylov", C.c_double), ("fd_rule", C.c_int), ("fd_eps", C.c_double), ("ls_c1", C.c_double),
                ("ls_min_alpha", C.c_double), ("born_start", C.c_int), ("ortho", C.c_int), ("precond", C.c_int),
                ("precond_damping", C.c_double)]


class jfnk_report(C.Structure):
    _fields_ = [("status", C.c_int), ("steps_done", C.c_int), ("steps_failed", C.c_int), ("newton_its", C.c_int),
                ("krylov_its", C.c_int), ("jvp_calls", C.c_int), ("ls_backtracks", C.c_int),
                ("ls_failures", C.c_int), ("krylov_failures", C.c_int), ("res0", C.c_double),
                ("res_final", C.c_double), ("ms", C.c_double), ("dt_last", C.c_double),
                ("ls_alpha", C.c_double * 16), ("restart_used", C.c_int)]

    def as_dict(self) -> dict:
        return {k: (list(getattr(self, k)) if k == "ls_alpha" else getattr(self, k)) for k, _ in self._fields_}


_P = C.c_void_p
_sigs = {
    "jfnk_default_opts": (None, [C.POINTER(jfnk_opts), C.c_int]),
    "jfnk_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_size_t, _P]),
    "jfnk_set_problem": (C.c_int, [_P, C.POINTER(jfnk_problem)]),
    "jfnk_jvp": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P, _P, _P, C.c_double]),
    "jfnk_residual": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "jfnk_solve": (C.c_int, [_P, C.POINTER(jfnk_opts), _P, _P, C.c_int, C.POINTER(jfnk_report)]),
    "jfnk_submit": (C.c_int, [_P, C.POINTER(jfnk_problem), C.POINTER(jfnk_opts), _P, _P, C.c_int,
                              C.POINTER(C.c_ulonglong)]),
    "jfnk_poll": (C.c_int, [_P, C.c_ulonglong, C.POINTER(jfnk_report)]),
    "jfnk_set_timing": (C.c_int, [_P, C.c_int]),
    "jfnk_kernel_stats": (C.c_int, [_P, C.POINTER(C.c_char_p), C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.c_int]),
    "jfnk_reset_stats": (None, [_P]),
    "jfnk_last_error": (C.c_char_p, [_P]),
    "jfnk_status_string": (C.c_char_p, [C.c_int]),
    "jfnk_destroy": (None, [_P]),
    "jfnk_jvp_fd_noalloc": (C.c_int, [C.POINTER(jfnk_problem), C.c_int, _P, _P, _P, _P, _P, C.c_double, _P]),
    "jfnk_solve_batch": (C.c_int, [_P, C.c_int, C.POINTER(jfnk_problem), C.POINTER(jfnk_opts), _P, _P,
                                   C.POINTER(C.c_int), C.POINTER(jfnk_report), C.POINTER(C.c_int)]),
    "jfnk_batch_stats": (C.c_int, [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int,
                                   C.c_int]),
    "jfnk_tune": (C.c_int, [_P, C.c_int, C.c_longlong]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if hasattr(a, "ctypes"):           # numpy array (host memory)
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


class JfnkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{lib.jfnk_status_string(status).decode()}: {msg}")
        self.status = status


# --- the C ABI, one function per entry point ---------------------------------------------------

def jfnk_default_opts(prec: int = JFNK_FP64) -> jfnk_opts:
    o = jfnk_opts()
    lib.jfnk_default_opts(C.byref(o), prec)
    return o


def jfnk_create(device: int = 0, hbm_budget: int = 0, stream: int | None = None) -> int:
    h = C.c_void_p()
    s = lib.jfnk_create(C.byref(h), device, hbm_budget, stream)
    if s != JFNK_OK:
        raise JfnkError(s, "jfnk_create")
    return h.value


def jfnk_set_problem(ctx: int, prob: jfnk_problem) -> int:
    return lib.jfnk_set_problem(ctx, C.byref(prob))


def jfnk_jvp(ctx: int, lin: int, prec: int, x, v, b, F_out, Jv_out, fd_eps: float = 0.0) -> int:
    return lib.jfnk_jvp(ctx, lin, prec, _ptr(x), _ptr(v), _ptr(b), _ptr(F_out), _ptr(Jv_out), fd_eps)


def jfnk_residual(ctx: int, prec: int, x, b, F_out) -> int:
    return lib.jfnk_residual(ctx, prec, _ptr(x), _ptr(b), _ptr(F_out))


def jfnk_solve(ctx: int, opts: jfnk_opts, x_prev, x_inout, steps: int, rep: jfnk_report | None = None) -> int:
    return lib.jfnk_solve(ctx, C.byref(opts), _ptr(x_prev), _ptr(x_inout), steps,
                          C.byref(rep) if rep is not None else None)


def jfnk_submit(ctx: int, prob: jfnk_problem, opts: jfnk_opts, x0, x_out, steps: int) -> tuple[int, int]:
    t = C.c_ulonglong()
    s = lib.jfnk_submit(ctx, C.byref(prob), C.byref(opts), _ptr(x0), _ptr(x_out), steps, C.byref(t))
    return s, t.value


def jfnk_poll(ctx: int, ticket: int, rep: jfnk_report | None = None) -> int:
    return lib.jfnk_poll(ctx, ticket, C.byref(rep) if rep is not None else None)


def jfnk_set_timing(ctx: int, enable: bool) -> int:
    return lib.jfnk_set_timing(ctx, 1 if enable else 0)


def jfnk_kernel_stats(ctx: int) -> dict:
    cap = 32
    names = (C.c_char_p * cap)()
    launches = (C.c_longlong * cap)()
    ms = (C.c_double * cap)()
    by = (C.c_double * cap)()
    n = lib.jfnk_kernel_stats(ctx, names, launches, ms, by, cap)
    return {names[i].decode(): {"launches": launches[i], "ms": ms[i], "bytes": by[i]} for i in range(n)}


def jfnk_reset_stats(ctx: int) -> None:
    lib.jfnk_reset_stats(ctx)


def jfnk_last_error(ctx: int) -> str:
    r = lib.jfnk_last_error(ctx)
    return r.decode() if r else ""


def jfnk_status_string(s: int) -> str:
    return lib.jfnk_status_string(s).decode()


def jfnk_destroy(ctx: int) -> None:
    lib.jfnk_destroy(ctx)


def jfnk_jvp_fd_noalloc(prob: jfnk_problem, prec: int, x, v, b, F_out, Jv_out, fd_eps: float = 0.0,
                        stream: int | None = None) -> int:
    """FD Jacobian-vector product without a context and without allocating (see include/jfnk.h)."""
    return lib.jfnk_jvp_fd_noalloc(C.byref(prob), prec, _ptr(x), _ptr(v), _ptr(b), _ptr(F_out), _ptr(Jv_out),
                                   fd_eps, stream)


def jfnk_solve_batch(ctx: int, probs, opts, x_prev, x_inout, steps) -> tuple[int, list, list]:
    """Solve len(probs) problems together; opts and steps may be one value for all.

    Returns (status, reports, statuses). x_prev may be None or contain None entries.
    """
    n = len(probs)
    if isinstance(opts, jfnk_opts):
        opts = [opts] * n
    if isinstance(steps, int):
        steps = [steps] * n
    P = (jfnk_problem * n)(*probs)
    O = (jfnk_opts * n)(*opts)
    xp = None if x_prev is None else (C.c_void_p * n)(*[_ptr(a) for a in x_prev])
    xi = (C.c_void_p * n)(*[_ptr(a) for a in x_inout])
    st = (C.c_int * n)(*steps)
    R = (jfnk_report * n)()
    S = (C.c_int * n)()
    s = lib.jfnk_solve_batch(ctx, n, P, O, C.cast(xp, C.c_void_p) if xp is not None else None,
                             C.cast(xi, C.c_void_p), st, R, S)
    return s, [R[i] for i in range(n)], [S[i] for i in range(n)]


def jfnk_batch_stats(ctx: int, pde: int = 0, prec: int = 0, nx: int = 0, ny: int = 0) -> tuple[int, int]:
    """(kernel launches of the batch engine so far, tuned tile cells for that problem class or 0)."""
    kl = C.c_longlong()
    tc = C.c_int()
    lib.jfnk_batch_stats(ctx, C.byref(kl), C.byref(tc), pde, prec, nx, ny)
    return kl.value, tc.value


def jfnk_tune(ctx: int, knob: int, value: int) -> int:
    """Set one tuning or diagnostic knob of a context (JFNK_TUNE_*; see include/jfnk.h)."""
    return lib.jfnk_tune(ctx, knob, value)


# --- small conveniences over the same calls ------------------------------------------------------

PDE_IDS = {"burgers1d": JFNK_BURGERS1D, "allen_cahn": JFNK_ALLEN_CAHN2D, "su_olson": JFNK_SU_OLSON2D,
           "maxwell": JFNK_MAXWELL_TE2D, "burgers2d": JFNK_BURGERS2D, "maxwell_vec": JFNK_MAXWELL_VEC2D}


def make_problem(pde: str, nx: int, ny: int = 1, dt: float = 0.0, theta: float = 1.0, params=(),
                 eps_r=None, source=None) -> jfnk_problem:
    """Fill a jfnk_problem; eps_r / source are FP64 arrays (host numpy or device tensors)."""
    p = jfnk_problem()
    p.pde = PDE_IDS[pde]
    p.nx, p.ny, p.dt, p.theta = nx, ny, dt, theta
    for i, v in enumerate(params):
        p.p[i] = float(v)
    p.aux[0] = _ptr(eps_r)
    p.aux[1] = _ptr(source)
    return p


def check(ctx: int, status: int, what: str = "") -> None:
    if status != JFNK_OK:
        raise JfnkError(status, f"{what}: {jfnk_last_error(ctx)}")
