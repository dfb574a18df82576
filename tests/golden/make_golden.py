"""Write the stored expected values under tests/golden/ by running the oracle.

Only oracle/ and synthetic_inputs are called here; nothing comes from the
CUDA library. Usage: python tests/golden/make_golden.py [name ...]

allen_cahn_2048_step1.json
    Allen-Cahn on the 2048^2 periodic grid (D = 1e-3, dt = 0.1, theta = 1/2,
    u0 ~ U[-0.1, 0.1] from seed 0): the first implicit step solved by the
    oracle's Newton + GMRES(40) with the complex-step (AD) JVP, tol_Newton
    1e-8, tol_Krylov 1e-8 (FP64). Stores the Newton and Krylov counts, the
    residual history and summary statistics and samples of the solution.

allen_cahn_2048_step1_ref.json
    The same step solved to the limit of FP64 (tol_Newton 1e-13, tol_Krylov
    1e-12), so that the stored values stand for the exact root to about
    1e-11 relative: the reference for the benchmark's FP64 and mixed-precision
    solves at their solution tolerances (1e-10 and 1e-5). Stores 4096
    solution samples at stride 1024 (offset (37 k) mod 1024 in stride k, so
    every row is hit twice at varying columns), all 2048 row sums, and the
    counts and summary statistics.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synthetic_inputs as si  # noqa: E402
from oracle import newton as onw, pdes as opdes  # noqa: E402

SAMPLE_IDX = [0, 1, 2047, 2048, 1234567, 2 ** 21 + 777, 4194303]


def allen_cahn_2048_step1():
    n = 2048
    p = opdes.AllenCahn2D(nx=n, ny=n, D=1e-3, dt=0.1, theta=0.5)
    u0 = si.allen_cahn_ic(n, n, 0)
    opt = onw.Options(lin="ad", krylov="gmres", restart=40, max_cycles=100, max_newton=15,
                      tol_newton=1e-8, tol_krylov=1e-8)
    t = time.time()
    x, reps = onw.time_steps(p, u0, 1, opt)
    r = reps[0]
    return {
        "workload": "allen_cahn 2048^2, D=1e-3, dt=0.1, theta=0.5, seed 0, step 1",
        "solver": "Newton + GMRES(40), AD (complex step), FP64, tol_newton 1e-8, tol_krylov 1e-8",
        "status": r.status, "newton_its": r.newton_its, "krylov_its": r.krylov_its,
        "jvp_calls": r.jvp_calls, "ls_backtracks": r.ls_backtracks, "res0": r.res0, "res_final": r.res_final,
        "history": r.history, "x_sum": float(x.sum()), "x_sumsq": float((x * x).sum()),
        "x_absmax": float(np.abs(x).max()), "sample_idx": SAMPLE_IDX,
        "x_samples": [float(x[i]) for i in SAMPLE_IDX], "oracle_seconds": time.time() - t,
    }


def ref_sample_idx(n: int = 2048, count: int = 4096) -> list:
    stride = n * n // count
    return [k * stride + (37 * k) % stride for k in range(count)]


def allen_cahn_2048_step1_ref():
    n = 2048
    p = opdes.AllenCahn2D(nx=n, ny=n, D=1e-3, dt=0.1, theta=0.5)
    u0 = si.allen_cahn_ic(n, n, 0)
    opt = onw.Options(lin="ad", krylov="gmres", restart=40, max_cycles=100, max_newton=15,
                      tol_newton=1e-13, tol_krylov=1e-12)
    t = time.time()
    x, reps = onw.time_steps(p, u0, 1, opt)
    r = reps[0]
    idx = ref_sample_idx(n)
    return {
        "workload": "allen_cahn 2048^2, D=1e-3, dt=0.1, theta=0.5, seed 0, step 1",
        "solver": "Newton + GMRES(40), AD (complex step), FP64, tol_newton 1e-13, tol_krylov 1e-12",
        "status": r.status, "newton_its": r.newton_its, "krylov_its": r.krylov_its,
        "res0": r.res0, "res_final": r.res_final, "history": r.history,
        "x_sum": float(x.sum()), "x_sumsq": float((x * x).sum()), "x_absmax": float(np.abs(x).max()),
        "row_sums": [float(v) for v in x.reshape(n, n).sum(axis=1)],
        "sample_idx": idx, "x_samples": [float(x[i]) for i in idx], "oracle_seconds": time.time() - t,
    }


JOBS = {"allen_cahn_2048_step1": allen_cahn_2048_step1, "allen_cahn_2048_step1_ref": allen_cahn_2048_step1_ref}

if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    for name in names:
        out = JOBS[name]()
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(out, f, indent=None if name.endswith("_ref") else 1)
        print(name, {k: out[k] for k in ("status", "newton_its", "krylov_its", "oracle_seconds")})
