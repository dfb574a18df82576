"""Benchmark: Newton solves/s of the JFNK hot path on the Allen-Cahn 2048^2 workload.

One benchmark step is one implicit time step of the 2D Allen-Cahn equation
(u_t = D lap u + u - u^3, periodic 2048 x 2048 grid, D = 1e-3, dt = 0.1,
Crank-Nicolson, u0 ~ U[-0.1, 0.1] from seed 0), solved by Newton with
backtracking line search and GMRES(40) whose operator is the forward-mode AD
JVP. K timed steps advance the trajectory from u0 (K = 10 is the workload's
ten implicit steps); W warm-up steps solve step 1 and are discarded.

Headline form: mixed precision (FP32 JVP sweeps and Krylov basis, FP64 Newton
residual, update, line search and Hessenberg). The plain per-solve FP64 AD
form is measured in the same run for comparison. All compute runs in
libjfnk's CUDA kernels through its C ABI; this script only allocates device
memory, times, and prints one JSON line.

Also reported: per-step p50/p99 latency, Newton/Krylov counts, the
dominant kernel's achieved HBM bandwidth against the measured peak, the
end-to-end rate through the C ABI with host buffers, the CPU oracle timed on
a bounded sample (--impl reference runs only that), and SM clocks sampled
during the timed region.

Multi-GPU (torchrun): the path does not shard; every rank solves its own
replica of the workload (weak scaling), value = all ranks' solves / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import re

import numpy as np
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Newton solves/s and JVP HBM GB/s (% peak): served FP32 vs plain FP64; p50/p99"
N_GRID = 2048
D_COEF, DT, THETA, SEED = 1e-3, 0.1, 0.5, 0
RESTART = 40
TOL_NEWTON = 1e-8
TOL_KRYLOV = {"mixed": 1e-6, "fp64": 1e-8}
WORKLOAD = "allen_cahn_2048x2048_cn_dt0.1_D1e-3_seed0"
GOLDEN = os.path.join(ROOT, "tests", "golden", "allen_cahn_2048_step1.json")
TRAFFIC = os.path.join(ROOT, "profiles", "ncu_traffic.json")
# FP64 on this part: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz = 1.26 TFLOP/s (nominal 1.25; a
# dependent-FMA probe measured 1.205). Flops per algorithmic byte of the FP64 kernel classes: one FMA per
# 8-byte basis element in the dots and update-norm passes, two in the update-and-dots pass (its second
# basis sweep comes from L2), and the AD JVP's dual-number stencil (~25 flops per 24-byte cell).
FP64_PEAK_GFLOPS = 1250.0
FP64_FLOP_PER_BYTE = {"arnoldi_dots": 0.25, "arnoldi_update_dots": 0.5, "arnoldi_update_norm_givens": 0.25,
                      "arnoldi_dcgs_dots": 0.25, "arnoldi_dcgs_update": 0.25, "gmres_backsolve_update": 0.25,
                      "jvp_ad": 25.0 / 24.0}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--ortho", default="dcgs2", choices=["cgs2", "dcgs2"],
                    help="GMRES Arnoldi form of the timed run (the other form is timed beside it)")
    ap.add_argument("--no-other-ortho", action="store_true", help="skip the run with the other Arnoldi form")
    ap.add_argument("--cpu-sample-iters", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-serve", action="store_true", help="skip the served request stream")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--configs", action="store_true",
                    help="instead of the timed benchmark: Newton/Krylov counts and completion per configuration, "
                         "AD vs FD, one JSON line")
    ap.add_argument("--config-seeds", type=int, default=32, help="Allen-Cahn seeds for the completion rate")
    ap.add_argument("--suite", choices=["burgers2d", "rd"], default=None,
                    help="one of the paper's benchmark suites instead of the benchmark: 2D Burgers (TGV, DSL, "
                         "4VC x nu x grid) or reaction-diffusion with Dirichlet walls (Gaussian, multi-Gaussian, "
                         "sinusoidal x D x grid), over the solver variants, with Dolan-More performance profiles")
    ap.add_argument("--suite-steps", type=int, default=100, help="implicit steps per suite run")
    ap.add_argument("--suite-grids", default="256,512", help="grid sizes of the suite")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------------
# CPU oracle sample (run in a child process, single-threaded BLAS)
# ------------------------------------------------------------------------------------------------
_CPU_SAMPLE = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import synthetic_inputs as si
from oracle import jvp as ojvp, krylov as okr, pdes as opdes
n, iters = {n}, {iters}
p = opdes.AllenCahn2D(nx=n, ny=n, D={D}, dt={dt}, theta={theta})
u0 = si.allen_cahn_ic(n, n, {seed})
b = p.rhs(u0)
t = time.perf_counter(); F = p.residual(u0, b); t_res = time.perf_counter() - t
A = lambda v: ojvp.jvp_complex_step(lambda z: p.residual(z, b), u0, v)[1]
t = time.perf_counter(); okr.gmres(A, -F, iters, 0.0, 1); t_gm = time.perf_counter() - t
print(json.dumps({{"t_res": t_res, "t_iter": t_gm / iters, "iters": iters}}))
"""


_ORACLE_ENV = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                   CUDA_VISIBLE_DEVICES="")


def cpu_oracle_sample(iters: int) -> dict:
    code = _CPU_SAMPLE.format(root=ROOT, n=N_GRID, iters=iters, D=D_COEF, dt=DT, theta=THETA, seed=SEED)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=_ORACLE_ENV, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=30).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    return "unknown"


def _projected(g: dict, s: dict) -> float:
    """Seconds of one oracle solve of the benchmark step: its own Krylov and residual counts times the
    timed cost of one Arnoldi step and one residual."""
    return g["krylov_its"] * s["t_iter"] + (1 + g["newton_its"] + g["ls_backtracks"]) * s["t_res"]


def cpu_all_cores(iters: int) -> dict:
    """The same bounded sample run as one independent single-threaded oracle process per host core, all at
    once: solves/s of the whole host (cores x each process's projected rate)."""
    cores = os.cpu_count() or 1
    code = _CPU_SAMPLE.format(root=ROOT, n=N_GRID, iters=iters, D=D_COEF, dt=DT, theta=THETA, seed=SEED)
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=_ORACLE_ENV) for _ in range(cores)]
    g = json.load(open(GOLDEN))
    rates = []
    for p in procs:
        out, err = p.communicate(timeout=900)
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        rates.append(1.0 / _projected(g, json.loads(out.strip().splitlines()[-1])))
    return {"value": sum(rates), "unit": "solves/s", "cores": cores, "cpu": cpu_model(),
            "sample": f"{cores} independent single-threaded oracle processes at once, each projected from "
                      f"{iters} timed Arnoldi steps and one residual as below"}


def cpu_baseline(iters: int, all_cores: bool = True) -> dict:
    """Oracle solves/s on this host, projected from a bounded sample by the oracle's own counts."""
    if not os.path.exists(GOLDEN):
        return {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle",
                "sample": "unavailable: tests/golden/allen_cahn_2048_step1.json missing"}
    g = json.load(open(GOLDEN))
    s = cpu_oracle_sample(iters)
    n_res = 1 + g["newton_its"] + g["ls_backtracks"]
    sec = _projected(g, s)
    out = {"value": 1.0 / sec, "unit": "solves/s", "cores": 1, "kind": "oracle", "projected": True,
           "cpu": cpu_model(),
           "sample": (f"projected: numpy FP64 oracle, 1 thread, {iters} GMRES(40) Arnoldi steps with complex-step "
                      f"JVPs and one residual timed on the 2048^2 step-1 system ({s['t_iter']:.3f} s/step, "
                      f"{s['t_res']:.3f} s/residual), scaled by the oracle's own counts for that solve "
                      f"({g['krylov_its']} Krylov steps, {n_res} residuals)"),
           "seconds_per_solve": sec}
    if all_cores:
        out["all_cores"] = cpu_all_cores(iters)
    return out


# ------------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [ln.split(",") for ln in self.f.read().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


class Replicas:
    """Multi-GPU runs of the benchmark: the path does not shard, so every rank solves its own replica of the
    workload (weak scaling). The ranks meet at a barrier around the timed region, the job time is the
    maximum of the ranks' times, and the whole-job rate is all ranks' solves over that time. `dist` is
    torch.distributed after init_process_group (None: one process); `device` holds the reduction tensor
    ("cuda" for NCCL, "cpu" for gloo)."""

    def __init__(self, dist=None, device: str = "cpu"):
        self.dist, self.device = dist, device

    @property
    def world(self) -> int:
        return self.dist.get_world_size() if self.dist is not None else 1

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def max(self, v: float) -> float:
        if self.dist is None:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def rate(self, solves_per_rank: int, max_seconds: float) -> float:
        return self.world * solves_per_rank / max_seconds


def _strip_comments(src: str) -> str:
    """C/C++/CUDA source without comments, runs of white space outside literals collapsed to one space:
    what the compiler sees of it. String and character literals are kept byte for byte."""
    out, code, i, n = [], [], 0, len(src)

    def flush():
        if code:
            out.append(re.sub(r"\s+", " ", "".join(code)))
            code.clear()

    while i < n:
        c = src[i]
        if c in "\"'":                       # string or character literal, kept whole
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            flush()
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            code.append(" ")
        else:
            code.append(c)
            i += 1
    flush()
    return "".join(out).strip()


def _src_hash() -> str:
    """Hash of the CUDA sources as compiled (comments and spacing left out) and of the nvcc architecture and
    flags they are built with, so that stored ncu counters stay tied to the kernels they were taken from."""
    from paper_2605_13378_gb300 import build as B
    h = hashlib.sha256()
    h.update(" ".join(B.ARCH + [f for f in B.FLAGS if not f.startswith("-I")]).encode() + b"\0")
    csrc = os.path.join(ROOT, "paper_2605_13378_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(f.encode() + b"\0")
        h.update(_strip_comments(open(os.path.join(csrc, f), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


# Per-PDE solver settings of the served stream: GMRES restart, Newton iterations, restart cycles. The
# Allen-Cahn step converges well inside its caps; restarted GMRES without a preconditioner does not converge
# on the radiation and the scalar Maxwell configurations at most grids (see the configuration sweep), so
# their caps bound the work of a request and such requests are reported as not completed.
SERVE_CAPS = {"allen_cahn": (40, 15, 100), "su_olson": (30, 6, 20), "maxwell": (60, 3, 10)}


def served_stream(J, device: int, n_req: int) -> dict:
    """The serving workload: Poisson arrivals (6/s) of solves drawn from the three 2D problems (Allen-Cahn,
    the radiation problem at dt = 1e-3, scalar TE Maxwell at ten points per wavelength) at grids log-uniform
    in 64..2048, 1..20 implicit steps (the Maxwell problem: one nonlinear solve from its Born start), precision
    mixed FP32 or FP64 per request (synthetic_inputs.serving_requests), through jfnk_submit / jfnk_poll,
    against the same requests solved one at a time in plain FP64. Both sides solve to tol_Newton 1e-10.
    A request completes when every step meets the Newton test; the accuracy is the largest difference,
    relative to max |x|, between a served result and its FP64 result over the requests both completed."""
    import synthetic_inputs as si
    reqs = si.serving_requests(n_req, rate=6.0, seed=7)
    keep = []   # host arrays borrowed by the problems until their requests have started

    def build(r, prec):
        n = r["n"]
        m, max_newton, max_cycles = SERVE_CAPS[r["pde"]]
        if r["pde"] == "allen_cahn":
            p = J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))
            x0 = si.allen_cahn_ic(n, n, r["seed"] % 1000)
        elif r["pde"] == "su_olson":
            p = J.make_problem("su_olson", n, n, 1e-3, 0.5, (1.0, 1.0, 1.0, 1e-6, 1.0))
            x0 = si.su_olson_ic(n, n)
        else:
            eps, f = si.maxwell_medium(n, n, r["seed"] % 1000), si.maxwell_point_source(n, n)
            keep.append((eps, f))
            p = J.make_problem("maxwell", n, n, 0.0, 1.0, (si.maxwell_wavenumber(n), 1e-3), eps_r=eps, source=f)
            x0 = np.zeros(2 * n * n)
        o = J.jfnk_default_opts(prec)
        o.restart, o.max_newton, o.max_krylov = m, max_newton, max_cycles
        o.tol_newton = 1e-10
        o.tol_krylov = 1e-6 if prec == J.JFNK_MIXED_FP32 else 1e-10
        # mixed requests use delayed CGS2: in the batch engine (small requests, any size) and on the slot
        # workers (large ones, whose streaming passes need a size divisible by 8); FP64 requests the plain CGS2
        big = x0.size > (1 << 20)
        dc = prec == J.JFNK_MIXED_FP32 and (not big or x0.size % 8 == 0)
        o.ortho = J.JFNK_DCGS2 if dc else J.JFNK_CGS2
        return p, o, x0

    solves = lambda r: 1 if r["pde"] == "maxwell" else r["steps"]
    ctx = J.jfnk_create(device)
    try:
        outs, tickets = [], []
        t0 = time.perf_counter()
        for r in reqs:
            while time.perf_counter() - t0 < r["t_arrival"]:
                time.sleep(0.0005)
            prec = J.JFNK_MIXED_FP32 if r["precision"] == "mixed" else J.JFNK_FP64
            p, o, x0 = build(r, prec)
            xo = np.zeros_like(x0)
            s, t = J.jfnk_submit(ctx, p, o, x0, xo, r["steps"])
            if s != J.JFNK_OK:
                raise RuntimeError("submit: " + J.jfnk_status_string(s))
            keep.append(x0)   # borrowed by the server until the request completes
            outs.append(xo)
            tickets.append(t)
        served = {}
        pending = dict(enumerate(tickets))
        while pending:
            for i, t in list(pending.items()):
                rep = J.jfnk_report()
                s = J.jfnk_poll(ctx, t, rep)
                if s != J.JFNK_E_BUSY:
                    served[i] = (s, rep.ms, s == J.JFNK_OK and rep.steps_failed == 0, time.perf_counter() - t0)
                    del pending[i]
            time.sleep(0.0005)
        wall = time.perf_counter() - t0
    finally:
        J.jfnk_destroy(ctx)
    # requests that ended in an error (not a missed tolerance): index, class, grid, status, completion time
    errors = [{"request": i, "pde": reqs[i]["pde"], "n": reqs[i]["n"], "precision": reqs[i]["precision"],
               "status": J.jfnk_status_string(served[i][0]), "t_done_s": round(served[i][3], 3)}
              for i in sorted(served) if served[i][0] not in (J.JFNK_OK, J.JFNK_E_NOT_CONVERGED)]
    if errors:
        return {"requests": len(reqs), "error": "served requests failed", "failed": errors}
    # the same requests, one at a time, plain FP64
    c1 = J.jfnk_create(device)
    x64, ok64 = [], []
    try:
        t1 = time.perf_counter()
        for r in reqs:
            p, o, x0 = build(r, J.JFNK_FP64)
            J.check(c1, J.jfnk_set_problem(c1, p), "set_problem")
            xa = x0.copy()
            rep = J.jfnk_report()
            s = J.jfnk_solve(c1, o, None, xa, r["steps"], rep)
            x64.append(xa)
            ok64.append(s == J.JFNK_OK and rep.steps_failed == 0)
        one = time.perf_counter() - t1
    finally:
        J.jfnk_destroy(c1)
    total = sum(solves(r) for r in reqs)
    pct = lambda v, q: sorted(v)[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))]
    classes = {}
    for i, r in enumerate(reqs):
        c = classes.setdefault(r["pde"], {"requests": 0, "completed": 0, "fp64_completed": 0, "lat": []})
        c["requests"] += 1
        c["completed"] += int(served[i][2])
        c["fp64_completed"] += int(ok64[i])
        c["lat"].append(served[i][1])
    per_class = {k: {"requests": c["requests"], "completed": c["completed"], "fp64_completed": c["fp64_completed"],
                     "p50_ms": pct(c["lat"], 0.5), "p99_ms": pct(c["lat"], 0.99)} for k, c in classes.items()}
    lat = [served[i][1] for i in range(len(reqs))]
    both = [i for i in range(len(reqs)) if served[i][2] and ok64[i]]
    rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    return {"requests": len(reqs), "solves": total, "value": total / wall, "unit": "solves/s",
            "completed": sum(1 for i in served if served[i][2]),
            "completed_solves_per_s": sum(solves(reqs[i]) for i in served if served[i][2]) / wall,
            "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99), "per_pde": per_class,
            "max_rel_diff_vs_fp64": max((rel(outs[i], x64[i]) for i in both), default=None),
            "compared_requests": len(both),
            "fp64_one_by_one": {"value": total / one, "unit": "solves/s", "completed": sum(ok64),
                                "completed_solves_per_s": sum(solves(reqs[i]) for i in range(len(reqs)) if ok64[i]) / one},
            "stream": ("Poisson 6/s, Allen-Cahn / radiation (dt 1e-3) / scalar Maxwell (10 points per wavelength), "
                       "grids log-uniform 64..2048, 1..20 steps, precision mixed|fp64, tol_Newton 1e-10; caps "
                       "(restart, Newton, cycles): " + ", ".join(f"{k} {v}" for k, v in SERVE_CAPS.items()))}


def config_sweep(a) -> None:
    """Newton/Krylov counts and completion per benchmark configuration, AD against FD.

    A run completes when every implicit step (or the nonlinear solve) ends with the Newton test met
    (status OK). Counts are per Newton step (Krylov) and per implicit step (Newton).
    """
    import torch
    import synthetic_inputs as si
    from paper_2605_13378_gb300 import jfnk as J
    torch.cuda.set_device(0)
    ctx = J.jfnk_create(0)
    out = {"mode": "configs", "data": "synthetic", "results": []}

    def opts(prec, lin, krylov="gmres", restart=40, tol_n=None, tol_k=None, max_newton=15, max_krylov=100,
             ortho="cgs2"):
        o = J.jfnk_default_opts(prec)
        o.lin = J.JFNK_AD if lin == "ad" else J.JFNK_FD
        o.krylov = J.JFNK_GMRES if krylov == "gmres" else J.JFNK_BICGSTAB
        o.restart, o.max_newton, o.max_krylov = restart, max_newton, max_krylov
        if tol_n is not None:
            o.tol_newton = tol_n
        if tol_k is not None:
            o.tol_krylov = tol_k
        o.ortho = J.JFNK_DCGS2 if ortho == "dcgs2" else J.JFNK_CGS2
        return o

    fatal = {J.JFNK_E_NONFINITE: "non-finite values", J.JFNK_E_BREAKDOWN: "Krylov breakdown"}

    def failure(r, s, steps):
        """Which of the paper's failure criteria (Sec. 3.4) a run meets, or None when it completed."""
        if s == J.JFNK_OK and r.steps_failed == 0:
            return None
        if s in fatal:
            return fatal[s]
        if r.steps_failed > 0.2 * steps:
            return f"{r.steps_failed} of {steps} steps missed 100 x tol_Newton"
        return J.jfnk_status_string(s)

    def summary(name, reps, sts, steps, t):
        done = [r for r, s in zip(reps, sts) if s == J.JFNK_OK and r.steps_failed == 0]
        newton = sum(r.newton_its for r in reps)
        krylov = sum(r.krylov_its for r in reps)
        fails = sorted({f for f in (failure(r, s, steps) for r, s in zip(reps, sts)) if f})
        return {"config": name, "runs": len(reps), "completed": len(done), "completion": len(done) / len(reps),
                "newton_per_step": newton / max(1, steps * len(reps)), "krylov_per_newton": krylov / max(1, newton),
                "ls_backtracks": sum(r.ls_backtracks for r in reps), "krylov_failures": sum(r.krylov_failures for r in reps),
                "res_final_over_res0": [r.res_final / r.res0 if r.res0 else 0.0 for r in reps][:4],
                "failure": fails, "statuses": sorted({J.jfnk_status_string(s) for s in sts}), "seconds": round(t, 3)}

    def solve_one(lp, o, x0, steps):
        J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
        x = torch.tensor(x0, device="cuda")
        rep = J.jfnk_report()
        s = J.jfnk_solve(ctx, o, None, x, steps, rep)
        return rep, s

    # 1D Burgers, one backward-Euler step, FP64, GMRES(30), tol 1e-10
    lp = J.make_problem("burgers1d", 1024, 1, 1e-3, 1.0, (1e-2,))
    for lin in ("ad", "fd"):
        t0 = time.perf_counter()
        rep, s = solve_one(lp, opts(J.JFNK_FP64, lin, restart=30, tol_n=1e-10, tol_k=1e-10), si.burgers_ic(1024, 0), 1)
        out["results"].append(summary(f"burgers 1024 fp64 gmres(30) {lin}", [rep], [s], 1, time.perf_counter() - t0))
    # Allen-Cahn 512^2, 10 steps, seeds 0..S-1: {FP64, FP32} x {AD, FD} x {GMRES(40), BiCGSTAB}
    n, steps = 512, 10
    lp = J.make_problem("allen_cahn", n, n, 0.1, 0.5, (1e-3, 1.0))
    seeds = list(range(a.config_seeds))
    for prec_name, prec in (("fp64", J.JFNK_FP64), ("fp32", J.JFNK_FP32)):
        for lin in ("ad", "fd"):
            for kr in ("gmres", "bicgstab"):
                o = opts(prec, lin, kr)
                t0 = time.perf_counter()
                if kr == "gmres":     # all seeds in one batched call
                    xs = [torch.tensor(si.allen_cahn_ic(n, n, sd), device="cuda") for sd in seeds]
                    _, reps, sts = J.jfnk_solve_batch(ctx, [lp] * len(seeds), o, None, xs, steps)
                else:
                    reps, sts = [], []
                    for sd in seeds:
                        rep, s = solve_one(lp, o, si.allen_cahn_ic(n, n, sd), steps)
                        reps.append(rep)
                        sts.append(s)
                torch.cuda.synchronize()
                out["results"].append(summary(f"allen_cahn 512^2 x{steps} steps {prec_name} {kr} {lin}", reps, sts,
                                              steps, time.perf_counter() - t0))
    # radiation 1024^2, dt in {1e-3, 1e-1}, mixed, GMRES(30) with the paper's cap of 100 restart cycles, one step
    n = 1024
    for dt in (1e-3, 1e-1):
        lp = J.make_problem("su_olson", n, n, dt, 0.5, (1.0, 1.0, 1.0, 1e-6, 1.0))
        for lin in ("ad", "fd"):
            t0 = time.perf_counter()
            rep, s = solve_one(lp, opts(J.JFNK_MIXED_FP32, lin, restart=30, tol_n=1e-8, tol_k=1e-6, max_krylov=100,
                                        ortho="dcgs2"), si.su_olson_ic(n, n), 1)
            out["results"].append(summary(f"radiation 1024^2 dt={dt:g} mixed gmres(30) x100 cycles {lin}", [rep], [s],
                                          1, time.perf_counter() - t0))
    # Maxwell 1024^2 at ten points per wavelength, chi3 in {1e-3, 1e-1}, GMRES(60) with an FP32 basis,
    # Born start, no preconditioner: bounded (the configuration needs the paper's preconditioner)
    k = si.maxwell_wavenumber(n)
    eps, f = si.maxwell_medium(n, n, 0), si.maxwell_point_source(n, n)
    for chi in (1e-3, 1e-1):
        lp = J.make_problem("maxwell", n, n, 0.0, 1.0, (k, chi), eps_r=eps, source=f)
        for lin in ("ad", "fd"):
            t0 = time.perf_counter()
            rep, s = solve_one(lp, opts(J.JFNK_MIXED_FP32, lin, restart=60, tol_n=1e-8, tol_k=1e-6, max_newton=3,
                                        max_krylov=10, ortho="dcgs2"), np.zeros(2 * n * n), 1)
            out["results"].append(summary(f"maxwell 1024^2 k={k:.0f} chi3={chi:g} mixed gmres(60) {lin}", [rep], [s],
                                          1, time.perf_counter() - t0))
    # the paper's vector TE Maxwell problem in its PEC cavity: 512^2 nodes, symmetric Gaussian current,
    # w = 18, chi = 0.05, Born start, GMRES(60) in FP64, with and without the CSLP preconditioner (bounded)
    n = 512
    jc = si.maxwell_vec_source(n, n, "gauss")
    lp = J.make_problem("maxwell_vec", n, n, 0.0, 1.0, (18.0, 0.05, 0.05), source=jc)
    for lin in ("ad", "fd"):
        for pre in ("none", "cslp"):
            o = opts(J.JFNK_FP64, lin, restart=60, tol_n=1e-6, tol_k=1e-8, max_newton=15, max_krylov=20, ortho="dcgs2")
            o.precond = J.JFNK_PRECOND_CSLP if pre == "cslp" else J.JFNK_PRECOND_NONE
            t0 = time.perf_counter()
            rep, s = solve_one(lp, o, np.zeros(4 * n * n), 1)
            out["results"].append(summary(f"maxwell_vec 512^2 w=18 chi=0.05 fp64 gmres(60)x20 {pre} {lin}", [rep],
                                          [s], 1, time.perf_counter() - t0))
    J.jfnk_destroy(ctx)
    print(json.dumps(out))


SUITE_VARIANTS = [(prec, lin, kr) for prec in ("fp64", "fp32") for lin in ("ad", "fd") for kr in ("gmres", "bicgstab")]
# the reaction-diffusion Jacobian is SPD, so CG joins the comparison
SUITE_VARIANTS_SPD = [(prec, lin, kr) for prec in ("fp64", "fp32") for lin in ("ad", "fd")
                      for kr in ("gmres", "bicgstab", "cg")]
PROFILE_TAUS = (1.0, 1.5, 2.0, 4.0, 8.0, 16.0, 32.0, 64.0, 128.0, 1024.0)


def run_failed(status_ok: bool, fatal: bool, steps: int, steps_failed: int) -> bool:
    """The paper's failure rule for a time-dependent run (Sec. 4, metrics and failure criteria): it fails when
    it stops early (non-finite values, breakdown, a library error) or when more than 20% of its implicit steps
    miss 100 x tol_Newton."""
    if fatal:
        return True
    return steps_failed > 0.2 * steps


def performance_profile(times: dict, taus=PROFILE_TAUS) -> dict:
    """Dolan-More profiles: times[solver][problem] = metric, None for a failed run.

    r_ps = t_ps / min_s t_ps over the solvers that completed p (a failed run has r = inf);
    rho_s(tau) = |{p : r_ps <= tau}| / |P|. Problems no solver completed count in |P| for every solver."""
    solvers = sorted(times)
    problems = sorted({p for s in solvers for p in times[s]})
    best = {}
    for p in problems:
        ok = [times[s][p] for s in solvers if times[s].get(p) is not None]
        best[p] = min(ok) if ok else None
    out = {}
    for s in solvers:
        r = []
        for p in problems:
            t = times[s].get(p)
            r.append(math.inf if (t is None or best[p] is None) else t / best[p])
        out[s] = {"rho": [sum(1 for x in r if x <= tau) / len(problems) for tau in taus],
                  "completion": sum(1 for x in r if x < math.inf) / len(problems)}
    return {"taus": list(taus), "problems": len(problems), "profiles": out}


def paper_suite(a) -> None:
    """One of the paper's benchmark suites (App. A; Sec. 4 setup) at Courant number 1, Crank-Nicolson, each
    run one jfnk_solve of --suite-steps implicit steps with the paper's tolerances and caps (FP64 1e-6 / 1e-8,
    FP32 1e-4 / 1e-6, 15 Newton iterations, 100 Krylov cycles or iterations, GMRES(30)); Dolan-More profiles
    by wall time and by Krylov iterations.

    burgers2d: TGV, DSL and 4VC at nu in {0.1, 0.05, 0.01}, adaptive CFL step, {FP64, FP32} x {AD, FD} x
    {GMRES, BiCGSTAB}. rd: u_t = D lap u - u^3 with Dirichlet walls, Gaussian, multi-Gaussian and sinusoidal
    data at D in {0.1, 0.01, 0.001}, dt = dx^2 / D, the same variants and CG."""
    import torch
    import synthetic_inputs as si
    from paper_2605_13378_gb300 import jfnk as J
    torch.cuda.set_device(0)
    ctx = J.jfnk_create(0)
    grids = [int(g) for g in a.suite_grids.split(",") if g]
    steps = a.suite_steps
    fatal_codes = {J.JFNK_E_NONFINITE, J.JFNK_E_BREAKDOWN, J.JFNK_E_CUDA, J.JFNK_E_TIMEOUT, J.JFNK_E_OOM,
                   J.JFNK_E_INVALID}
    kr_code = {"gmres": J.JFNK_GMRES, "bicgstab": J.JFNK_BICGSTAB, "cg": J.JFNK_CG}
    kr_name = {"gmres": "GMRES", "bicgstab": "BiCGSTAB", "cg": "CG"}
    if a.suite == "burgers2d":
        kinds, params, variants = si.BURGERS2D_KINDS, (0.1, 0.05, 0.01), SUITE_VARIANTS

        def problem(n, kind, nu):
            return (f"{kind} nu={nu:g} {n}^2", J.make_problem("burgers2d", n, n, 0.0, 0.5, (nu, 0.0, 1.0)),
                    si.burgers2d_ic(n, n, kind))
    else:
        kinds, params, variants = si.RD_KINDS, (0.1, 0.01, 0.001), SUITE_VARIANTS_SPD

        def problem(n, kind, D):
            dt = (1.0 / (n + 1)) ** 2 / D
            return (f"{kind} D={D:g} {n}^2", J.make_problem("allen_cahn", n, n, dt, 0.5, (D, 0.0, 1.0)),
                    si.rd_ic(n, n, kind))
    runs, t_wall, t_kry = [], {}, {}
    for n in grids:
        for kind in kinds:
            for par in params:
                prob, lp, x0 = problem(n, kind, par)
                J.check(ctx, J.jfnk_set_problem(ctx, lp), "set_problem")
                for prec, lin, kr in variants:
                    o = J.jfnk_default_opts(J.JFNK_FP64 if prec == "fp64" else J.JFNK_FP32)
                    o.lin = J.JFNK_AD if lin == "ad" else J.JFNK_FD
                    o.krylov = kr_code[kr]
                    o.restart = 30
                    x = torch.tensor(x0, device="cuda")
                    rep = J.jfnk_report()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    s = J.jfnk_solve(ctx, o, None, x, steps, rep)
                    torch.cuda.synchronize()
                    dt_wall = time.perf_counter() - t0
                    failed = run_failed(s == J.JFNK_OK, s in fatal_codes, steps, rep.steps_failed)
                    var = f"{lin.upper()}-{prec.upper()}-{kr_name[kr]}"
                    t_wall.setdefault(var, {})[prob] = None if failed else dt_wall
                    t_kry.setdefault(var, {})[prob] = None if failed else max(1, rep.krylov_its)
                    runs.append({"problem": prob, "solver": var, "status": J.jfnk_status_string(s),
                                 "failed": failed, "seconds": round(dt_wall, 4), "steps_done": rep.steps_done,
                                 "steps_failed": rep.steps_failed, "newton": rep.newton_its, "krylov": rep.krylov_its,
                                 "ls_backtracks": rep.ls_backtracks, "dt_last": rep.dt_last})
    J.jfnk_destroy(ctx)
    out = {"mode": "suite", "pde": a.suite, "data": "synthetic", "steps": steps, "grids": grids,
           "courant": 1.0, "restart": 30, "runs": runs,
           "profile_wall_time": performance_profile(t_wall), "profile_krylov_its": performance_profile(t_kry)}
    print(json.dumps(out))


def run_reference(a) -> None:
    """The oracle as it stands on this host's cores, one bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(a.warmup):
        cpu_oracle_sample(2)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(a.steps):
        last = cpu_baseline(2, all_cores=False)
        vals.append(last["seconds_per_solve"] if last["value"] else float("nan"))
    wall = time.perf_counter() - t0
    sec = sum(vals) / len(vals)
    value = 1.0 / sec if sec == sec else None
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "solver": "Newton + GMRES(40), AD (complex step), FP64 oracle"},
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "projected": True,
                            "sample": last["sample"] if last else None},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": wall}
    print(json.dumps(out))


def main() -> None:
    a = _args()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.suite:
        paper_suite(a)
        return
    if a.configs:
        config_sweep(a)
        return
    import torch

    import synthetic_inputs as si
    from paper_2605_13378_gb300 import jfnk as J

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    replicas = Replicas(dist, "cuda")

    def barrier():
        replicas.barrier()
        torch.cuda.synchronize()

    max_over_ranks = replicas.max

    stream = torch.cuda.Stream()
    ctx = J.jfnk_create(local, 0, stream.cuda_stream)
    J.check(ctx, J.jfnk_set_problem(ctx, J.make_problem("allen_cahn", N_GRID, N_GRID, DT, THETA, (D_COEF, 1.0))),
            "set_problem")
    u0 = si.allen_cahn_ic(N_GRID, N_GRID, SEED)
    u0_dev = torch.tensor(u0, device="cuda")
    x = torch.empty_like(u0_dev)

    def opts(form, ortho=None):
        o = J.jfnk_default_opts(J.JFNK_MIXED_FP32 if form == "mixed" else J.JFNK_FP64)
        o.restart, o.tol_newton, o.tol_krylov = RESTART, TOL_NEWTON, TOL_KRYLOV[form]
        o.max_newton, o.max_krylov = 15, 100
        o.ortho = J.JFNK_DCGS2 if (ortho or a.ortho) == "dcgs2" else J.JFNK_CGS2
        return o

    def run_steps(form, k, timing=False, ortho=None):
        """k trajectory steps from u0; returns (event ms per step, reports, final x)."""
        o = opts(form, ortho)
        J.jfnk_set_timing(ctx, timing)
        x.copy_(u0_dev)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
        reps = []
        barrier()
        with torch.cuda.stream(stream):
            evs[0].record(stream)
            for s in range(k):
                rep = J.jfnk_report()
                st = J.jfnk_solve(ctx, o, None, x, 1, rep)
                if st not in (J.JFNK_OK, J.JFNK_E_NOT_CONVERGED):
                    raise RuntimeError(J.jfnk_status_string(st) + ": " + J.jfnk_last_error(ctx))
                evs[s + 1].record(stream)
                reps.append(rep.as_dict())
        barrier()
        J.jfnk_set_timing(ctx, False)
        return [evs[s].elapsed_time(evs[s + 1]) for s in range(k)], reps, x.clone()

    # warm-up: step 1 solved W times
    o_m = opts("mixed")
    for _ in range(a.warmup):
        x.copy_(u0_dev)
        torch.cuda.synchronize()
        J.check(ctx, J.jfnk_solve(ctx, o_m, None, x, 1, None), "warmup")
    torch.cuda.synchronize()

    # timed region: K steps, device events on the library's stream
    clocks = Clocks(local)
    J.jfnk_reset_stats(ctx)
    ms, reps, x_mixed = run_steps("mixed", a.steps)
    clk = clocks.stop()
    gpu_launches = J.jfnk_kernel_stats(ctx)["all_launches"]["launches"]
    total_ms = max_over_ranks(sum(ms))
    value = world * a.steps / (total_ms / 1e3)
    srt = sorted(ms)
    p50 = srt[len(srt) // 2]
    p99 = srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]

    # per-kernel device times: the same steps again with events around every launch
    J.jfnk_reset_stats(ctx)
    ms_t, _, _ = run_steps("mixed", a.steps, timing=True)
    stats = J.jfnk_kernel_stats(ctx)
    stats.pop("all_launches", None)
    ktot = sum(v["ms"] for v in stats.values())
    kern = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                "share": round(v["ms"] / ktot, 4) if ktot else 0.0,
                "gbs": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] else None}
            for k, v in stats.items() if v["launches"]}
    dom = max(kern, key=lambda k: kern[k]["ms"])
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    ach = kern[dom]["gbs"]
    traffic = None
    if os.path.exists(TRAFFIC):
        tr = json.load(open(TRAFFIC))
        if tr.get("src_hash") == _src_hash() and dom in tr.get("kernels", {}):
            # ncu's DRAM bytes over the algorithmic bytes of the captured launches, scaled to this
            # class's mean algorithmic bytes per launch (launches differ in basis size k)
            traffic = round(tr["kernels"][dom]["dram_over_algorithmic"] * stats[dom]["bytes"] / stats[dom]["launches"])
    roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4) if ach else None, "traffic": traffic,
                "peak_source": "measured" if peaks else "fallback",
                "bytes_per_launch": stats[dom]["bytes"] / stats[dom]["launches"]}
    jv = stats.get("jvp_ad", {"ms": 0})
    jvp_gbs = jv["bytes"] / (jv["ms"] * 1e-3) / 1e9 if jv.get("ms") else None

    # plain per-solve FP64 AD form, same steps, with CGS2 (the faster Arnoldi form in FP64 on this part:
    # the fused dots pass's serial FP64 tail outweighs its saved pass when the streaming itself is FP64)
    fp64 = None
    if not a.no_fp64:
        ms64, reps64, x64 = run_steps("fp64", a.steps, ortho="cgs2")
        fp64 = {"value": world * a.steps / (max_over_ranks(sum(ms64)) / 1e3), "unit": "solves/s", "arnoldi": "cgs2",
                "ms_per_step": sum(ms64) / a.steps, "p50_ms": sorted(ms64)[len(ms64) // 2],
                "newton_its": sum(r["newton_its"] for r in reps64),
                "krylov_its": sum(r["krylov_its"] for r in reps64),
                "max_rel_diff_mixed_vs_fp64": float((x_mixed - x64).abs().max() / x64.abs().max())}
        # its dominant kernel against min(HBM, FP64 pipe): three steps again with events around every launch
        J.jfnk_reset_stats(ctx)
        run_steps("fp64", min(a.steps, 3), timing=True, ortho="cgs2")
        st64 = {k: v for k, v in J.jfnk_kernel_stats(ctx).items() if k != "all_launches" and v["launches"]}
        d64 = max(st64, key=lambda k: st64[k]["ms"])
        gbs = st64[d64]["bytes"] / (st64[d64]["ms"] * 1e-3) / 1e9
        fpb = FP64_FLOP_PER_BYTE.get(d64)
        if fpb is not None:
            alu_gbs = FP64_PEAK_GFLOPS / fpb
            fp64["roofline"] = {
                "bound": "alu" if alu_gbs < peak else "hbm", "kernel": d64,
                "share": round(st64[d64]["ms"] / sum(v["ms"] for v in st64.values()), 4),
                "achieved": round(gbs * fpb, 1), "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": round(gbs * fpb / FP64_PEAK_GFLOPS, 4), "flop_per_byte": fpb,
                "achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / peak, 4),
                "peak_source": "nominal FP64 of this part (152 SMs x 4 flop/clk x 2.07 GHz)"}

    # the same steps with the other Arnoldi form
    other = None
    if not a.no_other_ortho:
        oth = "cgs2" if a.ortho == "dcgs2" else "dcgs2"
        ms_o, reps_o, x_o = run_steps("mixed", a.steps, ortho=oth)
        other = {"arnoldi": oth, "value": world * a.steps / (max_over_ranks(sum(ms_o)) / 1e3), "unit": "solves/s",
                 "ms_per_step": sum(ms_o) / a.steps,
                 "newton_its": sum(r["newton_its"] for r in reps_o),
                 "krylov_its": sum(r["krylov_its"] for r in reps_o),
                 "max_rel_diff_vs_timed": float((x_mixed - x_o).abs().max() / x_o.abs().max())}

    # end to end through the C ABI with host buffers: H2D of each step's input, D2H of its result
    e2e = None
    if not a.no_e2e:
        pin_in = torch.empty(u0.size, dtype=torch.float64, pin_memory=True)
        pin_out = torch.empty_like(pin_in)
        pin_in.copy_(torch.from_numpy(u0))
        J.check(ctx, J.jfnk_solve(ctx, o_m, pin_in, pin_out, 1, None), "e2e warmup")
        barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            J.check(ctx, J.jfnk_solve(ctx, o_m, pin_in, pin_out, 1, None), "e2e")
            pin_in.copy_(pin_out)
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": world * a.steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": u0.size * 8,
               "d2h_bytes_per_step": u0.size * 8}

    cpu = cpu_baseline(a.cpu_sample_iters) if (rank == 0 and world == 1 and not a.no_cpu) else None
    J.jfnk_destroy(ctx)
    served = None
    if not a.no_serve:
        try:
            served = served_stream(J, local, a.serve_requests)
        except Exception as e:   # reported in the line; the measurements above stand
            served = {"error": f"{type(e).__name__}: {e}"}
    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [N_GRID, N_GRID], "steps_per_run": a.steps,
                   "form": "mixed: FP32 AD JVP + FP32 GMRES(40) basis, FP64 Newton residual/update/line search/"
                           "Hessenberg", "tol_newton": TOL_NEWTON, "tol_krylov": TOL_KRYLOV["mixed"],
                   "arnoldi": (a.ortho + "-fused") if "arnoldi_dcgs_fused" in kern else a.ortho,
                   "l2": "inputs larger than L2 (GMRES basis 656 MB, state 32 MB per vector)",
                   "parallelism": f"replicas x{world}"},
        "p50_ms": p50, "p99_ms": p99,
        "newton_its": sum(r["newton_its"] for r in reps), "krylov_its": sum(r["krylov_its"] for r in reps),
        "jvp_gbs": jvp_gbs, "jvp_frac": (jvp_gbs / peak) if jvp_gbs else None,
        "fp64_plain": fp64, "other_arnoldi": other, "roofline": roofline, "kernels": kern, "gpu_launches": gpu_launches,
        "timed_with_kernel_events_ms_per_step": sum(ms_t) / a.steps,
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clk, "served": served,
    }
    if served and "error" not in served:
        f = served["fp64_one_by_one"]
        out["served_fp32_vs_fp64"] = {
            "served_solves_per_s": served["value"], "fp64_one_by_one_solves_per_s": f["value"],
            "speedup": served["value"] / f["value"] if f["value"] else None,
            "served_completed_solves_per_s": served["completed_solves_per_s"],
            "fp64_completed_solves_per_s": f["completed_solves_per_s"],
            "max_rel_diff_vs_fp64": served["max_rel_diff_vs_fp64"], "compared_requests": served["compared_requests"],
            "p50_ms": served["p50_ms"], "p99_ms": served["p99_ms"]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
