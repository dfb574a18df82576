"""Host logic of the benchmark suite (CPU only): the paper's failure rule and Dolan-More profiles,
and the source hash that ties stored ncu counters to the kernels they were taken from.

Sec. 4 (metrics and failure criteria): a time-dependent run fails when it
stops early or when more than 20% of its steps miss 100 x tol_Newton;
r_ps = t_ps / min_s t_ps with failed runs at infinity, and rho_s(tau) is the
fraction of problems with r_ps <= tau. Checked on a hand-made table whose
profile is worked out by hand.
"""
import math

import bench


def test_failure_rule():
    assert not bench.run_failed(True, False, 10, 0)
    assert not bench.run_failed(False, False, 10, 2)       # two of ten steps: tolerated
    assert bench.run_failed(False, False, 10, 3)           # three of ten: more than 20%
    assert bench.run_failed(False, True, 10, 0)            # stopped early (non-finite, breakdown)
    assert not bench.run_failed(False, False, 5, 1) and bench.run_failed(False, False, 4, 1)


def test_performance_profile_by_hand():
    times = {"A": {"p1": 1.0, "p2": 2.0, "p3": None, "p4": None},
             "B": {"p1": 2.0, "p2": 1.0, "p3": 4.0, "p4": None},
             "C": {"p1": None, "p2": None, "p3": None, "p4": None}}
    out = bench.performance_profile(times, taus=(1.0, 2.0, 1e9))
    assert out["problems"] == 4
    pr = out["profiles"]
    # best: p1 = 1 (A), p2 = 1 (B), p3 = 4 (B), p4 unsolved
    assert pr["A"]["rho"] == [0.25, 0.5, 0.5] and pr["A"]["completion"] == 0.5
    assert pr["B"]["rho"] == [0.5, 0.75, 0.75] and pr["B"]["completion"] == 0.75
    assert pr["C"]["rho"] == [0.0, 0.0, 0.0] and pr["C"]["completion"] == 0.0
    # rho is non-decreasing in tau and its plateau is the completion rate
    for s in pr.values():
        assert all(x <= y for x, y in zip(s["rho"], s["rho"][1:]))
        assert math.isclose(s["rho"][-1], s["completion"])


def test_strip_comments_keeps_code_and_literals():
    src = 'int a = 1; // line\n/* block\n  comment */ const char* s = "a//b/*c*/"; char c = \'/\';\n\n  float d;'
    assert bench._strip_comments(src) == 'int a = 1; const char* s = "a//b/*c*/"; char c = \'/\'; float d;'
    assert bench._strip_comments('x = "q\\"//"; // tail') == 'x = "q\\"//";'


def test_src_hash_follows_code_not_comments(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2605_13378_gb300" / "csrc"
    csrc.mkdir(parents=True)
    k = csrc / "k.cu"
    k.write_text("__global__ void k(float* x) { x[0] = 1.0f; }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._src_hash()
    k.write_text("// a kernel\n__global__ void k(float* x) {\n  x[0] = 1.0f;   /* one */\n}\n")
    assert bench._src_hash() == h0
    k.write_text("__global__ void k(float* x) { x[0] = 2.0f; }\n")
    assert bench._src_hash() != h0
    k.write_text("__global__ void k(float* x) { x[0] = 1.0f; }\n")
    (csrc / "extra.cuh").write_text("")
    assert bench._src_hash() != h0          # a new file counts, even an empty one


def test_strip_comments_keeps_literal_spacing():
    assert bench._strip_comments('f("a  b",   1);') == 'f("a  b", 1);'
    assert bench._strip_comments('f("a b", 1);') != bench._strip_comments('f("a  b", 1);')
