"""Host logic of the benchmark suite (CPU only): the paper's failure rule and Dolan-More profiles.

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
