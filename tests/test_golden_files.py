"""The stored expected values under tests/golden/ are consistent with themselves (CPU only).

They are written by tests/golden/make_golden.py from the oracle alone; these
checks guard against a truncated or hand-edited file.
"""
import json
import os

import pytest

HERE = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    path = os.path.join(HERE, name)
    if not os.path.exists(path):
        pytest.skip(name + " not generated")
    return json.load(open(path))


def test_benchmark_tolerance_solve():
    g = _load("allen_cahn_2048_step1.json")
    assert g["status"] == "converged"
    assert g["res_final"] <= 1e-8 * g["res0"]
    assert g["history"][0] == g["res0"] and g["history"][-1] == g["res_final"]
    assert len(g["history"]) == g["newton_its"] + 1


def _ref_sample_idx(n):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.ref_sample_idx(n)


def test_reference_solve():
    g = _load("allen_cahn_2048_step1_ref.json")
    assert g["status"] == "converged"
    assert g["res_final"] <= 1e-13 * g["res0"]
    assert g["sample_idx"] == _ref_sample_idx(2048)
    assert len(set(i // 2048 for i in g["sample_idx"])) == 2048      # every row sampled
    assert len(g["x_samples"]) == 4096 and len(g["row_sums"]) == 2048
    assert abs(sum(g["row_sums"]) - g["x_sum"]) <= 1e-12 * g["x_absmax"] * 2048 * 2048
    assert max(abs(v) for v in g["x_samples"]) <= g["x_absmax"]
