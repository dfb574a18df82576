"""The C-ABI library builds, loads and exports every entry point of include/jfnk.h (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jfnk.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\*]+\s+)+\**(jfnk_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_13378_gb300 import build
    build.build()
    from paper_2605_13378_gb300 import jfnk
    return jfnk


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["jfnk_create", "jfnk_set_problem", "jfnk_jvp", "jfnk_solve", "jfnk_submit", "jfnk_poll",
              "jfnk_last_error", "jfnk_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib.lib, n), n
    assert sorted(lib.EXPORTED) == _declared()


def test_struct_layouts_match_the_header(lib, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "jfnk.h"\nint main(void){printf("%zu %zu %zu",'
                   'sizeof(jfnk_problem),sizeof(jfnk_opts),sizeof(jfnk_report));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I" + os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    sizes = [int(t) for t in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert sizes == [ctypes.sizeof(lib.jfnk_problem), ctypes.sizeof(lib.jfnk_opts), ctypes.sizeof(lib.jfnk_report)]


def test_constants_match_the_header(lib, tmp_path):
    """Every JFNK_* enumerator and numeric #define of the header has the same value in the binding."""
    txt = open(HEADER).read()
    names = sorted(set(re.findall(r"\b(JFNK_[A-Z0-9_]+)\s*=", txt))
                   | {n for n in re.findall(r"#define\s+(JFNK_[A-Z0-9_]+)\s+\S", txt) if n != "JFNK_H"})
    assert len(names) > 30
    body = "".join(f'printf("{n} %lld\\n", (long long)({n}));' for n in names)
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "jfnk.h"\nint main(void){' + body + "return 0;}\n")
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-I" + os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    vals = dict((ln.split()[0], int(ln.split()[1])) for ln in out if ln)
    assert set(vals) == set(names)
    for n, v in vals.items():
        assert getattr(lib, n) == v, n


def test_host_only_entry_points(lib):
    o = lib.jfnk_default_opts(lib.JFNK_FP64)
    assert (o.tol_newton, o.tol_krylov, o.max_newton, o.max_krylov) == (1e-6, 1e-8, 15, 100)
    o32 = lib.jfnk_default_opts(lib.JFNK_FP32)
    assert (o32.tol_newton, o32.tol_krylov) == (1e-4, 1e-6)
    assert o.ls_min_alpha == 2.0 ** -10 and o.ls_c1 == 1e-4
    assert lib.jfnk_status_string(lib.JFNK_E_BREAKDOWN) == "Krylov breakdown"
    assert lib.lib.jfnk_create(None, 0, 0, None) == lib.JFNK_E_INVALID
    assert lib.lib.jfnk_set_problem(None, None) == lib.JFNK_E_INVALID
    assert lib.lib.jfnk_solve(None, None, None, None, 1, None) == lib.JFNK_E_INVALID
    assert lib.jfnk_tune(None, lib.JFNK_TUNE_BATCH_TILE, 512) == lib.JFNK_E_INVALID


def test_no_cpu_fallback_in_the_product():
    """The package never imports the oracle; the oracle is test infrastructure."""
    pkg = os.path.join(ROOT, "paper_2605_13378_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
