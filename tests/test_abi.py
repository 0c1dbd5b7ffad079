"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/hyel.h declares; the Python binding's struct layouts equal the C
header's (checked by a gcc-compiled layout probe). No GPU is needed."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1809_06350_gb300 import build, hyel

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hyel.h")


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hyel_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_list_agree():
    assert declared_functions() == sorted(hyel.EXPORTS)


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hyel_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_loads_library(libpath):
    assert hyel.lib() is not None


_STRUCTS = {
    "hyel_material": hyel.HyelMaterial,
    "hyel_bc": hyel.HyelBC,
    "hyel_state": hyel.HyelState,
    "hyel_time_params": hyel.HyelTimeParams,
    "hyel_krylov_level": hyel.HyelKrylovLevel,
    "hyel_solver_params": hyel.HyelSolverParams,
    "hyel_solve_stats": hyel.HyelSolveStats,
    "hyel_newton_stats": hyel.HyelNewtonStats,
}


def test_struct_layouts_match_header(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hyel.h"', "int main(void){"]
    for cname, py in _STRUCTS.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split(" ") for line in out if line)
    for cname, py in _STRUCTS.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_create_reports_error_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hyel.HyelError):
        hyel.hyel_create(0, None)
