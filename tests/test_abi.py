"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/ttq.h declares; the binding's struct layouts match the header (no GPU
needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_1903_11554_gb300 import binding, build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ttq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ttq_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists(build.LIB):
        pytest.skip("no nvcc and no prebuilt library")
    build.build()
    return binding.load()


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("ttq_workspace_bytes", "ttq_plan_create", "ttq_plan_run", "ttq_plan_sweep",
                 "ttq_plan_eval_points", "ttq_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    assert set(binding.SIGNATURES) >= set(declared_functions()) - set()


def test_struct_layouts_match_the_header(tmp_path):
    """Every field offset and struct size of the ctypes mirrors equals what a C
    compiler makes of include/ttq.h."""
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"ttq_problem": binding.TTQProblem, "ttq_result": binding.TTQResult,
               "ttq_pivot": binding.TTQPivot}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ttq.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_workspace_size_and_validation(lib):
    p = inputs.config_d12()
    nb = binding.workspace_bytes(p)
    # cores of the 10 interior modes dominate: 64 * 385 * 64 doubles each
    assert nb >= 10 * 64 * 385 * 64 * 8
    assert nb % 256 == 0
    bad = inputs.config_c4(rank_cap=500)
    with pytest.raises(binding.TTQError):
        binding.workspace_bytes(bad)
    bad = inputs.make_problem("C", "rn", 4, 41, L=10.0)
    bad.nodes = bad.nodes[:3]
    bad.weights = bad.weights[:3]
    with pytest.raises(binding.TTQError):
        binding.workspace_bytes(bad)          # R^n form needs d == n
    for npiv in (-1, 5):                      # 0..TTQ_MAX_PIVOTS pivots per sweep
        with pytest.raises(binding.TTQError):
            binding.workspace_bytes(inputs.config_c4(npiv=npiv))
    # several pivots per sweep: each search's scratch beside the first's
    assert binding.workspace_bytes(inputs.config_c4(npiv=4)) > binding.workspace_bytes(inputs.config_c4())
    assert binding.workspace_bytes(inputs.config_c4(npiv=0)) == binding.workspace_bytes(inputs.config_c4())


def test_status_strings(lib):
    for code in (0, 1, 2, 3, -1, -2, -3, -5):
        assert lib.ttq_status_string(code)
