"""Host logic of the coarse problem's nested-dissection factorisation (no GPU).

tests/coarse_plan_check.cpp is compiled with the library's host mesh and plan
sources and carries the plan out literally on the CPU for a random coarse
matrix with the method's coupling (entities sharing a subdomain), comparing
the solve with a dense pivoted LU solve.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2501_01676_gb300", "csrc")


def _cuda_include():
    nv = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nv))), "include")
    return inc if os.path.exists(os.path.join(inc, "cuda_runtime.h")) else "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("ndplan") / "coarse_plan_check")
    cmd = [gxx, "-std=c++17", "-O2", "-I", _cuda_include(), "-x", "c++",
           os.path.join(ROOT, "tests", "coarse_plan_check.cpp"), "-x", "c++", os.path.join(CSRC, "host_mesh.cpp"),
           "-x", "c++", os.path.join(CSRC, "coarse_plan.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


@pytest.mark.parametrize("case", [
    (2, 2, 2, 3, 1),      # one level of faces around the centre
    (3, 3, 3, 3, 2),
    (4, 4, 4, 2, 3),
    (4, 3, 5, -5, 4),     # uneven slabs, unequal grid sides
    (8, 8, 8, 2, 5),      # the 8x8x8 grid of the large workloads
    (6, 6, 6, -6, 6),
    (1, 4, 4, 2, 7),      # a single slab in x
    (2, 1, 1, 3, 8),      # one face: a single front
])
def test_nested_dissection_solve_matches_dense(checker, case):
    r = subprocess.run([checker] + [str(v) for v in case], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    tok = r.stdout.split()
    assert tok[0] == "ok" and float(tok[1]) < 1e-9
