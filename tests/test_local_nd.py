"""Host logic of the local nested dissection (one level inside every subdomain;
no GPU).

tests/local_nd_check.cpp is compiled with the library's host mesh source and
checks the plan's structure (children tile the subdomains, the maps hold the
same global dofs, every interior dof is a separator or interior to one child)
and its algebra: for random child matrices the Schur complement onto the
interface by one dense elimination equals the children's Schur complements
extend-added by the plan's maps with the separators eliminated afterwards, and
condensation and recovery in the library's order (children, then separators;
separators, then children) equal one dense condensation and recovery.
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
    exe = str(tmp_path_factory.mktemp("localnd") / "local_nd_check")
    cmd = [gxx, "-std=c++17", "-O2", "-I", _cuda_include(), "-x", "c++",
           os.path.join(ROOT, "tests", "local_nd_check.cpp"), "-x", "c++", os.path.join(CSRC, "host_mesh.cpp"),
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


@pytest.mark.parametrize("case", [
    (2, 2, 2, 4, 1),      # even slabs: 8 children of 2^3 elements
    (2, 2, 2, 5, 2),      # odd slabs: children of 2 and 3 elements
    (3, 2, 2, -6, 3),     # uneven slabs 1..6 (a 1-element slab is not split)
    (1, 1, 1, 6, 4),      # one subdomain: every boundary node Dirichlet
    (2, 3, 1, -4, 5),
    (2, 2, 2, 1, 6),      # 1-element slabs: no split, no separators
])
def test_local_nested_dissection_plan(checker, case):
    r = subprocess.run([checker] + [str(v) for v in case], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    tok = r.stdout.split()
    assert tok[0] == "ok" and float(tok[1]) < 1e-10
