"""Host set-up of the XX^T reduced solver, checked on the CPU.

Compiles the library's host set-up (csrc/setup.cpp) with a small driver
(tests/host/xxt_check.cpp) and runs it on perturbed cubes whose reduced spaces
have 343, 1,331 and 4,913 unknowns.  The driver checks the nested-dissection
factors X against the dense explicit inverse the same set-up forms (X X^T =
A_r^{-1} to 1e-13 relative), the agreement of the column- and row-major
copies of X and the tiling of the first pass's segments.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_20496_b300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("xxt") / "xxt_check")
    cmd = [gxx, "-std=c++17", "-O2", "-fopenmp", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           "-I", "/usr/local/cuda/include", "-o", out, os.path.join(ROOT, "tests", "host", "xxt_check.cpp"),
           os.path.join(CSRC, "setup.cpp")]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    return out


@pytest.mark.parametrize("n,boxes,nr", [(12, 6, 343), (16, 10, 1331), (20, 16, 4913)])
def test_xxt_factors_equal_dense_inverse(driver, n, boxes, nr):
    res = subprocess.run([driver, str(n), str(boxes)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    m = re.search(r"nr=(\d+) nnz=(\d+) .* consistency errors=(\d+) \|XX\^T - inv\|/\|inv\| = (\S+)", res.stdout)
    assert m, res.stdout
    assert int(m.group(1)) == nr and int(m.group(3)) == 0
    assert 0 < int(m.group(2)) < nr * nr * 0.25          # sparse under nested dissection
    assert float(m.group(4)) <= 1e-13
