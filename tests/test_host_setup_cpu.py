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


def test_coarse_operators_match_oracle(tmp_path):
    """The library's host set-up of A_r (cell-wise Eq. (12), Galerkin J~^T A J~,
    vertex-based J^T A J) against the oracle's on a perturbed cube: the same
    active box vertices, the same nonzero count, A_r^{-1} to 1e-13."""
    import numpy as np

    from oracle import cgs_oracle as O
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "ar_check")
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-fopenmp", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                          "-I", "/usr/local/cuda/include", "-o", exe,
                          os.path.join(ROOT, "tests", "host", "ar_check.cpp"), os.path.join(CSRC, "setup.cpp")],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    dump = str(tmp_path / "ar.txt")
    assert subprocess.run([exe, dump], timeout=300).returncode == 0
    # the assembly does not depend on the number of threads
    one = str(tmp_path / "ar1.txt")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    assert subprocess.run([exe, one], timeout=300, env=env).returncode == 0
    assert open(one).read() == open(dump).read()
    lines = open(dump).read().split("\n")
    nv = int(lines[0])
    xyz = np.array([[float(t) for t in line.split()] for line in lines[1:1 + nv]])
    n = 8
    conn = np.array([[(i + (m & 1)) + (n + 1) * ((j + ((m >> 1) & 1)) + (n + 1) * (k + ((m >> 2) & 1)))
                      for m in range(8)] for k in range(n) for j in range(n) for i in range(n)])
    part = np.array([(i // 2) + (n // 2) * ((j // 2) + (n // 2) * (k // 2))
                     for k in range(n) for j in range(n) for i in range(n)])
    pos = 1 + nv
    nnzs = {}
    for op in ("broken", "galerkin", "vertex"):
        nr, nnz = map(int, lines[pos].split())
        active = np.array([int(t) for t in lines[pos + 1].split()])
        inv = np.array([float(t) for t in lines[pos + 2:pos + 2 + nr * nr]]).reshape(nr, nr)
        pos += 2 + nr * nr
        P = O.Problem(xyz, conn, part, (4, 4, 4), coarse_operator=op)
        ref = np.linalg.inv(P.Ar)
        assert nr == P.nr and np.array_equal(active, P.box_active)
        assert nnz == int(np.count_nonzero(P.Ar))
        assert np.abs(inv - ref).max() <= 1e-13 * np.abs(ref).max()
        nnzs[op] = nnz
    assert nnzs["galerkin"] > 2 * nnzs["broken"] and nnzs["vertex"] > 2 * nnzs["broken"]
