"""The library's host set-up (csrc/setup.cpp), checked on the CPU with small
drivers under tests/host/.

- XX^T reduced solver (xxt_check.cpp), on perturbed cubes whose reduced
  spaces have 343, 1,331 and 4,913 unknowns: the nested-dissection factors X
  against the dense explicit inverse the same set-up forms (X X^T = A_r^{-1}
  to 1e-13 relative), the agreement of the column- and row-major copies of X
  and the tiling of the first pass's segments.
- The three coarse operators (ar_check.cpp) against the oracle's.
- The lane packs of the mixed forms (pack_check.cpp) against the oracle's
  local inverses, size classes up to 64 dofs.
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


def test_lane_packs_hold_the_oracles_local_inverses(tmp_path):
    """The lane packs of the mixed forms, built by the library's host set-up
    on a perturbed 13^3 cube cut into 3- and 2-element segments (subdomains
    of 8 to 64 dofs, size classes up to 64): every subdomain is in a pack of
    the smallest class that holds it, once, and each lane's packed upper
    triangle is A_p^{-1} of the oracle's A_p (Sec. 3, Eq. (4)) for the same
    vertices, to 1e-12 of its largest entry."""
    import numpy as np

    from oracle import cgs_oracle as O
    from paper_2606_20496_b300 import meshes
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "pack_check")
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-fopenmp", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                          "-I", "/usr/local/cuda/include", "-o", exe,
                          os.path.join(ROOT, "tests", "host", "pack_check.cpp"), os.path.join(CSRC, "setup.cpp")],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    m = meshes.cube(13, perturb=0.15, seed=[2, 13], part_mode="mixed", name="cube13_mixed")
    src = tmp_path / "mesh.txt"
    with open(src, "w") as f:
        f.write(f"{m.nv} {m.ne} {m.boxes[0]} {m.boxes[1]} {m.boxes[2]}\n")
        f.write(" ".join("%.17g" % v for v in np.asarray(m.xyz).ravel()) + "\n")
        f.write(" ".join(str(int(v)) for v in np.asarray(m.conn).ravel()) + "\n")
        f.write(" ".join(str(int(v)) for v in np.asarray(m.part).ravel()) + "\n")
    dump = tmp_path / "packs.txt"
    out = subprocess.run([exe, str(src), str(dump)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    ref = {}
    for _, (ps, I, Ap, _L) in P.groups.items():
        for k in range(len(ps)):
            ref[tuple(sorted(int(v) for v in I[k]))] = (I[k], np.linalg.inv(Ap[k]))
    lines = open(dump).read().split("\n")
    n_wsub, n_pack = map(int, lines[0].split())
    assert n_wsub == 0                     # every subdomain (at most 64 dofs) is in a lane pack
    classes, seen, pos = set(), set(), 1
    for _ in range(n_pack):
        c = int(lines[pos])
        pos += 1
        classes.add(c)
        for _lane in range(32):
            ids = [int(t) for t in lines[pos].split()]
            tri = np.array([float(t) for t in lines[pos + 1].split()])
            pos += 2
            assert len(ids) == c and len(tri) == c * (c + 1) // 2
            live = [v for v in ids if v >= 0]
            if not live:
                assert not tri.any()
                continue
            key = tuple(sorted(live))
            assert key in ref and key not in seen
            seen.add(key)
            mm = len(live)
            assert ids[mm:] == [-1] * (c - mm)            # padding after the subdomain's dofs
            assert c == min(k for k in (8, 12, 16, 18, 20, 24, 27, 32, 40, 48, 56, 64) if k >= mm)
            I, inv = ref[key]
            perm = [int(np.flatnonzero(I == v)[0]) for v in live]
            want = inv[np.ix_(perm, perm)]
            got = np.zeros((c, c))
            got[np.triu_indices(c)] = tri
            assert np.abs(got[:mm, :mm] - np.triu(want)).max() <= 1e-12 * np.abs(want).max()
            assert not got[mm:, :].any() and not got[:, mm:].any()
    assert len(seen) == sum(len(ps) for ps, *_ in P.groups.values())
    assert {40, 48, 64} <= classes
