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
- The assembled rows of A (ell_check.cpp), float64 and float pairs, against
  the oracle's assembled operator, with and without an outflow Dirichlet
  set.
- The explicit rows of J~ and the hybrid restriction's (J~, A J~) entries
  (jt_check.cpp) against the oracle's interpolation and operator.
- The spectral-element levels of the p-multigrid wrap (sem_check.cpp):
  GLL rule, D, numbering, metric, Dirichlet nodes, multiplicities and the
  element smoothers against the SEM oracle.
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


@pytest.mark.parametrize("case", ["cube3_n7", "cyl16_n4"])
def test_sem_level_matches_oracle(tmp_path, case):
    """The spectral-element set-up of the p-multigrid wrap (host C++, Sec. 1
    and Eq. (14)) against the oracle's (numpy), on a perturbed 3^3 cube at
    order 7 and the 16-fold reduced hollow cylinder (periodic around) at
    order 4: the GLL nodes and D, the node numbering (the same partition of
    element-local nodes into global nodes), the metric w det J J^-1 J^-T at
    every node, the Dirichlet nodes and multiplicities, and the element
    smoother (the fast-diagonalisation inverse of each element applied to
    random vectors) to 1e-12."""
    import numpy as np

    from oracle import sem_oracle as SO
    from paper_2606_20496_b300 import meshes
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "sem_check")
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-fopenmp", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                          "-I", "/usr/local/cuda/include", "-o", exe,
                          os.path.join(ROOT, "tests", "host", "sem_check.cpp"), os.path.join(CSRC, "sem_setup.cpp")],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    if case == "cube3_n7":
        m, n = meshes.cube(3, perturb=0.15, seed=11, name="cube3"), 7
    else:
        m, _ = meshes.workload_cylinder(scale=16)
        n = 4
    src = tmp_path / "mesh.txt"
    with open(src, "w") as f:
        f.write(f"{n} {m.nv} {m.ne}\n")
        f.write(" ".join("%.17g" % v for v in np.asarray(m.xyz).ravel()) + "\n")
        f.write(" ".join(str(int(v)) for v in np.asarray(m.conn).ravel()) + "\n")
    dump = tmp_path / "sem.txt"
    out = subprocess.run([exe, str(src), str(dump)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = open(dump).read().split("\n")
    p, ng, nfree = map(int, lines[0].split())
    x = np.array(lines[1].split(), dtype=float)
    D = np.array(lines[2].split(), dtype=float).reshape(p, p)
    p3, ne = p ** 3, m.ne
    l2g = np.empty((ne, p3), dtype=np.int64)
    G = np.empty((ne, 6, p3))
    S = np.empty((ne, 3, p, p))
    lam = np.empty((ne, 3, p))
    pos = 3
    for e in range(ne):
        l2g[e] = np.array(lines[pos].split(), dtype=np.int64)
        G[e] = np.array(lines[pos + 1].split(), dtype=float).reshape(6, p3)
        S[e] = np.array(lines[pos + 2].split(), dtype=float).reshape(3, p, p)
        lam[e] = np.array(lines[pos + 3].split(), dtype=float).reshape(3, p)
        pos += 4
    tail = np.array([ln.split() for ln in lines[pos:pos + ng]], dtype=float)
    dirc, inv_mult = tail[:, 0].astype(bool), tail[:, 1]

    lev = SO.Level(m.xyz, m.conn, n)
    assert p == lev.p and ng == lev.ng and nfree == int((~lev.dir).sum())
    assert np.abs(x - lev.x).max() <= 1e-14
    assert np.abs(D - lev.D).max() <= 1e-12 * np.abs(lev.D).max()
    # numbering: one oracle node per library node and the other way round
    lo = lev.l2g.reshape(ne, p3)
    fwd = {}
    for a, b in zip(l2g.ravel(), lo.ravel()):
        assert fwd.setdefault(int(a), int(b)) == int(b)
    assert len(fwd) == ng and len(set(fwd.values())) == ng
    o_of = np.array([fwd[g] for g in range(ng)])
    assert np.array_equal(dirc, lev.dir[o_of])
    assert np.abs(inv_mult - 1.0 / lev.mult[o_of]).max() <= 1e-15
    # metric, entries 00 01 02 11 12 22 at node (k, j, i)
    Go = lev.G.reshape(ne, p3, 3, 3)
    for c, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        assert np.abs(G[:, c] - Go[:, :, a, b]).max() <= 1e-12 * np.abs(Go).max(), (a, b)
    # the element smoother: the library's S and eigenvalues in the oracle's
    # fast-diagonalisation apply against the oracle's own
    sm = SO.Smoother(lev)
    mine = SO.Smoother.__new__(SO.Smoother)
    mine.lev, mine.S, mine.lam = lev, S, lam
    rng = np.random.default_rng(4)
    for _ in range(2):
        rL = rng.standard_normal((ne, p, p, p))
        want = sm.local_solve(rL)
        got = mine.local_solve(rL)
        assert np.isfinite(got).all()
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("case", ["cube8", "cube8_outflow", "cyl8"])
def test_assembled_rows_match_oracle(tmp_path, case):
    """The sliced-ELL rows of the assembled free block A = Q^T A_L Q (Sec. 3)
    built by the library's host set-up: per vertex, the same columns as the
    oracle's assembled operator (none for a Dirichlet vertex), float64 values
    to 1e-14 of the row's largest, and the mixed forms' float pairs equal to
    them to 2^-46 (hi the rounded value, |lo| at most half an ulp of hi)."""
    import numpy as np

    from oracle import cgs_oracle as O
    from paper_2606_20496_b300 import meshes
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "ell_check")
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-fopenmp", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                          "-I", "/usr/local/cuda/include", "-o", exe,
                          os.path.join(ROOT, "tests", "host", "ell_check.cpp"), os.path.join(CSRC, "setup.cpp")],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    m, _ = meshes.workload_cylinder(scale=8) if case == "cyl8" else meshes.workload_cube8()
    d = meshes.outflow_dirichlet(m) if case.endswith("outflow") else None
    src = tmp_path / "mesh.txt"
    with open(src, "w") as f:
        f.write(f"{m.nv} {m.ne} {m.boxes[0]} {m.boxes[1]} {m.boxes[2]} {0 if d is None else 1}\n")
        f.write(" ".join("%.17g" % v for v in np.asarray(m.xyz).ravel()) + "\n")
        f.write(" ".join(str(int(v)) for v in np.asarray(m.conn).ravel()) + "\n")
        f.write(" ".join(str(int(v)) for v in np.asarray(m.part).ravel()) + "\n")
        if d is not None:
            f.write(" ".join(str(int(v)) for v in np.asarray(d).astype(int)) + "\n")
    dump = tmp_path / "ell.txt"
    out = subprocess.run([exe, str(src), str(dump)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes, dirichlet=None if d is None else d.astype(bool))
    A = P.A.tocsr()
    lines = open(dump).read().split("\n")
    pos = 0
    for pairs in (False, True):
        w, nsl = map(int, lines[pos].split())
        pos += 1
        assert nsl == (m.nv + 31) // 32 and w >= 1
        for v in range(m.nv):
            t = lines[pos].split()
            pos += 1
            if P.dir[v]:
                assert not t
                continue
            step = 3 if pairs else 2
            cols = np.array(t[0::step], dtype=np.int64)
            if pairs:
                hi = np.array(t[1::3], dtype=np.float32).astype(np.float64)
                lo = np.array(t[2::3], dtype=np.float32).astype(np.float64)
                vals = hi + lo
            else:
                vals = np.array(t[1::2], dtype=float)
            fv = P.free_pos[v]
            lo_, hi_ = A.indptr[fv], A.indptr[fv + 1]
            want_cols = P.free[A.indices[lo_:hi_]]         # vertex ids of the row's columns
            order = np.argsort(want_cols)
            assert np.array_equal(cols, want_cols[order]), v
            want = A.data[lo_:hi_][order]
            scale = np.abs(want).max()
            assert np.abs(vals - want).max() <= (2.0 ** -46 if pairs else 1e-14) * scale, v
            if pairs:
                assert np.array_equal(hi.astype(np.float32), want.astype(np.float32)) or \
                    np.abs(hi - want).max() <= 2.0 ** -24 * scale
                assert np.all(np.abs(lo) <= np.abs(np.spacing(hi.astype(np.float32)).astype(np.float64)))


@pytest.mark.parametrize("case", ["cube8", "cyl8"])
def test_interpolation_rows_and_hybrid_entries_match_oracle(tmp_path, case):
    """The explicit rows of J~ = W Q^T J_L (Sec. 4) and the hybrid
    restriction's entries (J~_vc, (A J~)_vc) (Eq. (5) without the residual
    update) built by the library's host set-up in the FP64 form, against the
    oracle's interpolation and operator applied to unit vectors of the
    reduced space: every nonzero present once, values to 1e-13."""
    import numpy as np

    from oracle import cgs_oracle as O
    from paper_2606_20496_b300 import meshes
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "jt_check")
    res = subprocess.run([gxx, "-std=c++17", "-O2", "-fopenmp", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                          "-I", "/usr/local/cuda/include", "-o", exe,
                          os.path.join(ROOT, "tests", "host", "jt_check.cpp"), os.path.join(CSRC, "setup.cpp")],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    m, _ = meshes.workload_cylinder(scale=8) if case == "cyl8" else meshes.workload_cube8()
    src = tmp_path / "mesh.txt"
    with open(src, "w") as f:
        f.write(f"{m.nv} {m.ne} {m.boxes[0]} {m.boxes[1]} {m.boxes[2]}\n")
        f.write(" ".join("%.17g" % v for v in np.asarray(m.xyz).ravel()) + "\n")
        f.write(" ".join(str(int(v)) for v in np.asarray(m.conn).ravel()) + "\n")
        f.write(" ".join(str(int(v)) for v in np.asarray(m.part).ravel()) + "\n")
    dump = tmp_path / "jt.txt"
    out = subprocess.run([exe, str(src), str(dump)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    # the oracle's J~ and A J~, column by column
    J = np.stack([P.interp(np.eye(P.nr)[c]) for c in range(P.nr)], axis=1)       # (nv, nr)
    AJ = np.stack([P.apply_A(J[:, c]) for c in range(P.nr)], axis=1)
    lines = open(dump).read().split("\n")
    nr, nrows, _ = map(int, lines[0].split())
    assert nr == P.nr
    sj, sg = np.abs(J).max(), np.abs(AJ).max()
    got = np.zeros_like(J)
    rows_seen = set()
    for ln in lines[1:1 + nrows]:
        t = ln.split()
        v = int(t[0])
        assert v not in rows_seen and not P.dir[v]
        rows_seen.add(v)
        for c, val in zip(t[1::2], t[2::2]):
            assert got[v, int(c)] == 0.0
            got[v, int(c)] = float(val)
    assert np.abs(got - J).max() <= 1e-13 * sj
    gj, gg = np.zeros_like(J), np.zeros_like(AJ)
    seen = set()
    for ln in lines[1 + nrows:]:
        if not ln.strip():
            continue
        v, c, jv, av = ln.split()
        key = (int(v), int(c))
        assert key not in seen
        seen.add(key)
        gj[key], gg[key] = float(jv), float(av)
    assert np.abs(gj - J).max() <= 1e-13 * sj
    assert np.abs(gg - AJ).max() <= 1e-13 * sg
