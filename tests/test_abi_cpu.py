"""Host-only checks: the C-ABI library builds for sm_103a, loads, and exports
every symbol include/cgs.h declares; the input generators have the workload
shapes.  No GPU computation happens here."""
import os
import re

import numpy as np
import pytest

from paper_2606_20496_b300 import build as B
from paper_2606_20496_b300 import cgs, meshes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return cgs.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "cgs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cgs_[a-z_A-Z0-9]+)\s*\(", text)))


def test_header_declarations_match_binding():
    assert set(_declared()) == set(cgs.EXPORTS)


def test_schedule_struct_matches_header():
    """The binding's cgs_schedule mirrors the header's fields, in order, all int32."""
    text = open(os.path.join(ROOT, "include", "cgs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*cgs_schedule;", text).group(1)
    fields = [f.strip() for f in re.sub(r"\bint32_t\b", "", body).replace(";", ",").split(",") if f.strip()]
    assert body.count("int32_t") == 1
    assert [f[0] for f in cgs.Schedule._fields_] == fields
    assert all(f[1] is cgs.C.c_int32 for f in cgs.Schedule._fields_)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for s in range(10):
        assert cgs.status_string(s)
    assert cgs.status_string(0) == "ok"


def test_create_without_gpu_reports_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(cgs.CGSError) as ei:
        cgs.cgs_create(0)
    assert ei.value.status in (cgs.ERR_CUDA, cgs.ERR_INVALID_ARG)


@pytest.mark.parametrize("fn,nv,ne,nsub", [
    (meshes.workload_cube8, 729, 512, 64),
    (meshes.workload_cube32, 35937, 32768, 4096),
])
def test_workload_shapes(fn, nv, ne, nsub):
    m, b = fn()
    assert (m.nv, m.ne, int(m.part.max()) + 1) == (nv, ne, nsub)
    assert b.shape == (nv,)
    assert m.conn.min() >= 0 and m.conn.max() < nv


def test_cylinder_shape_without_building():
    nr, nt, nz = 64, 128, 128
    assert (nr + 1) * nt * (nz + 1) == 1073280 and nr * nt * nz == 1048576
    m = meshes.cylinder(8, 16, 8, grading=1.05 ** 8, boxes=(2, 2, 2))
    assert m.nv == 9 * 16 * 9 and m.ne == 8 * 16 * 8
    r = np.hypot(m.xyz[:, 0], m.xyz[:, 1])
    assert abs(r.min() - 1.0) < 1e-12 and abs(r.max() - 2.0) < 1e-12


def test_segments_rule():
    assert meshes.segments(4, "mixed") == [2, 2]
    assert meshes.segments(5, "mixed") == [3, 2]
    assert meshes.segments(7, "mixed") == [3, 2, 2]
    assert meshes.segments(6, "mixed") == [3, 3]
    assert meshes.segments(7, "two") == [2, 2, 2, 1]
    for n in range(1, 30):
        assert sum(meshes.segments(n, "mixed")) == n


def test_binding_constants_match_header():
    text = open(os.path.join(ROOT, "include", "cgs.h")).read()
    defs = dict(re.findall(r"#define (CGS_\w+) (\d+)\b", text))
    assert int(defs["CGS_NOALLOC_MAX_NV"]) == cgs.NOALLOC_MAX_NV
    assert int(defs["CGS_NOALLOC_MAX_NR"]) == cgs.NOALLOC_MAX_NR
    assert int(defs["CGS_PROJECTION_MAX"]) == cgs.PROJECTION_MAX


def _struct_fields(name):
    text = open(os.path.join(ROOT, "include", "cgs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", text).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            m = re.search(r"(\w+)\s*(\[\d+\])?\s*$", part.strip())
            names.append(m.group(1))
    return names


@pytest.mark.parametrize("cname,py", [("cgs_params", "Params"), ("cgs_mesh_info_t", "MeshInfo"),
                                      ("cgs_schedule", "Schedule")])
def test_binding_structs_follow_the_header(cname, py):
    """Every ABI struct of the binding has the header's fields in its order."""
    assert [f[0] for f in getattr(cgs, py)._fields_] == _struct_fields(cname)
