"""Thin Python binding of the C ABI in include/cgs.h (argument marshalling only).

Every function keeps the C name.  Device vectors are passed as CUDA tensors
(float64, contiguous) or raw device addresses; host arrays as numpy arrays.
All computation happens in libcgs.so; if the library is missing this module
raises on import of the library instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcgs.so")

NOALLOC_MAX_NV, NOALLOC_MAX_NR = 131072, 8192
PROJECTION_MAX = 64
OK, ERR_INVALID_ARG, ERR_INVALID_MESH, ERR_NOT_SPD, ERR_NO_CONVERGENCE, ERR_BREAKDOWN, ERR_OOM, \
    ERR_ADMISSION, ERR_TIMEOUT, ERR_CUDA = range(10)
PREC = {"fp64": 0, "fp32": 1, "fp16": 2}
FORM = {"hybrid": 0, "additive": 1, "ras": 2}
COARSE = {"auto": 0, "dense": 1, "xxt": 2}
COARSE_OP = {"cellwise": 0, "galerkin": 1, "vertex": 2}
OP = {"fp64": 0, "inner": 1, "outer": 2}
METHOD = {"pcg": 0, "richardson": 1, "fgmres": 2}

# every symbol include/cgs.h declares
EXPORTS = (
    "cgs_create", "cgs_destroy", "cgs_ctx_bytes_in_use", "cgs_mesh_setup", "cgs_mesh_free", "cgs_mesh_info",
    "cgs_mesh_set_form", "cgs_mesh_export", "cgs_apply_A", "cgs_apply_A_prec", "cgs_mesh_step_status",
    "cgs_mesh_set_wait_limits", "cgs_apply_local", "cgs_restrict",
    "cgs_coarse_solve", "cgs_interp", "cgs_apply_preconditioner", "cgs_apply_preconditioner_noalloc",
    "cgs_solve", "cgs_solve_host", "cgs_solve_wrapped", "cgs_mesh_set_projection", "cgs_mesh_projection_size",
    "cgs_profile_enable", "cgs_profile_read", "cgs_batch_create", "cgs_batch_free", "cgs_batch_solve",
    "cgs_batch_launches", "cgs_solve_batched", "cgs_mesh_tune", "cgs_mesh_get_schedule", "cgs_mesh_set_schedule",
    "cgs_batch_tune",
    "cgs_server_create",
    "cgs_server_free", "cgs_submit", "cgs_server_step", "cgs_poll", "cgs_server_drain", "cgs_server_footprint",
    "cgs_server_stats",
    "cgs_server_launches", "cgs_status_string",
    "cgs_last_error",
    "cgs_pmg_setup", "cgs_pmg_free", "cgs_pmg_info", "cgs_pmg_node_map", "cgs_pmg_node_coords", "cgs_pmg_apply_A",
    "cgs_pmg_smooth", "cgs_pmg_restrict", "cgs_pmg_prolong", "cgs_pmg_apply_preconditioner", "cgs_pmg_solve",
)
KERNEL_CLASSES = ("apply_A64", "apply_A32", "local", "restrict", "coarse", "interp", "pcg_xr", "pcg_dots",
                  "pcg_p", "other", "loop")


class CGSError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class Params(C.Structure):
    _fields_ = [("box", C.c_int * 3), ("box_margin", C.c_double), ("overlap_layers", C.c_int),
                ("prec", C.c_int), ("form", C.c_int), ("coarse_solver", C.c_int), ("coarse_operator", C.c_int),
                ("local_cg_steps", C.c_int), ("fault_negate_subdomain", C.c_int)]


class MeshInfo(C.Structure):
    _fields_ = [("nv", C.c_int64), ("ne", C.c_int64), ("n_free", C.c_int64), ("n_sub", C.c_int64),
                ("n_r", C.c_int64), ("max_sub_dofs", C.c_int64), ("sum_sub_dofs", C.c_int64), ("sum_sub_tri", C.c_int64),
                ("footprint_bytes", C.c_size_t), ("setup_seconds", C.c_double),
                ("kernel_launches", C.c_int64), ("n_box_entries", C.c_int64), ("n_lane_packs", C.c_int64),
                ("loop", C.c_int32), ("coarse_solver", C.c_int32), ("xxt_nnz", C.c_int64), ("ar_nnz", C.c_int64),
                ("coarse_operator", C.c_int32), ("n_hyb_entries", C.c_int64), ("n_jt_entries", C.c_int64),
                ("ell_nnz", C.c_int64), ("ell_slots", C.c_int64)]


class Schedule(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ("vert_chunk", "sub_chunk", "pack_chunk", "box_chunk", "tile_tma",
                                         "persistent", "pdl", "row_packs", "interp_cells")]


_lib = None


def load(path: str = LIB_PATH):
    """Load libcgs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not built: run `python -m paper_2606_20496_b300.build`")
    lib = C.CDLL(path)
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "cgs_create": ([C.POINTER(P), I32, C.c_size_t], I32),
        "cgs_destroy": ([P], I32),
        "cgs_ctx_bytes_in_use": ([P], C.c_size_t),
        "cgs_mesh_setup": ([P, P, I64, P, I64, P, P, C.POINTER(Params), C.POINTER(P)], I32),
        "cgs_mesh_free": ([P], I32),
        "cgs_mesh_info": ([P, C.POINTER(MeshInfo)], I32),
        "cgs_mesh_set_form": ([P, I32], I32),
        "cgs_mesh_export": ([P, P, P, P, P], I32),
        "cgs_apply_A": ([P, P, P, P], I32),
        "cgs_apply_A_prec": ([P, P, P, I32, P], I32),
        "cgs_mesh_step_status": ([P, P], I32),
        "cgs_mesh_set_wait_limits": ([P, I32, I32], I32),
        "cgs_apply_local": ([P, P, P, I32, P], I32),
        "cgs_restrict": ([P, P, P, P], I32),
        "cgs_coarse_solve": ([P, P, P, P], I32),
        "cgs_interp": ([P, P, P, P], I32),
        "cgs_apply_preconditioner": ([P, P, P, P], I32),
        "cgs_apply_preconditioner_noalloc": ([P, P, P, P], I32),
        "cgs_solve": ([P, P, P, I32, D, I32, P, P, P], I32),
        "cgs_solve_host": ([P, P, P, I32, D, I32, P, P, P], I32),
        "cgs_solve_wrapped": ([P, P, P, I32, D, I32, I32, C.POINTER(I32), C.POINTER(D), P], I32),
        "cgs_mesh_set_projection": ([P, I32], I32),
        "cgs_mesh_projection_size": ([P, C.POINTER(I32)], I32),
        "cgs_profile_enable": ([P, I32], I32),
        "cgs_profile_read": ([P, P, P], I32),
        "cgs_batch_create": ([P, P, I32, I32, C.POINTER(P)], I32),
        "cgs_batch_free": ([P], I32),
        "cgs_batch_solve": ([P, P, P, D, I32, P, P, P, P], I32),
        "cgs_batch_launches": ([P], I64),
        "cgs_solve_batched": ([P, I32, P, P, I32, D, I32, P, P, P], I32),
        "cgs_mesh_tune": ([P, P], I32),
        "cgs_server_create": ([P, I32, I64, I64, I32, I32, D, I32, C.POINTER(P)], I32),
        "cgs_server_free": ([P], I32),
        "cgs_submit": ([P, P, P, P, C.POINTER(C.c_uint64)], I32),
        "cgs_server_step": ([P, I32, P, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32)], I32),
        "cgs_poll": ([P, C.c_uint64, C.POINTER(I32), C.POINTER(I32), C.POINTER(D), C.POINTER(I32)], I32),
        "cgs_server_drain": ([P, C.POINTER(C.c_uint64), C.POINTER(I32), C.POINTER(D), C.POINTER(I32), I32], I32),
        "cgs_server_footprint": ([P, P, C.POINTER(C.c_size_t)], I32),
        "cgs_server_stats": ([P, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), C.POINTER(I32), C.POINTER(I32)], I32),
        "cgs_server_launches": ([P], I64),
        "cgs_batch_tune": ([P, P], I32),
        "cgs_mesh_get_schedule": ([P, C.POINTER(Schedule)], I32),
        "cgs_mesh_set_schedule": ([P, C.POINTER(Schedule)], I32),
        "cgs_pmg_setup": ([P, P, I64, P, I64, P, I32, C.POINTER(P)], I32),
        "cgs_pmg_free": ([P], I32),
        "cgs_pmg_info": ([P, I32, C.POINTER(I32), C.POINTER(I64), C.POINTER(I64)], I32),
        "cgs_pmg_node_map": ([P, I32, P], I32),
        "cgs_pmg_node_coords": ([P, I32, P], I32),
        "cgs_pmg_apply_A": ([P, I32, P, P, P], I32),
        "cgs_pmg_smooth": ([P, I32, P, P, P], I32),
        "cgs_pmg_restrict": ([P, I32, P, P, P], I32),
        "cgs_pmg_prolong": ([P, I32, P, P, P], I32),
        "cgs_pmg_apply_preconditioner": ([P, P, P, P], I32),
        "cgs_pmg_solve": ([P, P, P, D, I32, I32, C.POINTER(I32), C.POINTER(D), P], I32),
        "cgs_status_string": ([I32], C.c_char_p),
        "cgs_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(a):
    """Address of a CUDA tensor, a numpy array, an int address or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


def _check(status: int, where: str, allow=()):
    if status != OK and status not in allow:
        lib = load()
        raise CGSError(status, where, lib.cgs_last_error().decode())
    return status


def status_string(status: int) -> str:
    return load().cgs_status_string(status).decode()


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------

def cgs_create(device: int = 0, hbm_budget_bytes: int = 0):
    ctx = C.c_void_p()
    _check(load().cgs_create(C.byref(ctx), device, hbm_budget_bytes), "cgs_create")
    return ctx


def cgs_destroy(ctx):
    _check(load().cgs_destroy(ctx), "cgs_destroy")


def cgs_ctx_bytes_in_use(ctx) -> int:
    return int(load().cgs_ctx_bytes_in_use(ctx))


def cgs_mesh_setup(ctx, xyz, conn, dirichlet=None, elem_part=None, boxes=(4, 4, 4), margin=0.0, overlap=1,
                   prec="fp64", form="hybrid", coarse="auto", coarse_operator="cellwise", local_cg_steps=0,
                   fault_negate_subdomain=0):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    d = None if dirichlet is None else np.ascontiguousarray(dirichlet, dtype=np.uint8)
    part = None if elem_part is None else np.ascontiguousarray(elem_part, dtype=np.int32)
    prm = Params((C.c_int * 3)(*[int(b) for b in boxes]), float(margin), int(overlap), PREC[prec], FORM[form],
                 COARSE[coarse] if isinstance(coarse, str) else int(coarse),
                 COARSE_OP[coarse_operator] if isinstance(coarse_operator, str) else int(coarse_operator),
                 int(local_cg_steps), int(fault_negate_subdomain))
    mesh = C.c_void_p()
    st = load().cgs_mesh_setup(ctx, _ptr(xyz), xyz.shape[0], _ptr(conn), conn.shape[0], _ptr(d), _ptr(part),
                               C.byref(prm), C.byref(mesh))
    _check(st, "cgs_mesh_setup")
    return mesh


def cgs_mesh_free(mesh):
    _check(load().cgs_mesh_free(mesh), "cgs_mesh_free")


def cgs_mesh_info(mesh) -> dict:
    info = MeshInfo()
    _check(load().cgs_mesh_info(mesh, C.byref(info)), "cgs_mesh_info")
    return {f: getattr(info, f) for f, _ in MeshInfo._fields_}


def cgs_mesh_set_form(mesh, form: str):
    _check(load().cgs_mesh_set_form(mesh, FORM[form]), "cgs_mesh_set_form")


def cgs_mesh_export(mesh) -> dict:
    info = cgs_mesh_info(mesh)
    out = {"dirichlet": np.zeros(info["nv"], np.uint8), "box_active": np.zeros(info["n_r"], np.int64),
           "sub_ptr": np.zeros(info["n_sub"] + 1, np.int64), "sub_idx": np.zeros(info["sum_sub_dofs"], np.int32)}
    _check(load().cgs_mesh_export(mesh, *(_ptr(out[k]) for k in ("dirichlet", "box_active", "sub_ptr", "sub_idx"))),
           "cgs_mesh_export")
    return out


def cgs_apply_A(mesh, x, y, stream=None):
    _check(load().cgs_apply_A(mesh, _ptr(x), _ptr(y), _stream(stream)), "cgs_apply_A")


def cgs_apply_A_prec(mesh, x, y, op="inner", stream=None):
    """y = A x by the operator kernel `op` ("fp64", "inner" or "outer")."""
    _check(load().cgs_apply_A_prec(mesh, _ptr(x), _ptr(y), OP[op], _stream(stream)), "cgs_apply_A_prec")


def cgs_mesh_step_status(mesh, stream=None) -> int:
    """Status of the single-step calls since the last query (OK or ERR_TIMEOUT); resets it."""
    st = load().cgs_mesh_step_status(mesh, _stream(stream))
    _check(st, "cgs_mesh_step_status", allow=(ERR_TIMEOUT,))
    return st


def cgs_mesh_set_wait_limits(mesh, tile_wait=1 << 20, barrier_wait=1 << 22):
    """Iteration limits of the bounded device waits (a testing aid; 0 = give up at once)."""
    _check(load().cgs_mesh_set_wait_limits(mesh, int(tile_wait), int(barrier_wait)), "cgs_mesh_set_wait_limits")


def cgs_apply_local(mesh, r, l, weighted=True, stream=None):
    _check(load().cgs_apply_local(mesh, _ptr(r), _ptr(l), int(bool(weighted)), _stream(stream)), "cgs_apply_local")


def cgs_restrict(mesh, s, rr, stream=None):
    _check(load().cgs_restrict(mesh, _ptr(s), _ptr(rr), _stream(stream)), "cgs_restrict")


def cgs_coarse_solve(mesh, rr, ur, stream=None):
    _check(load().cgs_coarse_solve(mesh, _ptr(rr), _ptr(ur), _stream(stream)), "cgs_coarse_solve")


def cgs_interp(mesh, ur, z, stream=None):
    _check(load().cgs_interp(mesh, _ptr(ur), _ptr(z), _stream(stream)), "cgs_interp")


def cgs_apply_preconditioner(mesh, r, z, stream=None):
    _check(load().cgs_apply_preconditioner(mesh, _ptr(r), _ptr(z), _stream(stream)), "cgs_apply_preconditioner")


def cgs_apply_preconditioner_noalloc(mesh, r, z, stream=None):
    """z = M r without allocating device memory (see include/cgs.h)."""
    _check(load().cgs_apply_preconditioner_noalloc(mesh, _ptr(r), _ptr(z), _stream(stream)),
           "cgs_apply_preconditioner_noalloc")


def cgs_solve(mesh, b, x, nrhs=1, rtol=1e-8, maxit=1000, stream=None, allow=(ERR_NO_CONVERGENCE, ERR_BREAKDOWN)):
    """Returns (status, iters ndarray, relres ndarray)."""
    iters = np.zeros(nrhs, np.int32)
    relres = np.zeros(nrhs, np.float64)
    st = load().cgs_solve(mesh, _ptr(b), _ptr(x), nrhs, float(rtol), int(maxit), _ptr(iters), _ptr(relres),
                          _stream(stream))
    _check(st, "cgs_solve", allow)
    return st, iters, relres


def cgs_solve_host(mesh, b, x, nrhs=1, rtol=1e-8, maxit=1000, stream=None,
                   allow=(ERR_NO_CONVERGENCE, ERR_BREAKDOWN)):
    """b, x host numpy float64 arrays (pinned tensors work too)."""
    iters = np.zeros(nrhs, np.int32)
    relres = np.zeros(nrhs, np.float64)
    st = load().cgs_solve_host(mesh, _ptr(b), _ptr(x), nrhs, float(rtol), int(maxit), _ptr(iters),
                               _ptr(relres), _stream(stream))
    _check(st, "cgs_solve_host", allow)
    return st, iters, relres


def cgs_solve_wrapped(mesh, b, x, method="fgmres", rtol=1e-8, maxit=1000, restart=30, stream=None,
                      allow=(ERR_NO_CONVERGENCE, ERR_BREAKDOWN)):
    """Schwarz-Richardson, flexible GMRES(restart) or the PCG around the
    mesh's preconditioner.  Returns (status, iters, relres)."""
    it, rr = C.c_int(0), C.c_double(0.0)
    st = load().cgs_solve_wrapped(mesh, _ptr(b), _ptr(x), METHOD[method], float(rtol), int(maxit), int(restart),
                                  C.byref(it), C.byref(rr), _stream(stream))
    _check(st, "cgs_solve_wrapped", allow)
    return st, it.value, rr.value


def cgs_mesh_set_projection(mesh, l: int):
    """Keep up to l prior solutions for the projected start of cgs_solve (0 = off)."""
    _check(load().cgs_mesh_set_projection(mesh, int(l)), "cgs_mesh_set_projection")


def cgs_mesh_projection_size(mesh) -> int:
    k = C.c_int(0)
    _check(load().cgs_mesh_projection_size(mesh, C.byref(k)), "cgs_mesh_projection_size")
    return k.value


def cgs_profile_enable(mesh, enable=True):
    _check(load().cgs_profile_enable(mesh, int(bool(enable))), "cgs_profile_enable")


def cgs_profile_read(mesh) -> dict:
    """{kernel class: (milliseconds, launches)} since the last read."""
    ms = np.zeros(len(KERNEL_CLASSES), np.float64)
    n = np.zeros(len(KERNEL_CLASSES), np.int64)
    _check(load().cgs_profile_read(mesh, _ptr(ms), _ptr(n)), "cgs_profile_read")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}


def _ptr_array(items):
    arr = (C.c_void_p * len(items))(*[_ptr(i) for i in items])
    return arr


def cgs_batch_create(ctx, meshes, nrhs=1):
    """meshes: list of Mesh or raw handles; slot = mesh_index * nrhs + rhs."""
    hs = [m.handle if isinstance(m, Mesh) else m for m in meshes]
    arr = (C.c_void_p * len(hs))(*[h.value if isinstance(h, C.c_void_p) else h for h in hs])
    out = C.c_void_p()
    _check(load().cgs_batch_create(ctx, arr, len(hs), int(nrhs), C.byref(out)), "cgs_batch_create")
    return out


def cgs_batch_free(batch):
    _check(load().cgs_batch_free(batch), "cgs_batch_free")


def cgs_batch_solve(batch, bs, xs, rtol=1e-8, maxit=1000, stream=None,
                    allow=(ERR_NO_CONVERGENCE, ERR_BREAKDOWN)):
    """bs, xs: lists (one per slot) of device vectors.  Returns (status,
    iters, relres, per-slot status)."""
    n = len(bs)
    iters = np.zeros(n, np.int32)
    relres = np.zeros(n, np.float64)
    status = np.zeros(n, np.int32)
    st = load().cgs_batch_solve(batch, _ptr_array(bs), _ptr_array(xs), float(rtol), int(maxit), _ptr(iters),
                                _ptr(relres), _ptr(status), _stream(stream))
    _check(st, "cgs_batch_solve", allow)
    return st, iters, relres, status


def cgs_mesh_tune(mesh, stream=None):
    _check(load().cgs_mesh_tune(mesh, _stream(stream)), "cgs_mesh_tune")


def cgs_mesh_get_schedule(mesh) -> dict:
    sch = Schedule()
    _check(load().cgs_mesh_get_schedule(mesh, C.byref(sch)), "cgs_mesh_get_schedule")
    return {f: getattr(sch, f) for f, _ in Schedule._fields_}


def cgs_mesh_set_schedule(mesh, **fields):
    """Change fields of the mesh's schedule (the others keep their values)."""
    cur = cgs_mesh_get_schedule(mesh)
    unknown = set(fields) - set(cur)
    if unknown:
        raise ValueError(f"unknown schedule fields {sorted(unknown)}")
    cur.update({k: int(v) for k, v in fields.items()})
    sch = Schedule(**cur)
    _check(load().cgs_mesh_set_schedule(mesh, C.byref(sch)), "cgs_mesh_set_schedule")


def cgs_batch_tune(batch, stream=None):
    _check(load().cgs_batch_tune(batch, _stream(stream)), "cgs_batch_tune")


def cgs_batch_launches(batch) -> int:
    return int(load().cgs_batch_launches(batch))


def cgs_solve_batched(meshes, bs, xs, nrhs=1, rtol=1e-8, maxit=1000, stream=None,
                      allow=(ERR_NO_CONVERGENCE, ERR_BREAKDOWN)):
    hs = [m.handle if isinstance(m, Mesh) else m for m in meshes]
    arr = (C.c_void_p * len(hs))(*[h.value if isinstance(h, C.c_void_p) else h for h in hs])
    n = len(bs)
    iters = np.zeros(n, np.int32)
    relres = np.zeros(n, np.float64)
    st = load().cgs_solve_batched(arr, len(hs), _ptr_array(bs), _ptr_array(xs), int(nrhs), float(rtol), int(maxit),
                                  _ptr(iters), _ptr(relres), _stream(stream))
    _check(st, "cgs_solve_batched", allow)
    return st, iters, relres


def cgs_server_create(ctx, max_slots, pool_nv, pool_nr, prec="fp32", form="hybrid", rtol=1e-8, maxit=1000):
    """Server with up to max_slots solves in flight whose vectors share an
    arena of pool_nv vertex entries and pool_nr reduced entries."""
    out = C.c_void_p()
    _check(load().cgs_server_create(ctx, int(max_slots), int(pool_nv), int(pool_nr), PREC[prec], FORM[form],
                                    float(rtol), int(maxit), C.byref(out)), "cgs_server_create")
    return out


def cgs_server_drain(server, cap=4096):
    """Requests finished since the last drain: list of (ticket, iters, relres, status)."""
    t = (C.c_uint64 * cap)()
    it = (C.c_int * cap)()
    rr = (C.c_double * cap)()
    st = (C.c_int * cap)()
    n = load().cgs_server_drain(server, t, it, rr, st, int(cap))
    if n < 0:
        _check(ERR_INVALID_ARG, "cgs_server_drain")
    return [(int(t[i]), int(it[i]), float(rr[i]), int(st[i])) for i in range(n)]


def cgs_server_footprint(server, mesh) -> int:
    """Arena bytes one request on this mesh holds while it runs."""
    n = C.c_size_t()
    h = mesh.handle if isinstance(mesh, Mesh) else mesh
    _check(load().cgs_server_footprint(server, h, C.byref(n)), "cgs_server_footprint")
    return int(n.value)


def cgs_server_stats(server) -> dict:
    ab, ub = C.c_size_t(), C.c_size_t()
    a, q = C.c_int(), C.c_int()
    _check(load().cgs_server_stats(server, C.byref(ab), C.byref(ub), C.byref(a), C.byref(q)), "cgs_server_stats")
    return {"arena_bytes": int(ab.value), "bytes_in_use": int(ub.value), "active": a.value, "queued": q.value}


def cgs_server_free(server):
    _check(load().cgs_server_free(server), "cgs_server_free")


def cgs_submit(server, mesh, b, x) -> int:
    t = C.c_uint64()
    h = mesh.handle if isinstance(mesh, Mesh) else mesh
    _check(load().cgs_submit(server, h, _ptr(b), _ptr(x), C.byref(t)), "cgs_submit")
    return int(t.value)


def cgs_server_step(server, iterations=4, stream=None):
    """Returns (active, queued, finished) slot counts."""
    a, q, f = C.c_int(), C.c_int(), C.c_int()
    _check(load().cgs_server_step(server, int(iterations), _stream(stream), C.byref(a), C.byref(q), C.byref(f)),
           "cgs_server_step")
    return a.value, q.value, f.value


def cgs_poll(server, ticket):
    """Returns None while pending, else (iters, relres, status)."""
    d, it, st = C.c_int(), C.c_int(), C.c_int()
    rr = C.c_double()
    _check(load().cgs_poll(server, C.c_uint64(ticket), C.byref(d), C.byref(it), C.byref(rr), C.byref(st)),
           "cgs_poll")
    return (it.value, rr.value, st.value) if d.value else None


def cgs_server_launches(server) -> int:
    return int(load().cgs_server_launches(server))


# ---- p-multigrid wrap -------------------------------------------------------

def cgs_pmg_setup(mesh, xyz, conn, orders=(7, 3)):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    ords = np.ascontiguousarray(orders, dtype=np.int32)
    out = C.c_void_p()
    _check(load().cgs_pmg_setup(mesh, _ptr(xyz), xyz.shape[0], _ptr(conn), conn.shape[0], _ptr(ords), len(ords),
                                C.byref(out)), "cgs_pmg_setup")
    return out


def cgs_pmg_free(pmg):
    _check(load().cgs_pmg_free(pmg), "cgs_pmg_free")


def cgs_pmg_info(pmg, level) -> dict:
    o, n, f = C.c_int(0), C.c_int64(0), C.c_int64(0)
    _check(load().cgs_pmg_info(pmg, level, C.byref(o), C.byref(n), C.byref(f)), "cgs_pmg_info")
    return {"order": o.value, "n_nodes": n.value, "n_free": f.value}


def cgs_pmg_node_map(pmg, level, ne) -> np.ndarray:
    p = cgs_pmg_info(pmg, level)["order"] + 1
    out = np.empty((ne, p, p, p), dtype=np.int32)
    _check(load().cgs_pmg_node_map(pmg, level, _ptr(out)), "cgs_pmg_node_map")
    return out


def cgs_pmg_node_coords(pmg, level) -> np.ndarray:
    out = np.empty((cgs_pmg_info(pmg, level)["n_nodes"], 3), dtype=np.float64)
    _check(load().cgs_pmg_node_coords(pmg, level, _ptr(out)), "cgs_pmg_node_coords")
    return out


def cgs_pmg_apply_A(pmg, level, x, y, stream=None):
    _check(load().cgs_pmg_apply_A(pmg, level, _ptr(x), _ptr(y), _stream(stream)), "cgs_pmg_apply_A")


def cgs_pmg_smooth(pmg, level, r, z, stream=None):
    _check(load().cgs_pmg_smooth(pmg, level, _ptr(r), _ptr(z), _stream(stream)), "cgs_pmg_smooth")


def cgs_pmg_restrict(pmg, level, rf, rc, stream=None):
    _check(load().cgs_pmg_restrict(pmg, level, _ptr(rf), _ptr(rc), _stream(stream)), "cgs_pmg_restrict")


def cgs_pmg_prolong(pmg, level, uc, uf, stream=None):
    _check(load().cgs_pmg_prolong(pmg, level, _ptr(uc), _ptr(uf), _stream(stream)), "cgs_pmg_prolong")


def cgs_pmg_apply_preconditioner(pmg, r, z, stream=None):
    _check(load().cgs_pmg_apply_preconditioner(pmg, _ptr(r), _ptr(z), _stream(stream)),
           "cgs_pmg_apply_preconditioner")


def cgs_pmg_solve(pmg, b, x, rtol=1e-8, maxit=500, restart=30, stream=None,
                  allow=(ERR_NO_CONVERGENCE, ERR_BREAKDOWN)):
    """Flexible GMRES on the finest level with the p-multigrid preconditioner.
    Returns (status, iters, relres)."""
    it, rr = C.c_int(0), C.c_double(0.0)
    st = load().cgs_pmg_solve(pmg, _ptr(b), _ptr(x), float(rtol), int(maxit), int(restart), C.byref(it),
                              C.byref(rr), _stream(stream))
    _check(st, "cgs_pmg_solve", allow)
    return st, it.value, rr.value


class PMG:
    """Owning handle around cgs_pmg_setup / cgs_pmg_free."""

    def __init__(self, mesh, xyz, conn, orders=(7, 3)):
        self.handle = cgs_pmg_setup(mesh.handle if isinstance(mesh, Mesh) else mesh, xyz, conn, orders)
        self.orders = tuple(orders)
        self.ne = int(np.asarray(conn).shape[0])
        self.levels = [cgs_pmg_info(self.handle, l) for l in range(len(self.orders) + 1)]

    def free(self):
        if self.handle is not None:
            cgs_pmg_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()


class Mesh:
    """Owning handle around cgs_mesh_setup / cgs_mesh_free."""

    def __init__(self, ctx, xyz, conn, part=None, boxes=(4, 4, 4), dirichlet=None, margin=0.0, overlap=1,
                 prec="fp64", form="hybrid", coarse="auto", coarse_operator="cellwise", local_cg_steps=0):
        self.handle = cgs_mesh_setup(ctx, xyz, conn, dirichlet, part, boxes, margin, overlap, prec, form, coarse,
                                     coarse_operator, local_cg_steps)
        self.info = cgs_mesh_info(self.handle)
        self.prec = prec

    def free(self):
        if self.handle is not None:
            cgs_mesh_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()
