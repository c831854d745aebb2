"""Run a few complete coarse solves of one workload through the C ABI.

    python -m paper_2606_20496_b300.run_case --workload cylinder --prec fp32 --solves 2

Used as the target of profiler runs (ncu) and for quick timing; prints one
JSON line with the setup time, iteration counts, relative residuals and the
mean event time per solve.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def load_workload(name: str):
    from . import meshes
    if name == "cube8":
        return meshes.workload_cube8()
    if name == "cube32":
        return meshes.workload_cube32()
    if name == "cylinder":
        return meshes.workload_cylinder()
    if name.startswith("cylinder/"):
        return meshes.workload_cylinder(scale=int(name.split("/")[1]))
    raise ValueError(name)


def main():
    import torch

    from . import build, cgs
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cube32")
    ap.add_argument("--prec", default="fp32", choices=list(cgs.PREC))
    ap.add_argument("--form", default="hybrid", choices=list(cgs.FORM))
    ap.add_argument("--coarse-operator", default="cellwise", choices=list(cgs.COARSE_OP),
                    help="A_r: cell-wise (Eq. (12)), galerkin (J~^T A J~) or vertex (vertex-based J^T A J)")
    ap.add_argument("--coarse", default="auto", choices=list(cgs.COARSE),
                    help="reduced solver: auto (XX^T above 1500 unknowns), dense or xxt")
    ap.add_argument("--solves", type=int, default=2)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=1000)
    ap.add_argument("--tune", action="store_true", help="run the schedule autotuner after setup")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="also solve in the FP64 form and report the relative solution difference")
    ap.add_argument("--profile", action="store_true", help="per-kernel CUDA-event times (host-driven loop)")
    ap.add_argument("--tile-tma", type=int, choices=(0, 1), default=None,
                    help="force the element-tile loading of the mixed-form applies (default: setup's choice)")
    ap.add_argument("--persistent", type=int, choices=(-1, 0, 1), default=None,
                    help="persistent loop: 1 on, 0 or -1 off (default: setup's choice)")
    ap.add_argument("--pdl", type=int, choices=(0, 1), default=None,
                    help="programmatic dependent launch: 1 on, 0 off (default: setup's choice)")
    ap.add_argument("--row-packs", type=int, choices=(0, 1), default=None,
                    help="four lanes per small subdomain where the mesh has row packs: 1 on, 0 off")
    ap.add_argument("--interp-cells", type=int, choices=(0, 1), default=None,
                    help="interpolation by cell-sorted entries (1) or by vertex with the dots fused (0)")
    ap.add_argument("--sequence", type=int, default=0,
                    help="also solve a slowly varying series of this many right-hand sides, plain and with "
                         "the projection onto prior solutions")
    ap.add_argument("--projection", type=int, default=8, help="prior solutions kept for --sequence")
    for name in ("vert-chunk", "sub-chunk", "pack-chunk", "box-chunk"):
        ap.add_argument(f"--{name}", type=int, default=None, help=f"force the schedule's {name.replace('-', '_')}")
    args = ap.parse_args()
    build.build()
    m, b = load_workload(args.workload)
    ctx = cgs.cgs_create(0)
    t0 = time.perf_counter()
    h = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=args.prec, form=args.form, coarse=args.coarse,
                 coarse_operator=args.coarse_operator)
    setup_s = time.perf_counter() - t0
    if args.tune:
        cgs.cgs_mesh_tune(h.handle)
    forced = {k: v for k, v in (("tile_tma", args.tile_tma), ("persistent", args.persistent), ("pdl", args.pdl),
                                ("row_packs", args.row_packs), ("interp_cells", args.interp_cells),
                                ("vert_chunk", args.vert_chunk), ("sub_chunk", args.sub_chunk),
                                ("pack_chunk", args.pack_chunk), ("box_chunk", args.box_chunk)) if v is not None}
    if forced:
        cgs.cgs_mesh_set_schedule(h.handle, **forced)
    bd = torch.as_tensor(b, dtype=torch.float64, device="cuda")
    x = torch.empty_like(bd)
    if args.profile:
        cgs.cgs_profile_enable(h.handle, True)
    its, rels, ms = [], [], []
    for _ in range(args.solves):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, it, rel = cgs.cgs_solve(h.handle, bd, x, rtol=args.rtol, maxit=args.maxit)
        e1.record()
        torch.cuda.synchronize()
        its.append(int(it[0]))
        rels.append(float(rel[0]))
        ms.append(e0.elapsed_time(e1))
        if st != cgs.OK and not (st == cgs.ERR_NO_CONVERGENCE and it[0] == args.maxit):
            raise SystemExit(f"solve failed: {cgs.status_string(st)}")
    info = cgs.cgs_mesh_info(h.handle)
    out = {"workload": args.workload, "prec": args.prec, "form": args.form, "nv": h.info["nv"],
           "schedule": cgs.cgs_mesh_get_schedule(h.handle), "loop": info["loop"],
           "ne": h.info["ne"], "n_sub": h.info["n_sub"], "n_r": h.info["n_r"],
           "sum_sub_dofs": info["sum_sub_dofs"], "sum_sub_tri": info["sum_sub_tri"],
           "n_box_entries": info["n_box_entries"],
           "coarse_solver": {v: k for k, v in cgs.COARSE.items()}[info["coarse_solver"]], "xxt_nnz": info["xxt_nnz"],
           "coarse_operator": args.coarse_operator, "ar_nnz": info["ar_nnz"],
           "footprint_mb": h.info["footprint_bytes"] / 2 ** 20, "setup_s": setup_s, "iters": its,
           "relres": rels, "ms_per_solve": float(np.mean(ms[1:] if len(ms) > 1 else ms))}
    if args.sequence > 0:
        # b_k = b + 0.05 sin(0.3 k) b1 + 0.02 k b2: a time series of right-hand sides
        rng = np.random.default_rng(17)
        b1, b2 = rng.standard_normal(m.nv), rng.standard_normal(m.nv)
        seq = [bd + torch.as_tensor(0.05 * np.sin(0.3 * k) * b1 + 0.02 * k * b2, device="cuda")
               for k in range(args.sequence)]
        res = {}
        for mode, l in (("plain", 0), ("projected", args.projection)):
            cgs.cgs_mesh_set_projection(h.handle, l)
            its_s, ms_s, rels = [], [], []
            for bk in seq:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                st, it, rel = cgs.cgs_solve(h.handle, bk, x, rtol=args.rtol, maxit=args.maxit)
                e1.record()
                torch.cuda.synchronize()
                its_s.append(int(it[0]))
                ms_s.append(e0.elapsed_time(e1))
                rels.append(float(rel[0]))
            res[mode] = {"iters": its_s, "ms_per_solve": float(np.mean(ms_s)), "max_relres": max(rels)}
        cgs.cgs_mesh_set_projection(h.handle, 0)
        out["sequence"] = {"n": args.sequence, "kept": args.projection, **res}
    if args.profile:
        out["profile"] = cgs.cgs_profile_read(h.handle)
    if args.compare_fp64 and args.prec != "fp64":
        with cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64", form=args.form,
                      coarse=args.coarse) as h64:
            x64 = torch.empty_like(bd)
            st, it, rel = cgs.cgs_solve(h64.handle, bd, x64, rtol=args.rtol, maxit=args.maxit)
            torch.cuda.synchronize()
            out["fp64"] = {"iters": int(it[0]), "relres": float(rel[0]),
                           "rel_diff_x": float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))}
    print(json.dumps(out))
    h.free()
    cgs.cgs_destroy(ctx)


if __name__ == "__main__":
    main()
