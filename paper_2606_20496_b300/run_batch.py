"""Batched coarse solves: many meshes and right-hand sides per launch.

    python -m paper_2606_20496_b300.run_batch [--count 256] [--nrhs 4] [--prec fp32] [--reps 5]

Builds the batched workload (perturbed cubes with edges of 4..24 elements
drawn with seed 2, mixed 2/3-element subdomains, 4 N(0,1) right-hand sides
each), solves every (mesh, right-hand side) pair to 1e-8 through one batch
(one launch per kernel per PCG iteration for all slots, device-side loop),
and times the same solves through the plain FP64 per-request path (one
cgs_solve per right-hand side).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def run(ctx, count=256, nrhs=4, prec="fp32", rtol=1e-8, reps=5, plain=True, tune=False, plain_budget_s=None):
    """Time the batched solves (median of `reps` after one warm-up) and, if
    `plain`, the same (mesh, right-hand side) pairs through the FP64
    per-request path (all of them, or as many as fit `plain_budget_s`
    seconds).  Returns the result dict."""
    import torch

    from . import cgs, meshes
    work = meshes.workload_batch(count)
    t0 = time.perf_counter()
    hs = [cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec) for m, _ in work]
    setup_s = time.perf_counter() - t0
    bs, xs = [], []
    for (m, B), h in zip(work, hs):
        for r in range(nrhs):
            bs.append(torch.as_tensor(B[r % B.shape[0]], dtype=torch.float64, device="cuda"))
            xs.append(torch.empty(m.nv, dtype=torch.float64, device="cuda"))
    t0 = time.perf_counter()
    batch = cgs.cgs_batch_create(ctx, hs, nrhs)
    create_s = time.perf_counter() - t0
    if tune:
        cgs.cgs_batch_tune(batch)
    st, its, rel, sts = cgs.cgs_batch_solve(batch, bs, xs, rtol=rtol)   # warm-up (builds the graph)
    assert st == cgs.OK, cgs.status_string(st)
    times = []
    n0 = cgs.cgs_batch_launches(batch)
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, its, rel, sts = cgs.cgs_batch_solve(batch, bs, xs, rtol=rtol)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        assert st == cgs.OK and np.all(rel <= 1.5 * rtol)
    launches = (cgs.cgs_batch_launches(batch) - n0) / reps
    nslots = len(bs)
    ms = float(np.median(times))
    out = {"workload": f"batch: {count} perturbed cubes (edge 4..24, seed 2) x {nrhs} RHS",
           "prec": prec, "slots": nslots, "elements": int(sum(m.ne for m, _ in work)),
           "vertices": int(sum(m.nv for m, _ in work)), "setup_s": setup_s, "batch_create_s": create_s,
           "ms_per_batch": ms, "solves_per_s": nslots / (ms * 1e-3),
           "iters": {"min": int(its.min()), "max": int(its.max()), "mean": float(its.mean())},
           "graph_launches_per_batch": launches, "max_relres": float(rel.max())}
    cgs.cgs_batch_free(batch)
    for h in hs:
        h.free()
    if plain:
        h64 = [cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64") for m, _ in work]
        for s in range(min(8, nslots)):   # warm-up: graphs of the first meshes
            cgs.cgs_solve(h64[s // nrhs].handle, bs[s], xs[s], rtol=rtol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its64 = []
        for s in range(nslots):
            st, it, r = cgs.cgs_solve(h64[s // nrhs].handle, bs[s], xs[s], rtol=rtol)
            its64.append(int(it[0]))
            if plain_budget_s and time.perf_counter() - t0 > plain_budget_s:
                break
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - t0
        k = len(its64)
        out["fp64_plain_per_request"] = {"solves_per_s": k / plain_s, "s_total": plain_s, "solves": k,
                                         "iters_mean": float(np.mean(its64))}
        out["iters_vs_plain_max_abs_delta"] = int(np.max(np.abs(np.array(its64) - its[:k])))
        for h in h64:
            h.free()
    return out


def main():
    from . import build, cgs
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--nrhs", type=int, default=4)
    ap.add_argument("--prec", default="fp32", choices=list(cgs.PREC))
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--no-plain", action="store_true", help="skip the FP64 per-request comparison")
    ap.add_argument("--tune", action="store_true")
    args = ap.parse_args()
    build.build()
    ctx = cgs.cgs_create(0)
    out = run(ctx, args.count, args.nrhs, args.prec, args.rtol, args.reps, not args.no_plain, args.tune)
    print(json.dumps(out))
    cgs.cgs_destroy(ctx)


if __name__ == "__main__":
    main()
