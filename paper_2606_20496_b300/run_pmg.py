"""Time the p-multigrid wrap (Sec. 1, Sec. 5, Eqs. (13) and (14)) on one
workload through the C ABI: flexible GMRES on the order-N spectral-element
Poisson problem, the additive multilevel preconditioner with the two-level
Schwarz solver as its order-1 level.

    python -m paper_2606_20496_b300.run_pmg [--small] [--solves 3]

Prints one JSON line: levels, set-up time, iterations, solve time, and the
per-step event times with the rates they reach.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

# FP64 FMA issue rate of B300: 2 per clock per SM, 148 SMs, 2032 MHz
FP64_PEAK_TFLOPS = 2 * 2 * 148 * 2.032e9 / 1e12
# FP32 instruction issue rate: 128 lanes per clock per SM
FP32_PEAK_TOPS = 128 * 148 * 2.032e9 / 1e12
# FP32 instructions per node of the float-pair operator: 57 pair
# multiply-adds of 12 instructions (two-product 4, two-sum 6, 2 adds) and six
# renormalisations of 3
PAIR_OPS_PER_NODE = 57 * 12 + 6 * 3


def sem_flops_bytes(p: int, ne: int, ng: int, ng_c: int = 0, pc: int = 0) -> dict:
    """Algorithmic float64 flops and bytes of one launch of each step on a
    level with p nodes per direction (a multiply-add counts 2 flops)."""
    p3, p4 = p ** 3, p ** 4
    out = {
        # Dhat (3 p^4 multiply-adds), the metric (15 flops per node), Dhat^T (3 p^4)
        "ax": {"flops": ne * (12 * p4 + 15 * p3), "bytes": ne * (6 * 8 * p3 + 4 * p3) + ng * (8 + 8)},
        # S^T and S along three directions (6 p^4), the diagonal and W (2 per node)
        "fdm": {"flops": ne * (12 * p4 + 2 * p3),
                "bytes": ne * (3 * 8 * p * p + 3 * 8 * p + 4 * p3) + ng * (8 + 8 + 8)},
    }
    if pc:
        # three contractions of decreasing size, p^3 pc + p^2 pc^2 + p pc^3 multiply-adds
        f = 2 * (p3 * pc + p * p * pc * pc + p * pc ** 3)
        b = ne * (4 * p3 + 4 * pc ** 3) + ng * 16 + ng_c * 8
        out["restrict"] = {"flops": ne * f, "bytes": b}
        out["prolong"] = {"flops": ne * f, "bytes": b}
    return out


def run(ctx, small: bool = False, solves: int = 3, rtol: float = 1e-8, restart: int = 30, prec: str = "fp64"):
    import torch

    from . import cgs, meshes
    m, orders = meshes.workload_sem_small() if small else meshes.workload_sem()
    t0 = time.perf_counter()
    h = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec)
    t1 = time.perf_counter()
    g = cgs.PMG(h, m.xyz, m.conn, orders)
    t2 = time.perf_counter()
    levels = g.levels
    n0 = levels[0]["n_nodes"]
    b = torch.as_tensor(meshes.sem_rhs(cgs.cgs_pmg_node_coords(g.handle, 0)), device="cuda")
    x = torch.zeros(n0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def events(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # solves: events around each solve (the call synchronises at its end)
    its, rels, ms = [], [], []
    cgs.cgs_pmg_solve(g.handle, b, x, rtol=rtol, maxit=500, restart=restart)
    for _ in range(solves):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, it, rel = cgs.cgs_pmg_solve(g.handle, b, x, rtol=rtol, maxit=500, restart=restart)
        e1.record(stream)
        torch.cuda.synchronize()
        assert st == cgs.OK, st
        its.append(it)
        rels.append(rel)
        ms.append(e0.elapsed_time(e1))
    # single steps on every level: each launch's mean event time (memset of the
    # output included) and the rate it reaches
    steps = {}
    for l in range(len(orders)):
        n_l = levels[l]["n_nodes"]
        p = orders[l] + 1
        pc = (orders[l + 1] + 1) if l + 1 < len(orders) else 2
        n_c = levels[l + 1]["n_nodes"]
        u = torch.randn(n_l, dtype=torch.float64, device="cuda")
        y = torch.empty_like(u)
        uc = torch.randn(n_c, dtype=torch.float64, device="cuda")
        yc = torch.empty_like(uc)
        fb = sem_flops_bytes(p, m.ne, n_l, n_c, pc)
        reps = 20
        t = {"ax": events(lambda: cgs.cgs_pmg_apply_A(g.handle, l, u, y), reps),
             "fdm": events(lambda: cgs.cgs_pmg_smooth(g.handle, l, u, y), reps),
             "restrict": events(lambda: cgs.cgs_pmg_restrict(g.handle, l, u, yc), reps),
             "prolong": events(lambda: cgs.cgs_pmg_prolong(g.handle, l, uc, y), reps)}
        for k, v in t.items():
            steps[f"{k}_N{orders[l]}"] = {
                "ms": v, "tflops": fb[k]["flops"] / (v * 1e-3) / 1e12,
                "fp64_frac": fb[k]["flops"] / (v * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                "gbs": fb[k]["bytes"] / (v * 1e-3) / 1e9, "flops": fb[k]["flops"], "bytes": fb[k]["bytes"]}
        if prec != "fp64":   # the operator in float pairs: FP32 instructions
            ops = m.ne * p ** 3 * PAIR_OPS_PER_NODE
            steps[f"ax_N{orders[l]}"].update({"pair_ops": ops, "tops": ops / (t["ax"] * 1e-3) / 1e12,
                                               "fp32_frac": ops / (t["ax"] * 1e-3) / 1e12 / FP32_PEAK_TOPS})
    r = torch.randn(n0, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    m_ms = events(lambda: cgs.cgs_pmg_apply_preconditioner(g.handle, r, z), 10)
    out = {"workload": ("cube32 deformed (32^3 hexes), spectral elements of order %d, schedule %s -> 1, "
                        "%d nodes" % (orders[0], " -> ".join(map(str, orders)), n0)) if not small else
           "cube8 perturbed, order %d" % orders[0],
           "orders": list(orders), "levels": levels, "coarse_prec": prec,
           "setup_s": {"mesh": t1 - t0, "pmg": t2 - t1},
           "iters": int(np.median(its)), "relres": float(max(rels)), "rtol": rtol, "restart": restart,
           "ms_per_solve": float(np.median(ms)), "solves_per_s": 1e3 / float(np.median(ms)),
           "dofs_per_s": n0 * 1e3 / float(np.median(ms)),
           "precond_ms": m_ms, "steps": steps}
    g.free()
    h.free()
    return out


def profile_target(ctx, mode: str, prec: str, maxit: int, small: bool = False) -> dict:
    """A short run for a profiler: `solve` = one GMRES solve of at most maxit
    products (restart 30); `steps` = three launches each of the finest
    level's operator and smoother."""
    import torch

    from . import cgs, meshes
    m, orders = meshes.workload_sem_small() if small else meshes.workload_sem()
    h = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec)
    g = cgs.PMG(h, m.xyz, m.conn, orders)
    b = torch.as_tensor(meshes.sem_rhs(cgs.cgs_pmg_node_coords(g.handle, 0)), device="cuda")
    y = torch.empty_like(b)
    out = {"mode": mode, "prec": prec}
    if mode == "solve":
        st, its, rel = cgs.cgs_pmg_solve(g.handle, b, y, rtol=1e-12, maxit=maxit, restart=30)
        out.update({"iters": its, "relres": rel})
    else:
        for _ in range(3):
            cgs.cgs_pmg_apply_A(g.handle, 0, b, y)
        for _ in range(3):
            cgs.cgs_pmg_smooth(g.handle, 0, b, y)
    torch.cuda.synchronize()
    g.free()
    h.free()
    return out


def main():
    from . import build, cgs
    ap = argparse.ArgumentParser()
    ap.add_argument("--small", action="store_true")
    ap.add_argument("--solves", type=int, default=3)
    ap.add_argument("--prec", default="fp64",
                    help="coarse mesh precision; fp32/fp16 also run the smoothers and transfers in float")
    ap.add_argument("--only", choices=("solve", "steps"), default=None,
                    help="a short run for a profiler: one solve (--maxit products) or three launches per step")
    ap.add_argument("--maxit", type=int, default=8)
    args = ap.parse_args()
    build.build()
    ctx = cgs.cgs_create(0)
    if args.only:
        print(json.dumps(profile_target(ctx, args.only, args.prec, args.maxit, args.small)))
    else:
        print(json.dumps(run(ctx, args.small, args.solves, prec=args.prec)))
    cgs.cgs_destroy(ctx)


if __name__ == "__main__":
    main()
