#!/usr/bin/env python
"""Coarse-solve throughput of the two-level Schwarz PCG solver on one B300.

Workload: the 32^3 smoothly deformed unit cube with randomly renumbered
elements (35,937 vertices, 4,096 overlapping 2^3-element subdomains, 8^3 box
coarse space), hybrid Schwarz (ASM_1 + ASM_2) inside flexible PCG to a
relative residual of 1e-8.  One step = one complete coarse solve of one
N(0,1) right-hand side.  The headline form is FP32 bulk / FP64 outer; the FP64
plain form runs beside it for the iteration-count comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun, one rank per GPU) every rank solves its own replica of
the workload (the path has no data exchange between problems), and value is
the aggregate over ranks.  --impl reference times the FP64 CPU oracle on the
same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coarse-solve apps/s & PCG iters to 1e-8 vs FP64 plain; p50/p99 serve latency"
UNIT = "solves/s"
RTOL = 1e-8
L2_FLUSH_BYTES = 256 << 20


def workload():
    from paper_2606_20496_b300 import meshes
    return meshes.workload_cube32()


def config_block(extra=None):
    c = {"workload": "cube32_deformed_permuted: 32^3 trilinear hexes, 35,937 vertices, elements renumbered "
                     "by a seeded permutation, 4,096 2^3-element subdomains grown by one layer, 8^3 boxes; "
                     "hybrid Schwarz (ASM_1+ASM_2) in flexible PCG to rtol 1e-8, one N(0,1) RHS per step",
         "form": "hybrid", "precision": "fp32 bulk (local solves, inner A, J, J^T), fp64 outer PCG and A_r^-1",
         "rtol": RTOL, "l2": "flushed between steps (256 MB device write outside the timed events)"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes per launch of each kernel class (HBM roofline)
# ---------------------------------------------------------------------------

def algorithmic_bytes(info, prec, interp_cells=False):
    """Bytes each kernel class must move at least once per launch: every
    mandatory array once, each gathered vertex value once, padding not
    counted.  Mixed forms (fp32/fp16): float-pair outer vectors (8 B),
    float-pair element matrices (28 x 8 B), lane-pack local solves; FP64 form:
    float64 everything.  interp_cells: the interpolation runs over the
    cell-sorted entries (z added to once per entry) and the dots kernel
    reads z, r, q (and clears q in the mixed forms)."""
    E, nv, nr = info["ne"], info["nv"], info["n_r"]
    sm = info["sum_sub_dofs"]
    nb = info["n_box_entries"]
    sb = 8 if prec == "fp64" else 4
    sl = {"fp64": 8, "fp32": 4, "fp16": 2}[prec]
    packed = info["_packed_entries"]
    # reduced solve per launch: the dense inverse once, or one XX^T pass (X's
    # 8-byte values and 2-byte indices once, r_r or t gathered, t or u_r out)
    xnnz = info.get("xxt_nnz", 0)
    coarse = xnnz * 10 + nr * 12 if info.get("coarse_solver") == 2 else nr * nr * 8 + nr * 12
    if prec == "fp64":
        return {
            "apply_A64": E * (36 * 8 + 32) + nv * (8 + 16),
            "local": packed * sl + sm * 4 + nv * (8 + 2 * sb + sb),
            "restrict": nb * 16 + nv * (32 + sb) + nr * 16,
            "coarse": coarse + (nr * 4 if info.get("coarse_solver") != 2 else 0),
            "interp": (nb * 16 + nv * (32 + 2 * sb) + nr * 8) if interp_cells
            else nb * 16 + nv * (4 + 32 + 2 * sb + 16) + nr * 8,
            "pcg_xr": nv * (8 * 6 + 2 * sb),
            "pcg_dots": nv * (sb + 16),
            "pcg_p": nv * (sb + 24),
        }
    return {
        # q = A p: hi/lo off-diagonals and 16-bit local indices per element;
        # p and z gathered (p = z + beta p on the fly), q written, once per vertex
        "apply_A64": E * (28 * 8 + 16) + nv * (8 + sb + 8),
        # s -= A l: float off-diagonals and indices; l read, s read and written
        "apply_A32": E * (28 * 4 + 16) + nv * (4 + 2 * 4),
        # upper triangles, vertex ids, W_ov; r gathered, z read and written
        "local": packed * sl + sm * 4 + nv * (4 + sb + 2 * sb),
        # (vertex, cell, weight) entries; coordinates and s per vertex; r_r pairs
        "restrict": nb * 12 + nv * (16 + sb) + nr * 8,
        # per-vertex lists, coordinates, z read and written, r and q pairs
        # read (dots), q cleared
        "interp": (nb * 12 + nv * (16 + 2 * sb) + nr * 4) if interp_cells
        else nv * 8 + nb * 8 + nv * (16 + 2 * sb + 16 + 8) + nr * 4,
        "coarse": coarse,
        # p, q, x, r read; p, x, r written; z read and cleared; s written
        "pcg_xr": nv * (8 * 7 + 3 * sb),
        # z, r and q read, q cleared
        "pcg_dots": nv * (sb + 16 + 8),
        "pcg_p": nv * (sb + 24),
    }


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def traffic_for(kernel_class):
    """dram read+write bytes per launch from a committed ncu summary, if one
    exists for the current kernel source (kernels.cu; else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        ent = d.get("kernels", {}).get(kernel_class)
        if not ent:
            return None
        import hashlib
        h = hashlib.sha256(open(os.path.join(ROOT, "paper_2606_20496_b300", "csrc", "kernels.cu"), "rb").read())
        h = h.hexdigest()[:16]
        return ent["bytes_per_launch"] if ent.get("source_hash") == h else None
    except Exception:
        return None


# ---------------------------------------------------------------------------
# the CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def time_oracle(budget_s=15.0, max_solves=None):
    """Time complete oracle solves in a fresh single-threaded interpreter
    (BLAS/OpenMP pools pinned to one thread through the environment)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(budget_s), str(max_solves or 0)]
    res = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=budget_s * 4 + 300)
    if res.returncode:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: " + res.stderr[-300:]}
    return json.loads(res.stdout.strip().splitlines()[-1])


def oracle_sample(budget_s, max_solves):
    from oracle import cgs_oracle as O
    m, b = workload()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    times, iters = [], []
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        x, its, rel, ok = P.solve(b, rtol=RTOL)
        times.append(time.perf_counter() - t0)
        iters.append(its)
        if time.perf_counter() - t_all >= budget_s or (max_solves and len(times) >= max_solves):
            break
    print(json.dumps({"value": len(times) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
                      "sample": f"{len(times)} complete FP64 oracle solves of the same workload (numpy/scipy, "
                                f"one thread, setup excluded), {sum(times):.1f} s; iters {iters[0]}"}))


def max_over_ranks(dist, value: float, device: str) -> float:
    """The maximum of `value` over all ranks (the slowest rank's time); the
    value itself without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, ms_max: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank / (ms_max * 1e-3)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sample = time_oracle(budget_s=90.0, max_solves=max(1, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": sample["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / sample["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_block({"precision": "fp64 (CPU oracle)"}),
            "cpu_baseline": sample,
            "e2e": {"value": sample["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def serve_probe(ctx, args):
    """Continuous-batching server on a Poisson stream (this rank's replica):
    pool meshes drawn like the serving workload (cubes and cylinders with
    k^3 elements, k log-uniform in [8, 64], seed 3), FP32 bulk to 1e-8,
    latency from arrival to completion on the wall clock."""
    from paper_2606_20496_b300 import cgs, serve
    import torch
    pool = serve.make_pool(args.serve_pool)
    hs = [cgs.Mesh(ctx, mm.xyz, mm.conn, part=mm.part, boxes=mm.boxes, prec="fp32") for mm in pool]
    try:
        # warm-up: every pool mesh once
        serve.run_server(ctx, hs, pool, np.zeros(len(pool)), np.arange(len(pool)), min(256, len(pool)), 8,
                         RTOL, "fp32", 2048.0)
        torch.cuda.synchronize()
        t_arr, which = serve.arrivals(args.serve_rate, args.serve_seconds, len(pool))
        r = serve.run_server(ctx, hs, pool, t_arr, which, 256, 8, RTOL, "fp32", 2048.0)
    finally:
        for h in hs:
            h.free()
    return {"p50": r["p50_ms"], "p99": r["p99_ms"], "solves_per_s": r["solves_per_s"],
            "offered_req_per_s": args.serve_rate, "requests": int(t_arr.size), "seconds": args.serve_seconds,
            "workload": f"Poisson stream over {len(pool)} cube/cylinder meshes, k^3 elements, k log-uniform in "
                        "[8, 64] (seed 3), one N(0,1) RHS per request, rtol 1e-8, FP32 bulk",
            "server": {"slots": 256, "iters_per_step": 8, "arena_mb": 2048, "mean_active": r["mean_active_after_step"]}}


def run_ours(args):
    import torch

    from paper_2606_20496_b300 import build as B
    from paper_2606_20496_b300 import cgs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    B.build()
    m, b = workload()
    ctx = cgs.cgs_create(local)
    h32 = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp32")
    h64 = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64")
    # the library's autotuner picks the block sizes on this mesh (untimed setup)
    cgs.cgs_mesh_tune(h32.handle)
    cgs.cgs_mesh_tune(h64.handle)
    sched = cgs.cgs_mesh_get_schedule(h32.handle)
    sched64 = cgs.cgs_mesh_get_schedule(h64.handle)
    bd = torch.as_tensor(b, dtype=torch.float64, device="cuda")
    x = torch.empty_like(bd)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(h, steps, warmup):
        for _ in range(warmup):
            cgs.cgs_solve(h.handle, bd, x, rtol=RTOL)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        its = []
        n0 = cgs.cgs_mesh_info(h.handle)["kernel_launches"]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        wall0 = time.perf_counter()
        for s in range(steps):
            flush.zero_()
            ev[s][0].record(stream)
            st, it, rel = cgs.cgs_solve(h.handle, bd, x, rtol=RTOL)
            ev[s][1].record(stream)
            its.append(int(it[0]))
            assert st == cgs.OK and rel[0] <= 1.5 * RTOL, (st, rel)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        launches = cgs.cgs_mesh_info(h.handle)["kernel_launches"] - n0
        ms = max_over_ranks(dist, sum(a.elapsed_time(c) for a, c in ev), "cuda")
        if dist:
            dist.barrier()
        return ms, its, launches, wall

    with ClockSampler(local) as clk:
        ms32, its32, launches32, wall32 = timed(h32, args.steps, args.warmup)
    clocks = clk.summary()
    ms64, its64, _, _ = timed(h64, args.steps, args.warmup)

    # per-kernel event timing (separate pass, same workload and launches)
    def profile(h, n):
        cgs.cgs_profile_enable(h.handle, True)
        for _ in range(n):
            flush.zero_()
            cgs.cgs_solve(h.handle, bd, x, rtol=RTOL)
        prof = cgs.cgs_profile_read(h.handle)
        cgs.cgs_profile_enable(h.handle, False)
        return prof

    nprof = min(args.steps, 50)
    prof = profile(h32, nprof)
    info = dict(h32.info)
    info.update(cgs.cgs_mesh_info(h32.handle))
    info["_packed_entries"] = info["sum_sub_tri"]
    algo = algorithmic_bytes(info, "fp32", interp_cells=bool(sched.get("interp_cells")))
    iters32 = int(np.median(its32))
    # the persistent loop runs every phase of every iteration in one launch
    # (interpolating by vertex)
    per_iter = ["apply_A64", "pcg_xr", "local", "apply_A32", "restrict", "coarse", "interp"]
    by_vertex = algorithmic_bytes(info, "fp32")
    algo["loop"] = iters32 * sum(by_vertex[k] for k in per_iter)
    total_ms = sum(t for t, n in prof.values())
    dom = max((k for k in prof if k in algo and prof[k][1]), key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    achieved = algo[dom] / (dom_ms * 1e-3) / 1e9
    peaks, peak_kind = measured_peaks()
    traffic = traffic_for(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": algo[dom],
                "avg_launch_us": dom_ms * 1e3}
    if dom == "loop":
        roofline["note"] = (f"persistent loop: {iters32} iterations per launch, algorithmic bytes = iterations x "
                            "(q = A p, x/r/p update, local solves, s -= A l, restriction, reduced solve, "
                            "interpolation with the dots)")
    shares = {k: {"share": round(t / total_ms, 4), "launches": n, "avg_us": round(1e3 * t / n, 2)}
              for k, (t, n) in prof.items() if n}
    # the same solves one launch per phase (per-phase attribution)
    p0 = cgs.cgs_mesh_get_schedule(h32.handle)["persistent"]
    cgs.cgs_mesh_set_schedule(h32.handle, persistent=0)
    prof_s = profile(h32, nprof)
    cgs.cgs_mesh_set_schedule(h32.handle, persistent=p0)
    total_s = sum(t for t, n in prof_s.values())
    shares_stepwise = {k: {"share": round(t / total_s, 4), "launches": n, "avg_us": round(1e3 * t / n, 2),
                           "achieved_gbs": round(algo[k] / (t / n * 1e-3) / 1e9, 1) if k in algo else None}
                       for k, (t, n) in prof_s.items() if n}

    # end to end through the host-buffer entry point
    bh = torch.empty(m.nv, dtype=torch.float64, pin_memory=True)
    bh.copy_(torch.as_tensor(b))
    xh = torch.empty(m.nv, dtype=torch.float64, pin_memory=True)
    for _ in range(args.warmup):
        cgs.cgs_solve_host(h32.handle, bh, xh, rtol=RTOL)
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, it, rel = cgs.cgs_solve_host(h32.handle, bh, xh, rtol=RTOL)
        e2e_ms += (time.perf_counter() - t0) * 1e3
        assert st == cgs.OK
    e2e_ms = max_over_ranks(dist, e2e_ms, "cuda")

    serving = serve_probe(ctx, args) if args.serve_seconds > 0 else None

    line = None
    if rank == 0:
        ms_per_step = ms32 / args.steps
        value = whole_job_rate(world, args.steps, ms32)
        cpu = time_oracle(budget_s=args.cpu_seconds) if world == 1 else None
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": config_block({"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                        "schedule": sched}),
                "iters": {"fp32_bulk": int(np.median(its32)), "fp64_plain": int(np.median(its64)),
                          "delta": int(np.median(its32)) - int(np.median(its64))},
                "fp64_plain": {"value": whole_job_rate(world, args.steps, ms64), "unit": UNIT,
                               "ms_per_step": ms64 / args.steps, "schedule": sched64},
                "serve_latency_ms": serving,
                "roofline": roofline, "kernel_shares": shares, "kernel_shares_stepwise": shares_stepwise,
                "cpu_baseline": cpu,
                "e2e": {"value": whole_job_rate(world, args.steps, e2e_ms), "unit": UNIT,
                        "h2d_bytes_per_step": m.nv * 8, "d2h_bytes_per_step": m.nv * 8 + 16},
                "gpu_launches": int(launches32), "clocks": clocks,
                "impl": "ours"}
        print(json.dumps(line))
    h32.free()
    h64.free()
    cgs.cgs_destroy(ctx)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="serving probe length (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-pool", type=int, default=32)
    ap.add_argument("--oracle-sample", nargs=2, type=float, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:
        oracle_sample(args.oracle_sample[0], int(args.oracle_sample[1]))
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
