#!/usr/bin/env python
"""Coarse-solve throughput of the two-level Schwarz PCG solver on one B300.

Headline workload: the hollow cylinder of 64 x 128 x 128 trilinear hexes
(1,073,280 vertices; radial grading 1.05, inner-wall aspect ratio 1:100;
131,072 overlapping 2^3-element subdomains; a 16^3 box coarse space with
3,876 active vertices), hybrid Schwarz (ASM_1 + ASM_2) inside flexible PCG to
a relative residual of 1e-8, in the plain FP64 form (every step in float64,
the precision of the paper's Schwarz solves).  One step = one complete coarse
solve of one N(0,1) right-hand side.  Beside it, on the same mesh: the FP32
bulk and FP16 local forms (rate, iterations, difference from the FP64
solution); the batched form (256 perturbed cubes x 4 right-hand sides in one
graph) against the FP64 per-request path; the serving form (a 10 s Poisson
stream at 2,000 req/s over a 64-mesh pool) against the FP64 per-request
path; and the p-multigrid wrap (GMRES on the order-7 spectral-element Poisson
problem of the 32^3 deformed cube, 11.4 M nodes, schedule 7 -> 3 -> 1, with
this solver as the order-1 level), with float64 and with float smoothers.

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
# FP64 FMA issue rate of B300: 2 per clock per SM (148 SMs, 2032 MHz maximum
# SM clock) -> 1.203 TFLOP/s; this repository's dependent-FMA probe measured
# 1.10 TFLOP/s, the nominal figure is 1.25
FP64_PEAK_TFLOPS = 2 * 2 * 148 * 2.032e9 / 1e12
WORKLOAD = ("hollow_cylinder_1M: 64 x 128 x 128 trilinear hexes (1,073,280 vertices), radial grading 1.05, "
            "inner-wall aspect 1:100, 131,072 2^3-element subdomains grown by one layer, 16^3 boxes "
            "(3,876 active vertices, XX^T reduced solve); hybrid Schwarz (ASM_1+ASM_2) in flexible PCG to "
            "rtol 1e-8, one N(0,1) RHS (seed 6) per step")


def workload():
    from paper_2606_20496_b300 import meshes
    return meshes.workload_cylinder()


def config_block(extra=None):
    c = {"workload": WORKLOAD, "form": "hybrid",
         "precision": "fp64 plain: every step in float64 (local solves, operator applies, J, J^T, XX^T, "
                      "PCG vectors and dots)",
         "rtol": RTOL, "l2": "inputs larger than L2: the mesh's resident data is 885 MB (126 MB L2), no flush"}
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
# algorithmic bytes and flops per launch of each kernel class
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
    packed = info["sum_sub_tri"]
    # reduced solve per launch: the dense inverse once, or one XX^T pass (X's
    # 8-byte values and 2-byte indices once, r_r or t gathered, t or u_r out)
    xnnz = info.get("xxt_nnz", 0)
    coarse = xnnz * 10 + nr * 12 if info.get("coarse_solver") == 2 else nr * nr * 8 + nr * 12
    nh = info.get("n_hyb_entries", 0)
    nj = info.get("n_jt_entries", 0)
    nvb = info.get("n_free", nv)
    # the row applies over the assembled A: column and value of every
    # nonzero once, x (or p) gathered once, y read and written once
    ell = info.get("ell_nnz", 0)
    if prec == "fp64":
        return {
            "apply_A64": ell * (4 + 8) + nv * (8 + 16) if ell else E * (36 * 8 + 32) + nv * (8 + 16),
            "local": packed * sl + sm * 4 + nv * (8 + 2 * sb + sb),
            # hybrid: (vertex, J~, A J~) entries, r and l gathered, r_r; else
            # the cell-sorted restriction of s
            "restrict": (nh * (4 + 16) + nv * 16 + nr * 8) if nh else nb * 16 + nv * (32 + sb) + nr * 16,
            "coarse": coarse + (nr * 4 if info.get("coarse_solver") != 2 else 0),
            # explicit J~ rows (column, weight), z read and written, r and q
            # read for the fused dots
            "interp": nj * 12 + nvb * 8 + nv * 32 + nr * 8,
            # x, p, r, q read; x, r, z written
            "pcg_xr": nv * (4 * 8 + 3 * 8),
            "pcg_dots": nv * (sb + 16),
            # z, p read; p, q written
            "pcg_p": nv * 32,
        }
    return {
        # q = A p: by rows, column and (hi, lo) value per nonzero, p gathered,
        # q written; else hi/lo off-diagonals and 16-bit local indices per
        # element, p and z gathered (p = z + beta p on the fly), q written
        "apply_A64": ell * (4 + 8) + nv * (8 + 8) if ell else E * (28 * 8 + 16) + nv * (8 + sb + 8),
        # s -= A l: float off-diagonals and indices; l read, s read and written
        "apply_A32": E * (28 * 4 + 16) + nv * (4 + 2 * 4),
        # upper triangles, vertex ids, W_ov; r gathered, z read and written
        "local": packed * sl + sm * 4 + nv * (4 + sb + 2 * sb),
        # hybrid: (vertex, J~, A J~) float entries, r and l gathered, r_r
        # pairs; else (vertex, cell, weight) entries, coordinates and s
        "restrict": (nh * (4 + 8) + nv * 8 + nr * 8) if nh else nb * 12 + nv * (16 + sb) + nr * 8,
        # per-vertex lists, coordinates, z read and written, r and q pairs
        # read (dots), q cleared
        "interp": (nb * 12 + nv * (16 + 2 * sb) + nr * 4) if interp_cells
        else nv * 8 + nb * 8 + nv * (16 + 2 * sb + 16 + 8) + nr * 4,
        "coarse": coarse,
        # p, q, x, r read; x, r (and p without the row apply) written; z read
        # and cleared; s written
        "pcg_xr": nv * (8 * (6 if ell else 7) + 3 * sb),
        # z, r and q read, q cleared
        "pcg_dots": nv * (sb + 16 + 8),
        # z read, p read and written (the row apply's p update)
        "pcg_p": nv * (sb + 16),
    }


def algorithmic_flops(info, prec):
    """Float64 flops per launch of the FP64-form kernels (an FMA counts 2): the
    operator by rows (one FMA per nonzero and one per row for p.Ap; 64 FMAs
    per element in the element form), the local solves (m_p^2 FMAs per
    subdomain), the hybrid restriction (2 FMAs per entry) and the
    interpolation by rows (1 FMA per entry, 2 per vertex for the dots)."""
    if prec != "fp64":
        return {}
    sum_m2 = 2 * info["sum_sub_tri"] - info["sum_sub_dofs"]
    ell = info.get("ell_nnz", 0)
    out = {"apply_A64": 2 * ell + 2 * info["nv"] if ell else 2 * 64 * info["ne"], "local": 2 * sum_m2}
    if info.get("n_hyb_entries"):
        out["restrict"] = 4 * info["n_hyb_entries"]
    if info.get("n_jt_entries"):
        out["interp"] = 2 * info["n_jt_entries"] + 4 * info.get("n_free", info["nv"])
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def traffic_for(kernel_class, workload_key, source="kernels.cu"):
    """dram read+write bytes per launch from a committed ncu summary, if one
    exists for this kernel class and workload, taken with the current kernel
    source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        ent = d.get(workload_key, {}).get(kernel_class)
        if not ent:
            return None
        import hashlib
        h = hashlib.sha256(open(os.path.join(ROOT, "paper_2606_20496_b300", "csrc", source), "rb").read())
        return ent["bytes_per_launch"] if ent.get("source_hash") == h.hexdigest()[:16] else None
    except Exception:
        return None


def roofline_of(prof, info, prec, interp_cells, peaks, peak_kind, workload_key):
    """Per-kernel achieved rates from the event profile, and the roofline
    object of the dominant (most time) kernel: HBM-bound unless its FP64-ALU
    fraction is the larger."""
    algo = algorithmic_bytes(info, prec, interp_cells)
    flops = algorithmic_flops(info, prec)
    total = sum(t for t, n in prof.values()) or 1.0
    per = {}
    for k, (t, n) in prof.items():
        if not n:
            continue
        us = 1e3 * t / n
        e = {"share": round(t / total, 4), "launches": n, "avg_us": round(us, 2)}
        if k in algo:
            gbs = algo[k] / (us * 1e-6) / 1e9
            e.update(achieved_gbs=round(gbs, 1), hbm_frac=round(gbs / peaks["hbm_gbs"], 3))
        if k in flops:
            tf = flops[k] / (us * 1e-6) / 1e12
            e.update(achieved_fp64_tflops=round(tf, 3), fp64_frac=round(tf / FP64_PEAK_TFLOPS, 3))
        per[k] = e
    dom = max((k for k in per if k in algo), key=lambda k: per[k]["share"])
    d = per[dom]
    if d.get("fp64_frac", 0.0) > d["hbm_frac"]:
        roof = {"bound": "alu", "kernel": dom, "achieved": d["achieved_fp64_tflops"], "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": d["fp64_frac"], "traffic": traffic_for(dom, workload_key),
                "peak_source": "derived: 2 FP64 FMA per clock per SM x 148 SMs x 2032 MHz (probe measured 1.10)",
                "algorithmic_flops_per_launch": flops[dom], "algorithmic_bytes_per_launch": algo[dom],
                "hbm_frac": d["hbm_frac"], "avg_launch_us": d["avg_us"]}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": d["achieved_gbs"], "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": d["hbm_frac"], "traffic": traffic_for(dom, workload_key),
                "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": algo[dom],
                "avg_launch_us": d["avg_us"]}
    return roof, per


# ---------------------------------------------------------------------------
# the CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def _oracle_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    return env


def oracle_iters_per_solve():
    """The oracle's own iteration count for this workload (hybrid, rtol 1e-8),
    stored by tests/golden/make_cylinder_golden.py from an oracle solve."""
    p = os.path.join(ROOT, "tests", "golden", "cylinder_oracle.json")
    return int(json.load(open(p))["solve"]["iters"])


def pmg_oracle_iters():
    """The oracle's GMRES products for the p-multigrid workload, stored by
    tests/golden/make_pmg_golden.py (None when the file is absent)."""
    p = os.path.join(ROOT, "tests", "golden", "pmg_oracle.json")
    return int(json.load(open(p))["solve"]["iters"]) if os.path.exists(p) else None


def start_oracle_sample(iters):
    """Start the cpu_baseline sample in a fresh single-threaded interpreter
    (it runs on the host cores while the GPU work proceeds)."""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(iters)]
    return subprocess.Popen(cmd, env=_oracle_env(), stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)


def finish_oracle_sample(proc, timeout=900):
    try:
        out, err = proc.communicate(timeout=timeout)
    except subprocess.TimeoutExpired:
        proc.kill()
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "timed out"}
    if proc.returncode:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: " + err[-300:]}
    return json.loads(out.strip().splitlines()[-1])


def oracle_problem():
    from oracle import cgs_oracle as O
    m, b = workload()
    t0 = time.perf_counter()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    return P, b, time.perf_counter() - t0


def oracle_step(P, b):
    """One preconditioned flexible-PCG iteration of the oracle (its solve
    with maxit = 1: z = M r, q = A p, the x, r update, and the true-residual
    product at the end); returns seconds."""
    t0 = time.perf_counter()
    P.solve(b, rtol=RTOL, maxit=1)
    return time.perf_counter() - t0


def oracle_sample(iters):
    """cpu_baseline: the oracle on the full cylinder, a bounded sample of 6
    iterations (about 20 s on one core; set-up excluded), scaled to solves/s
    by the oracle's own iteration count per solve."""
    P, b, setup_s = oracle_problem()
    ts = [oracle_step(P, b) for _ in range(6)]
    t = float(np.median(ts))
    print(json.dumps({"value": 1.0 / (t * iters), "unit": UNIT, "cores": 1, "kind": "oracle",
                      "sample": f"{len(ts)} preconditioned PCG iterations of the FP64 oracle (numpy/scipy, one "
                                f"thread) on the same cylinder, median {t:.2f} s each, scaled by the oracle's "
                                f"{iters} iterations per solve (tests/golden/cylinder_oracle.json); oracle "
                                f"set-up {setup_s:.0f} s excluded"}))


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
    """The oracle, as it stands, on the host cores: set-up untimed, then W + K
    steps of one preconditioned PCG iteration each; value = solves/s, the
    mean step time scaled by the oracle's iterations per solve."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    iters = oracle_iters_per_solve()
    P, b, setup_s = oracle_problem()
    for _ in range(args.warmup):
        oracle_step(P, b)
    ts = [oracle_step(P, b) for _ in range(args.steps)]
    t = float(np.mean(ts))
    value = 1.0 / (t * iters)
    sample = (f"{args.steps} timed steps (after {args.warmup} warm-up) of one preconditioned PCG iteration of the "
              f"FP64 oracle (numpy/scipy, one thread), mean {t:.2f} s, scaled by its {iters} iterations per solve; "
              f"set-up {setup_s:.0f} s excluded")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_block({"precision": "fp64 (CPU oracle)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the CPU baseline runs on the host cores while the GPU work proceeds
    # (started before the first CUDA call)
    cpu_proc = start_oracle_sample(oracle_iters_per_solve()) if (rank == 0 and world == 1 and
                                                                  args.cpu_baseline) else None
    import torch

    from paper_2606_20496_b300 import build as B
    from paper_2606_20496_b300 import cgs

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    B.build()
    m, b = workload()
    ctx = cgs.cgs_create(local)
    stream = torch.cuda.current_stream()
    bd = torch.as_tensor(b, dtype=torch.float64, device="cuda")
    peaks, peak_kind = measured_peaks()

    def timed(h, steps, warmup, clocks=False):
        x = torch.empty_like(bd)
        for _ in range(warmup):
            cgs.cgs_solve(h.handle, bd, x, rtol=RTOL)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        its = []
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.__enter__()
        for s in range(steps):
            ev[s][0].record(stream)
            st, it, rel = cgs.cgs_solve(h.handle, bd, x, rtol=RTOL)
            ev[s][1].record(stream)
            its.append(int(it[0]))
            assert st == cgs.OK and rel[0] <= 1.5 * RTOL, (st, rel)
        torch.cuda.synchronize()
        if sampler:
            sampler.__exit__(None, None, None)
        ms = max_over_ranks(dist, sum(a.elapsed_time(c) for a, c in ev), "cuda")
        if dist:
            dist.barrier()
        return ms, its, x, (sampler.summary() if sampler else None)

    def profile(h, n):
        """Per-kernel-class CUDA-event times over n solves (host-driven loop,
        events on the launching stream); also the kernels one solve launches."""
        x = torch.empty_like(bd)
        cgs.cgs_profile_enable(h.handle, True)
        for _ in range(n):
            cgs.cgs_solve(h.handle, bd, x, rtol=RTOL)
        prof = cgs.cgs_profile_read(h.handle)
        cgs.cgs_profile_enable(h.handle, False)
        return prof, sum(nl for _, nl in prof.values()) / n

    # ---- headline: FP64 plain form ------------------------------------------------
    h64 = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64")
    cgs.cgs_mesh_tune(h64.handle)
    sched64 = cgs.cgs_mesh_get_schedule(h64.handle)
    ms64, its64, x64, clocks = timed(h64, args.steps, args.warmup, clocks=True)
    x64 = x64.clone()
    prof64, launches_per_solve = profile(h64, 2)
    info64 = dict(h64.info)
    info64.update(cgs.cgs_mesh_info(h64.handle))
    roofline, kernels64 = roofline_of(prof64, info64, "fp64", bool(sched64["interp_cells"]), peaks, peak_kind,
                                      "hollow_cylinder_1M_fp64")

    # end to end through the host-buffer entry point (H2D of b and D2H of x in
    # the timed region)
    bh = torch.empty(m.nv, dtype=torch.float64, pin_memory=True)
    bh.copy_(torch.as_tensor(b))
    xh = torch.empty(m.nv, dtype=torch.float64, pin_memory=True)
    for _ in range(2):
        cgs.cgs_solve_host(h64.handle, bh, xh, rtol=RTOL)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_ms = 0.0
    e2e_steps = max(3, args.steps // 2)
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        st, it, rel = cgs.cgs_solve_host(h64.handle, bh, xh, rtol=RTOL)
        e2e_ms += (time.perf_counter() - t0) * 1e3
        assert st == cgs.OK
    e2e_ms = max_over_ranks(dist, e2e_ms, "cuda")
    h64.free()

    # ---- the reduced-precision forms on the same mesh --------------------------------
    forms = {}
    for prec in ("fp32", "fp16"):
        h = cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec)
        cgs.cgs_mesh_tune(h.handle)
        sch = cgs.cgs_mesh_get_schedule(h.handle)
        ms, its, x, _ = timed(h, args.steps, max(2, args.warmup // 2))
        prof, _ = profile(h, 2)
        info = dict(h.info)
        info.update(cgs.cgs_mesh_info(h.handle))
        roof, per = roofline_of(prof, info, prec, bool(sch["interp_cells"]), peaks, peak_kind,
                                f"hollow_cylinder_1M_{prec}")
        forms[prec] = {"value": whole_job_rate(world, args.steps, ms), "unit": UNIT,
                       "ms_per_step": ms / args.steps, "iters": int(np.median(its)),
                       "iters_delta_vs_fp64": int(np.median(its)) - int(np.median(its64)),
                       "x_rel_diff_vs_fp64": float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64)),
                       "schedule": sch, "roofline": roof, "kernels": per}
        h.free()

    # ---- the p-multigrid wrap: order-7 SEM levels around the coarse solve -------------
    pmg = None
    if args.pmg:
        from paper_2606_20496_b300 import run_pmg
        pmg = {"iters_oracle": pmg_oracle_iters()}
        for prec in ("fp64", "fp32"):
            r = run_pmg.run(ctx, solves=3, prec=prec)
            ax = r["steps"]["ax_N%d" % r["orders"][0]]
            if prec == "fp64":
                r["roofline"] = {"kernel": "sem_ax_kernel<%d>" % (r["orders"][0] + 1), "bound": "alu",
                                 "achieved": ax["tflops"], "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                 "frac": ax["fp64_frac"],
                                 "traffic": traffic_for("sem_ax", "pmg_cube32_order7", "sem.cu"),
                                 "peak_note": "FP64 FMA issue rate, 2 per clock per SM at 2032 MHz"}
            else:
                r["roofline"] = {"kernel": "sem_ax_pair_kernel<%d>" % (r["orders"][0] + 1), "bound": "alu",
                                 "achieved": ax["tops"], "peak": run_pmg.FP32_PEAK_TOPS,
                                 "unit": "T FP32 instructions/s", "frac": ax["fp32_frac"],
                                 "traffic": traffic_for("sem_ax_pair", "pmg_cube32_order7", "sem.cu"),
                                 "peak_note": "FP32 issue rate, 128 lanes per clock per SM at 2032 MHz; "
                                              "instructions counted per node of the pair arithmetic"}
            pmg["fp64_smoothers" if prec == "fp64" else "fp32_smoothers"] = r

    # ---- batched form (256 meshes x 4 right-hand sides in one graph) -----------------
    batch = None
    if args.batch:
        from paper_2606_20496_b300 import run_batch
        batch = run_batch.run(ctx, 256, 4, "fp32", RTOL, reps=3, plain=True, plain_budget_s=args.plain_seconds)
    cgs.cgs_destroy(ctx)

    # ---- serving form ----------------------------------------------------------------
    serving = None
    if args.serve_seconds > 0:
        from paper_2606_20496_b300 import serve
        serving = serve.serve(rate=args.serve_rate, seconds=args.serve_seconds, pool_n=args.serve_pool, slots=256,
                              iters_per_step=8, rtol=RTOL, prec="fp32", plain=True,
                              plain_budget_s=args.plain_seconds)

    if rank == 0:
        value = whole_job_rate(world, args.steps, ms64)
        cpu = finish_oracle_sample(cpu_proc) if cpu_proc else None
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms64 / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config_block({"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                        "schedule": sched64}),
                "iters": {"fp64_plain": int(np.median(its64)), "fp32_bulk": forms["fp32"]["iters"],
                          "fp16_local": forms["fp16"]["iters"],
                          "delta_fp32": forms["fp32"]["iters_delta_vs_fp64"],
                          "delta_fp16": forms["fp16"]["iters_delta_vs_fp64"],
                          "oracle": oracle_iters_per_solve()},
                "fp32_bulk": forms["fp32"], "fp16_local": forms["fp16"],
                "batch": batch, "serve": serving, "pmg": pmg,
                "roofline": roofline, "kernels": kernels64,
                "cpu_baseline": cpu,
                "e2e": {"value": whole_job_rate(world, e2e_steps, e2e_ms), "unit": UNIT,
                        "h2d_bytes_per_step": m.nv * 8, "d2h_bytes_per_step": m.nv * 8 + 16},
                "gpu_launches": int(round(launches_per_solve * args.steps)),
                "gpu_launches_note": "kernels per solve counted in a profiled solve (the graph loop runs the same "
                                     "kernels) x timed solves",
                "clocks": clocks, "impl": "ours"}
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false", help="skip the batched form")
    ap.add_argument("--no-pmg", dest="pmg", action="store_false", help="skip the p-multigrid wrap")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="serving stream length (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--plain-seconds", type=float, default=10.0,
                    help="time budget of each FP64 per-request comparison (batch, serving)")
    ap.add_argument("--oracle-sample", type=int, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample is not None:
        oracle_sample(args.oracle_sample)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
