"""Serving benchmark: a Poisson stream of coarse-solve requests.

    python -m paper_2606_20496_b300.serve [--rate 2000] [--seconds 10] [--pool 64] [--slots 256] [--arena-mb 2048]

A pool of meshes (unit cubes or hollow cylinders with k^3 elements, k drawn
log-uniformly in [8, 64] with seed 3; cylinders graded like the 1M-vertex
cylinder with inner-wall aspect ratio 10) is set up once and stays resident on
the device (the operator cache).  Requests arrive as a Poisson process of the
given rate; each picks a pool mesh and a fresh N(0,1) right-hand side and is
solved to 1e-8.  The continuous-batching server admits arriving requests
into free slots while others iterate, all running slots sharing each launch;
a request is admitted when a slot is free and its vectors fit the server's
arena (admission by device-memory footprint).
Latency is measured from arrival to completion on the wall clock; the same
stream is then replayed through the plain FP64 per-request path (one solve
at a time, first come first served).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def make_pool(n: int, seed: int = 3, kmax: int = 64):
    from . import meshes
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(n):
        cyl = rng.random() < 0.5
        k = int(round(np.exp(rng.uniform(np.log(8), np.log(kmax)))))
        b = int(min(max(-(-k // 4), 2), 16))
        if cyl:
            m = meshes.cylinder(k, max(k, 8), k, grading=1.05 ** (64.0 / k), aspect=10.0, boxes=(b, b, b),
                                name=f"cyl{k}")
        else:
            m = meshes.cube(k, perturb=0.15, seed=[seed, i], boxes=(b, b, b), name=f"cube{k}")
        pool.append(m)
    return pool


def arrivals(rate: float, seconds: float, npool: int, seed: int = 3):
    rng = np.random.default_rng([seed, 1])
    t = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * seconds * 1.2) + 16))
    t = t[t < seconds]
    which = rng.integers(0, npool, size=t.size)
    return t, which


def percentile(a, q):
    return float(np.percentile(np.asarray(a), q)) if len(a) else None


def run_server(ctx, hs, pool, t_arr, which, slots, iters_per_step, rtol, prec, arena_mb):
    import torch

    from . import cgs
    max_nr = max(h.info["n_r"] for h in hs)
    # vector arena: 56 bytes per vertex entry; the reduced space per slot
    pool_nv = max(int(arena_mb * 2 ** 20 / 56), max(m.nv for m in pool))
    server = cgs.cgs_server_create(ctx, slots, pool_nv, slots * max_nr, prec=prec, rtol=rtol)
    peak_use, active_sum = 0, 0
    gen = torch.Generator(device="cuda")
    n = t_arr.size
    lat = np.full(n, np.nan)
    its = np.zeros(n, np.int32)
    pending = {}
    nxt = 0
    steps = 0
    t0 = time.perf_counter()
    done = 0
    while done < n:
        now = time.perf_counter() - t0
        while nxt < n and t_arr[nxt] <= now:
            m = pool[which[nxt]]
            gen.manual_seed(1000003 * 3 + nxt)
            b = torch.randn(m.nv, dtype=torch.float64, device="cuda", generator=gen)
            x = torch.empty_like(b)
            tk = cgs.cgs_submit(server, hs[which[nxt]], b, x)
            pending[tk] = (nxt, b, x)
            nxt += 1
        if pending:
            active, _, _ = cgs.cgs_server_step(server, iterations=iters_per_step)
            steps += 1
            active_sum += active
            peak_use = max(peak_use, cgs.cgs_server_stats(server)["bytes_in_use"])
            tnow = time.perf_counter() - t0
            for tk, it, rel, st in cgs.cgs_server_drain(server):
                i, _, _ = pending.pop(tk)
                lat[i] = tnow - t_arr[i]
                its[i] = it
                assert st == cgs.OK and rel <= rtol * 1.5, (st, rel)
                done += 1
        elif nxt < n:
            time.sleep(max(0.0, min(1e-3, t_arr[nxt] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    launches = cgs.cgs_server_launches(server)
    arena = cgs.cgs_server_stats(server)["arena_bytes"]
    cgs.cgs_server_free(server)
    return {"p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
            "mean_ms": 1e3 * float(np.nanmean(lat)), "solves_per_s": n / wall, "wall_s": wall,
            "steps": steps, "iters_mean": float(its.mean()), "kernel_launches": int(launches),
            "arena_mb": arena / 2 ** 20, "peak_arena_mb_in_use": peak_use / 2 ** 20,
            "mean_active_after_step": active_sum / max(steps, 1)}


def run_plain(ctx, h64, pool, t_arr, which, rtol, budget_s):
    """FIFO single-request path: each request solved alone in arrival order."""
    import torch

    from . import cgs
    gen = torch.Generator(device="cuda")
    n = t_arr.size
    lat = []
    t0 = time.perf_counter()
    served = 0
    for i in range(n):
        now = time.perf_counter() - t0
        if t_arr[i] > now:
            time.sleep(t_arr[i] - now)
        m = pool[which[i]]
        gen.manual_seed(1000003 * 3 + i)
        b = torch.randn(m.nv, dtype=torch.float64, device="cuda", generator=gen)
        x = torch.empty_like(b)
        st, it, rel = cgs.cgs_solve(h64[which[i]].handle, b, x, rtol=rtol)
        lat.append(time.perf_counter() - t0 - t_arr[i])
        served += 1
        if time.perf_counter() - t0 > budget_s:
            break
    wall = time.perf_counter() - t0
    return {"p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
            "solves_per_s": served / wall, "served": served, "of": int(n), "wall_s": wall}


def serve(rate=2000.0, seconds=10.0, pool_n=64, slots=256, iters_per_step=4, rtol=1e-8, prec="fp32",
          plain=True, kmax=64, arena_mb=2048.0, plain_budget_s=None):
    import torch

    from . import build, cgs
    build.build()
    pool = make_pool(pool_n, kmax=kmax)
    ctx = cgs.cgs_create(0)
    t0 = time.perf_counter()
    hs = [cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec=prec) for m in pool]
    setup_s = time.perf_counter() - t0
    t_arr, which = arrivals(rate, seconds, len(pool))
    # warm-up: one request per pool mesh through a small server
    run_server(ctx, hs, pool, np.zeros(len(pool)), np.arange(len(pool)), min(slots, len(pool)), iters_per_step,
               rtol, prec, arena_mb)
    torch.cuda.synchronize()
    ours = run_server(ctx, hs, pool, t_arr, which, slots, iters_per_step, rtol, prec, arena_mb)
    out = {"workload": f"Poisson stream {rate:g} req/s for {seconds:g} s over a pool of {len(pool)} cube/cylinder "
                       f"meshes (k^3 elements, k log-uniform in [8, {kmax}], seed 3), rtol {rtol:g}",
           "requests": int(t_arr.size), "pool_elements": int(sum(m.ne for m in pool)), "setup_s": setup_s,
           "server": {"slots": slots, "iters_per_step": iters_per_step, "prec": prec, **ours}}
    for h in hs:
        h.free()
    if plain:
        h64 = [cgs.Mesh(ctx, m.xyz, m.conn, part=m.part, boxes=m.boxes, prec="fp64") for m in pool]
        for i in range(len(pool)):   # warm-up (graphs)
            b = torch.ones(pool[i].nv, dtype=torch.float64, device="cuda")
            cgs.cgs_solve(h64[i].handle, b, torch.empty_like(b), rtol=rtol)
        out["fp64_plain_per_request"] = run_plain(ctx, h64, pool, t_arr, which, rtol,
                                                  budget_s=plain_budget_s or 3 * seconds)
        for h in h64:
            h.free()
    cgs.cgs_destroy(ctx)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--pool", type=int, default=64)
    ap.add_argument("--slots", type=int, default=256)
    ap.add_argument("--arena-mb", type=float, default=2048.0, help="vector arena for admission by footprint")
    ap.add_argument("--iters-per-step", type=int, default=4)
    ap.add_argument("--kmax", type=int, default=64)
    ap.add_argument("--prec", default="fp32")
    ap.add_argument("--no-plain", action="store_true")
    a = ap.parse_args()
    print(json.dumps(serve(a.rate, a.seconds, a.pool, a.slots, a.iters_per_step, prec=a.prec, plain=not a.no_plain,
                           kmax=a.kmax, arena_mb=a.arena_mb)))


if __name__ == "__main__":
    main()
