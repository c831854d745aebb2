"""The multi-rank paths of bench.py on the CPU: two gloo ranks on 127.0.0.1.

Each rank contributes a different time; both must see the maximum (the
slowest rank bounds the whole job) and compute the same whole-job rate.  The
reference arm under torchrun runs on rank 0 only: rank 1 returns at once
without touching the oracle, rank 0 prints one JSON line.
"""
import contextlib
import io
import json
import os
import socket
import sys
import types

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = bench.max_over_ranks(dist, 10.0 + 5.0 * rank, "cpu")
    rate = bench.whole_job_rate(world, 100, ms)
    dist.barrier()
    # reference arm: rank 0 only (the oracle timing replaced by a stub)
    called = []

    def fake_problem():
        called.append(rank)
        return None, None, 0.0

    bench.oracle_iters_per_solve = lambda: 5
    bench.oracle_problem = fake_problem
    bench.oracle_step = lambda P, b: 0.1          # 0.1 s per iteration, 5 per solve: 2 solves/s
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(types.SimpleNamespace(gpus=world, steps=3, warmup=0))
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ms": ms, "rate": rate, "called": called, "stdout": buf.getvalue()}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_rank0_reference(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    assert r[0]["ms"] == r[1]["ms"] == 15.0
    assert r[0]["rate"] == r[1]["rate"] == pytest.approx(2 * 100 / 15e-3)
    assert r[0]["called"] == [0] and r[1]["called"] == []
    assert r[1]["stdout"] == ""
    line = json.loads(r[0]["stdout"].strip())
    assert line["impl"] == "reference" and line["value"] == pytest.approx(2.0) and line["n_gpus"] == 2
