"""Multi-rank path of bench.py on CPU: two gloo ranks, as torchrun starts them.

The workload shards into independent replicas (no data-path collective), so what
the ranks share is the job clock: the slowest rank's time, and the units of all
ranks divided by it.  The reference arm runs on rank 0 only.
"""

import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench

    w, r, local, dist = bench.dist_context("gloo")
    try:
        # rank r measured (10 + r) ms for the step loop and (30 - r) ms end to end
        t = bench.max_over_ranks(dist, [10.0 + r, 30.0 - r], device="cpu")
        rate = bench.job_rate(1000.0, w, t[0])
        # the reference arm prints on rank 0 only; other ranks return without work
        buf = io.StringIO()
        if r != 0:
            with redirect_stdout(buf):
                bench.run_reference(None, None)
        q.put((r, w, local, t, rate, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_job_time():
    import torch.multiprocessing as mp

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for r, w, local, t, rate, printed in out:
        assert w == world and local == r
        assert t == [11.0, 30.0]  # element-wise max: slowest step loop, slowest e2e
        assert rate == pytest.approx(2 * 1000.0 / 11e-3)
        assert printed == ""


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    w, r, local, dist = bench.dist_context("gloo")
    assert (w, r, local, dist) == (1, 0, 0, None)
    assert bench.max_over_ranks(None, [3, 4.5]) == [3.0, 4.5]
    assert bench.job_rate(50.0, 1, 2.0) == pytest.approx(25000.0)


def test_reference_line_keys(monkeypatch, oracle_lib):
    """The reference arm's JSON line on a tiny workload (FP64 oracle)."""
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    wl = bench.make_workload("sine", 16)
    args = argparse.Namespace(steps=3, warmup=3, cpu_budget=0.05)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, wl)
    d = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["unit"] == "GLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
