"""The benchmark's multi-rank plumbing on CPU with the gloo backend and two
ranks: process-group set-up, the barrier, the slowest rank's time reaching
every rank, the whole-job rate over all ranks, and the reference arm running
once on rank 0 only (the other ranks exit without work)."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    sys.path.insert(0, ROOT)
    import bench

    d = bench.dist_init(world, "gloo")
    bench.barrier(d)
    ms = bench.max_over_ranks(d, 10.0 * (rank + 1), "cpu")  # rank r "took" 10 (r + 1) ms
    v = bench.whole_job_rate(1000, world, ms)
    bench.dist_finish(d)
    q.put((rank, ms, v))


def test_two_gloo_ranks_share_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for _, ms, v in out:
        assert ms == 20.0  # the slower rank's time on both
        assert v == pytest.approx(1000 * 2 / 0.020 / 1e6)  # units of both ranks over the job time


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.dist_init(1, "gloo") is None
    assert bench.max_over_ranks(None, 12.5, "cpu") == 12.5
    assert bench.whole_job_rate(3e6, 1, 1000.0) == pytest.approx(3.0)
    bench.barrier(None)
    bench.dist_finish(None)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
