"""Host logic of bench.py's multi-process runs (CPU, gloo, world size 2).

The path does not shard (every rank runs its own domain), so the only
exchange is the timing reduction: each rank's times are replaced by the
maximum over ranks, and the job's rate counts the cell updates of all ranks
over that slowest time. The reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist = bench.init_dist(world, "gloo")
    times = bench.max_over_ranks(dist, [10.0 + rank, 5.0 - rank, 1.0 * rank], "cpu")
    value = bench.job_glups(world, 1000, 4, times[0])
    out.put((rank, times, value))
    dist.barrier()
    dist.destroy_process_group()


def test_timing_is_the_maximum_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, times, value in got:
        assert times == [11.0, 5.0, 1.0]
        # 2 ranks x 1000 cells x 4 steps over the slowest 11 ms
        assert value == pytest.approx(2 * 1000 * 4 / 11e-3 / 1e9)


def test_single_process_keeps_its_own_times():
    pytest.importorskip("torch")
    assert bench.max_over_ranks(None, [3.0, 2.0], "cpu") == [3.0, 2.0]
    assert bench.job_glups(1, 512 ** 3, 200, 1000.0) == pytest.approx(512 ** 3 * 200 / 1e9)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun a non-zero rank of the reference arm exits 0 at once,
    printing nothing and running no oracle work."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "3", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_one_line_on_rank_zero():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "GLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
