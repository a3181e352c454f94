"""The replicated (N > 1) bench path on CPU: two gloo ranks reduce their
timings the way bench.py does under torchrun (slowest rank's time, all
ranks' active cell-steps), and the reference arm prints only on rank 0."""
import json
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


def _worker(rank, world, port, ms, act, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        q.put((rank, bench.reduce_over_ranks(dist, ms[rank], act[rank], "cpu")))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_like_the_bench():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms, act = [41.5, 43.25], [2_000_000, 2_097_152]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ms, act, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert out[r] == (43.25, float(sum(act)))


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


@pytest.mark.timeout(600)
def test_reference_arm_line():
    """Rank 0 of the reference arm: one JSON line with the contract's keys."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-n", "8"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "active cell-steps/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["steps"] == 1 and line["cpu_baseline"]["steps"] == 1 and line["cpu_baseline"]["host"]["nproc"] >= 1


def test_casting_bands():
    """The casting study's binning: shares 1.0 and 0.8 fall in the top band,
    0.79 in the next, steps with no active cell in none; per band the mean
    step time, iterations, full setups and active cell-steps per second."""
    sys.path.insert(0, ROOT)
    import bench
    n = 1000
    rows = [(0.010, 1000, 20, 1), (0.012, 800, 22, 2), (0.008, 790, 18, 2), (0.004, 150, 10, 1), (0.002, 0, 0, 0)]
    b = bench.active_share_bands(rows, n)
    assert [x["active_share"] for x in b] == ["0.8-1.0", "0.6-0.8", "0.0-0.2"]
    assert [x["steps"] for x in b] == [2, 1, 1]
    assert b[0]["ms_per_step"] == 11.0 and b[0]["p_its"] == 21.0 and b[0]["rebuilds"] == 1
    assert abs(b[0]["active_cell_steps_per_s"] - 1800 / 0.022) < 0.1
    assert b[2]["rebuilds"] == 1 and abs(b[2]["active_cell_steps_per_s"] - 150 / 0.004) < 0.1
