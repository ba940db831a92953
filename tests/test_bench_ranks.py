"""The multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2)
agree on the slowest rank's time and on the whole-job throughput, and the
reference arm runs on rank 0 only.  Replicas share nothing on the data path,
so the timing reduction is the only collective."""
import json
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def _rank_main(rank, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, str(ROOT))
    import torch

    import bench
    dist, r, ws = bench._dist()
    assert dist.get_backend() == "gloo"
    bench._barrier(dist, torch)
    my_seconds = 2.0 if r == 0 else 3.5
    slowest = bench._max_over_ranks(dist, torch, my_seconds)
    value = bench.whole_job_gvox_s(512 ** 3, 10, ws, slowest)
    dist.destroy_process_group()
    q.put((r, ws, slowest, value))


def test_two_gloo_ranks_take_the_slowest_time():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = 512 ** 3 * 10 * 2 / 3.5 / 1e9
    for r, (rank, ws, slowest, value) in enumerate(res):
        assert (rank, ws, slowest) == (r, 2, 3.5)
        assert value == pytest.approx(want)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    p = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0
    assert p.stdout.strip() == ""


def test_whole_job_value_counts_all_replicas():
    sys.path.insert(0, str(ROOT))
    import bench
    one = bench.whole_job_gvox_s(1 << 27, 4, 1, 0.5)
    assert bench.whole_job_gvox_s(1 << 27, 4, 4, 0.5) == pytest.approx(4 * one)
    assert one == pytest.approx((1 << 27) * 4 / 0.5 / 1e9)
    assert json.dumps(one)


def test_gpus_flag_must_match_the_ranks():
    """--gpus N under a launcher that started a different number of ranks is
    refused (no rank silently runs a one-GPU job)."""
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--gpus", "2", "--steps", "1"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 2
    assert "WORLD_SIZE=1" in r.stderr
