"""Multi-rank logic of the benchmark on CPU (gloo, world size 2).

The fit itself has no collective: frames are independent and every rank runs
the same batch (replicas, weak scaling).  What the ranks share is the timing:
the job's time is the slowest rank's, and the job's rate counts the pixels of
every rank.  The reference arm runs on rank 0 only.
"""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    try:
        # per-rank step times: the slowest rank sets the job's time
        ms = bench.rank_max(1.0 + 0.5 * rank, world, torch.device("cpu"))
        rate = bench.whole_job_rate(world, 1000000, ms)
        q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_rank_max_and_whole_job_rate_gloo_world2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ms, rate in res:
        assert ms == 1.5                      # max over ranks, seen by every rank
        assert rate == pytest.approx(2 * 1e6 / 1.5e-3 / 1e6)  # both ranks' pixels over the max time


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.rank_max(3.25, 1, None) == 3.25
    assert bench.whole_job_rate(1, 2000000, 2.0) == pytest.approx(1000.0)


def test_reference_arm_runs_on_rank0_only():
    """Under torchrun every rank but 0 exits at once, without work and without output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
