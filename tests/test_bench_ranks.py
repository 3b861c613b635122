"""The multi-rank path of bench.py on CPU (gloo, world size 2): the timing is
the slowest rank's, the rate counts every rank's cell updates, and the
reference arm runs on rank 0 only."""
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


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench._dist()
    slowest = bench._max_over_ranks(1.5 + rank, w)      # rank 1 is the slow one
    rate = bench._aggregate_rate(1000.0, 10, slowest, w)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, r, w, slowest, rate))


def test_two_ranks_take_the_slowest_time_and_count_all_cells():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, slowest, rate in out:
        assert r == rank and w == 2
        assert slowest == 2.5
        assert rate == pytest.approx(1000.0 * 10 * 2 / 2.5 / 1e9)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.0, 1) == 3.0
    assert bench._aggregate_rate(4.0, 5, 2.0, 1) == pytest.approx(10.0 / 1e9)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
