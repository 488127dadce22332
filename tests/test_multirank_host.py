"""Multi-rank host logic on the CPU (gloo, world size 2): bench.py runs one
replica per GPU and reports the units of all ranks over the slowest rank's
time.  No GPU and no collective on the data path are involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        # rank r processed 1000 * (r + 1) units in (r + 1) seconds, end to end 2 (r + 1)
        got = bench.reduce_over_ranks(1000 * (r + 1), float(r + 1), 2.0 * (r + 1), w, torch.device("cpu"))
        q.put((r, w, local, got))
    finally:
        dist.destroy_process_group()


def test_two_replicas_sum_units_and_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, w, local, got) in enumerate(results):
        assert (r, w, local) == (rank, world, rank)
        assert got == (3000.0, 2.0, 4.0)  # every rank sees the whole-job figures


def test_single_rank_passes_through():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(7, 1.5, 2.5, 1, None) == (7.0, 1.5, 2.5)
