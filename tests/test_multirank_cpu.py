"""The N > 1 path of bench.py (independent replicas, one problem per GPU):
the timed value is the maximum over ranks, every rank gets the same value,
and only rank 0 runs the oracle arm.  World size 2 on the gloo backend, CPU
only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 17.25][rank]
        got = bench.max_over_ranks(ms, world, torch.device("cpu"))
        bench.barrier(world)
        r, w, lr = bench.dist_env()

        class Args:
            gpus, steps, warmup = world, 1, 0
        # the oracle arm: rank 0 alone would run it; the other ranks exit at once
        rc = bench.run_reference(Args()) if rank != 0 else None
        q.put((rank, got, (r, w, lr), rc))
    finally:
        dist.destroy_process_group()


def test_replica_timing_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(2))
    assert [x[1] for x in res] == [17.25, 17.25]
    assert res[0][2] == (0, 2, 0) and res[1][2] == (1, 2, 1)
    assert res[1][3] == 0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
