"""The N > 1 data path of bench.py: local rank 0 generates the headline
matrix once into /dev/shm and every rank maps that one host copy.  Two gloo
ranks on the CPU, at a reduced size: each rank's view must equal the matrix
the generator gives on its own, in the same Fortran order, and the file is
gone afterwards."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
M, N = 4096, 256


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, path = bench.shared_head(M, N, rank, world)
        ref = bench.make_head(M, N)
        same = A is not None and A.shape == ref.shape and bool(np.array_equal(np.asarray(A), ref))
        q.put((rank, path, same, bool(A is not None and A.flags["F_CONTIGUOUS"])))
        del A
        bench.barrier(world)
        if rank == 0 and path:
            os.remove(path)
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


@pytest.mark.skipif(not os.path.isdir("/dev/shm"), reason="no /dev/shm")
def test_replicas_share_one_host_copy_of_the_headline_matrix():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.spawn(_worker, args=(2, _free_port(), q), nprocs=2, join=True)
    got = sorted(q.get() for _ in range(2))
    paths = {g[1] for g in got}
    assert len(paths) == 1 and None not in paths
    assert all(g[2] for g in got), got
    assert all(g[3] for g in got), got
    assert not os.path.exists(paths.pop())
