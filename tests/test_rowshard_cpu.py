"""The row-sharded multi-GPU design of the hot path, run as two gloo ranks on
the CPU: rows of A split unevenly between the ranks, the small partials (s,
U^T C, the CGS2 second projection, both CholeskyQR Grams, A^T U, the sign
dots) summed with all_reduce, the draws replicated.  Every round's draws must
equal the single-rank oracle's, and the gathered modes and singular values
must agree with it to FP64 rounding.  With row sampling (ICRS) the row
draws each rank resolves, put together, must be the oracle's."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
M, N = 601, 90
SPLIT = 277          # rank 0 holds rows [0, 277), rank 1 rows [277, 601)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _matrix():
    from paper_1905_05107_gb300 import synth
    return synth.planted(M, N, 0.8 ** np.arange(30), 1e-6, 41, np.float64)


def _worker(rank, world, port, strategy, rows, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle import isma as O
    import rowshard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A = _matrix()
        r0, r1 = (0, SPLIT) if rank == 0 else (SPLIT, M)
        p = O.Params(k=5, c=12, col_strategy=strategy, tol=1e-8, rows=rows, w=300)
        U, sig, draws, meas, rdraws = rowshard.isma_sharded(A[r0:r1], M, r0, p)
        q.put((rank, U, sig, [d.tolist() for d in draws], meas,
               [(rr.tolist(), cc.tolist()) for rr, cc in rdraws]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("strategy,rows", [("unf", 0), ("ort", 0), ("unf", 1)])
def test_row_sharded_isma_matches_single_rank_oracle(strategy, rows):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, strategy, rows, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in range(2)), key=lambda x: x[0])
    for pr in procs:
        pr.join(timeout=60)
    assert all(pr.exitcode == 0 for pr in procs)

    from oracle import isma as O
    A = _matrix()
    ref = O.isma(A, O.Params(k=5, c=12, col_strategy=strategy, tol=1e-8, rows=rows, w=300))
    (_, U0, s0, d0, m0, rd0), (_, U1, s1, d1, m1, rd1) = res
    # replicated quantities agree across ranks exactly
    assert d0 == d1 and m0 == m1
    np.testing.assert_array_equal(s0, s1)
    # and with the single-rank oracle
    assert len(d0) == len(ref.trace)
    for t, rec in enumerate(ref.trace):
        assert d0[t] == rec.idx.tolist(), t
        assert abs(m0[t] - rec.sin_max) <= 1e-9, t
        if rows:
            # the two ranks' row draws together are the oracle's, bit for bit
            got_rows = rd0[t][0] + rd1[t][0]
            got_counts = rd0[t][1] + rd1[t][1]
            assert got_rows == rec.rows.tolist(), t
            assert got_counts == rec.row_counts.tolist(), t
            assert all(r < SPLIT for r in rd0[t][0]) and all(r >= SPLIT for r in rd1[t][0])
    np.testing.assert_allclose(s0, ref.sigma, rtol=1e-10)
    U = np.vstack([U0, U1])
    assert O.sin_principal_max(ref.U, U) <= 1e-9
    np.testing.assert_allclose(U, ref.U, atol=1e-8)
