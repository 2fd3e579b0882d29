"""Row-sharded ISMA on torch.distributed ranks (test infrastructure).

The multi-GPU design of the hot path shards the rows of A (and of U) across
ranks: every rank holds rows [m0, m1) of every column.  Each step then needs
one exchange, a fixed-order sum of small partials:

* column squared norms (Eq. 2): local partials of s, summed (n values);
* the draws (Algorithm 1, GET UPDATE) are replicated: every rank computes the
  same integer weights from the same s and the same Philox counters, so no
  broadcast is needed;
* BLOCK MERGE (Algorithm 2): P = U^T C, the second projection P2 = U^T Z and
  the two CholeskyQR Grams G1 = Z^T Z, G2 = W^T W are local partials summed
  across ranks; the Cholesky factors, the core E (Eq. 8) and its SVD (Eq. 9)
  are replicated; U is updated on local rows only;
* ORT values (Eq. 6) and the closing refinement need A^T U: local partials
  summed (n x r);
* the sign reference of the output modes: local dots summed;
* ICRS row sampling (SAMPLE AND SCALE UNIQUE ROWS): the largest row value
  (for the integer weights) is a max-reduction, the ranks' weight totals are
  gathered, and each row draw is resolved by the rank whose part of the
  prefix sums holds it; the Gram W^T W of the scaled rows is a sum of local
  partials, its SVD (V_r) replicated, C = D V_r formed on local rows.

The arithmetic is FP64 NumPy, the same steps the CUDA kernels take (CGS2 and
CholeskyQR2 for the residual block, explicit Q = Z R1^{-1} R2^{-1}), written
here only to check that the sharded exchanges reproduce the single-rank
result.  The sampling helpers are the oracle's; nothing here is imported by
the library.
"""
import numpy as np
import torch
import torch.distributed as dist

from oracle import isma as O


def allreduce(x: np.ndarray) -> np.ndarray:
    """Sum of a FP64 array over all ranks (gloo all_reduce)."""
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def allreduce_max(x: float) -> float:
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allgather_int(v: int) -> list:
    t = torch.tensor([int(v)], dtype=torch.int64)
    out = [torch.zeros(1, dtype=torch.int64) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return [int(x.item()) for x in out]


def sample_scale_rows_sharded(D_local: np.ndarray, values_local: np.ndarray, w: int, seed: int, t: int,
                              m_global: int, row0: int):
    """SAMPLE AND SCALE UNIQUE ROWS (Algorithm 1) over row shards: the same
    integer weights, draws and scaling as the single-rank oracle, with the
    weights' maximum and total reduced across ranks.  Returns this rank's
    scaled rows of W, their global indices and counts."""
    L = O.weight_bits(m_global)
    vmax = allreduce_max(values_local.max() if values_local.size else 0.0)
    if vmax > 0:
        wq = np.floor(np.ldexp(np.asarray(values_local, dtype=np.float64) / vmax, L)).astype(np.uint64)
    else:
        wq = np.zeros(values_local.shape[0], dtype=np.uint64)
    totals = allgather_int(int(wq.sum(dtype=np.uint64)))
    if sum(totals) == 0:                        # uniform over all rows
        wq = np.ones(values_local.shape[0], dtype=np.uint64)
        totals = allgather_int(int(wq.sum(dtype=np.uint64)))
    total = sum(totals)
    offset = sum(totals[:dist.get_rank()])
    cdf = np.cumsum(wq, dtype=np.uint64)
    hits = []
    for u in O.uniform_u64(seed, t, O.STREAM_ROWS, w):
        v = (u * total) >> 64
        if offset <= v < offset + totals[dist.get_rank()]:
            hits.append(int(np.searchsorted(cdf, np.uint64(v - offset), side="right")))
    rows, counts = np.unique(np.asarray(hits, dtype=np.int64), return_counts=True)
    q = wq[rows].astype(np.float64) / float(total)
    scale = np.sqrt(counts / (w * q)) if rows.size else np.zeros(0)
    return D_local[rows, :] * scale[:, None], rows + row0, counts


def merge_sharded(U: np.ndarray, s1: np.ndarray, C: np.ndarray, r: int, m_global: int):
    """BLOCK MERGE with local rows of U and C (Algorithm 2, Eqs. 8-9)."""
    r1, g = U.shape[1], C.shape[1]
    P = allreduce(U.T @ C)
    Z = C - U @ P
    P2 = allreduce(U.T @ Z)
    Z = Z - U @ P2
    G1 = allreduce(Z.T @ Z)
    R1 = np.linalg.cholesky(G1).T
    W = np.linalg.solve(R1.T, Z.T).T          # Z R1^{-1}
    G2 = allreduce(W.T @ W)
    R2 = np.linalg.cholesky(G2).T
    Q = np.linalg.solve(R2.T, W.T).T          # W R2^{-1}
    E = np.zeros((r1 + g, r1 + g))
    E[:r1, :r1] = np.diag(s1)
    E[:r1, r1:] = P + P2
    E[r1:, r1:] = R2 @ R1
    UE, sE, _ = np.linalg.svd(E)
    if sE.size == 0 or sE[0] == 0:
        keep = 0
    else:
        thresh = max(m_global, r1 + g) * np.finfo(np.float64).eps * sE[0]
        keep = min(r, int(np.count_nonzero(sE > thresh)))
    Unew = np.hstack([U, Q]) @ UE[:, :keep]
    return Unew, sE[:keep].copy(), UE


def isma_sharded(A_local: np.ndarray, m_global: int, row0: int, p: "O.Params"):
    """Algorithm 1 on this rank's rows (ICS, or ICRS with L2N row values when
    p.rows == 1); returns (local U, sigma, column draws per round, measures
    per round, this rank's (rows, counts) per round)."""
    n = A_local.shape[1]
    r = p.carried_rank()
    s = allreduce(np.einsum("ij,ij->j", A_local, A_local))
    in_S = np.ones(n, dtype=bool)
    U = np.zeros((A_local.shape[0], 0))
    sig = np.zeros(0)
    draws, measures, row_draws = [], [], []
    t = 0
    while True:
        if t > 0 and p.col_strategy == "ort":
            Y = allreduce(A_local.T @ U)
            vals = np.maximum(0.0, s - np.sum(Y * Y, axis=1))
        else:
            vals = O.column_values("l2n" if t == 0 else p.col_strategy, t, s, None, None)
        idx, _ = O.sample_columns(vals, in_S, p.c, p.seed, t)
        in_S[idx] = False
        D = A_local[:, idx]
        if p.rows == 1:
            wdraws = p.w if p.w > 0 else min(m_global, O.rows_eq5(p.k, 0.6, 0.6))
            W, rows, counts = sample_scale_rows_sharded(D, np.sum(D * D, axis=1), wdraws, p.seed, t,
                                                        m_global, row0)
            Vg, _, _ = np.linalg.svd(allreduce(W.T @ W))
            D = D @ Vg[:, :r]
            row_draws.append((rows, counts))
        r_prev = U.shape[1]
        U, sig, UE = merge_sharded(U, sig, D, r, m_global)
        sin_max, _ = O.convergence_measures(UE, p.k, r_prev)
        draws.append(idx)
        measures.append(sin_max)
        t += 1
        if (t > 1 and r_prev >= p.k and sin_max <= p.tol) or not in_S.any():
            break
    if p.refine and U.shape[1] > 0:
        Y = allreduce(A_local.T @ U)
        _, R = np.linalg.qr(Y, mode="reduced")
        _, SR, VRt = np.linalg.svd(R)
        U, sig = U @ VRt.T, SR
    kk = min(p.k, U.shape[1])
    U, sig = U[:, :kk], sig[:kk]
    z = O.sign_reference(p.seed, m_global)[row0:row0 + U.shape[0]]
    sgn = np.sign(allreduce(U.T @ z))
    sgn[sgn == 0] = 1.0
    return U * sgn, sig, draws, measures, row_draws
