"""Plain FP64 CPU oracle of the iterative sampling-and-merging POD (ISMA).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code with
the CUDA library; the two meet only at the seeded input generators.

What it follows (arXiv 1905.05107, Charumathi, Ramakrishna, Vasudevan):

* Algorithm 1 (ISMA, GET UPDATE, SAMPLE AND SCALE UNIQUE ROWS), Sec. 3.
* Sec. 3.1 sampling strategies: column L2-norm probabilities (Eq. 2), uniform
  (UNF), orthogonal complement (ORT, Eq. 6); row L2 norms and leverage scores.
* Algorithm 2 (BLOCK MERGE / merge-and-truncate), Eqs. 8-9, Sec. 3.2.
* The convergence test of Algorithm 1 (cosines of modes or principal cosines
  of the subspaces) and the closing refinement QR(A^T U), SVD(R).
* Algorithm 3 (incremental POD over column blocks), Sec. 4.2.
* Eq. 3 and Eq. 5 for default sample counts.
* The quality measure of Sec. 3.3 (Wedin's bound, Eq. 7).

Everything is NumPy FP64; LAPACK (``numpy.linalg.qr`` / ``svd``) serves as the
QR and SVD steps, exactly as the paper's SciPy/LAPACK runs did (Sec. 4).  The
QR is Householder, never CholeskyQR.

Readings where the paper is silent or ambiguous (each is repeated in the
design notes of the repository):

* Random draws use a counter-based Philox4x32-10 generator (Salmon et al.,
  SC'11), written here from its published definition, instead of NumPy's
  stateful generator, so that a second implementation can reproduce every
  draw.  Counter = (draw index j, iteration t, stream id, 0), key = (seed low
  32 bits, seed high 32 bits); stream 0 = column draws, 1 = row draws,
  3 = the sign-reference vector.  One 64-bit uniform per Philox call:
  u = (x0 << 32) | x1.
* Probabilities are quantised to integer weights before drawing so that the
  draw is pure integer arithmetic: w_j = floor((s_j / s_max) * 2^L) over the
  remaining set S, L = 62 - ceil(log2(n + 1)); a draw picks the smallest i
  whose inclusive prefix sum exceeds v = floor(u * W / 2^64), W = sum of w.
  If every remaining weight is zero the draw falls back to uniform over S.
* The draw set I_c is the sorted list of distinct draws; S loses I_c.
* "Direct merge" (default): the raw sampled columns D enter BLOCK MERGE as the
  new block's scaled factor U_2 Sigma_2.  This equals Algorithm 2 whenever the
  new block is not truncated, because [U_1 Sigma_1, D] and
  [U_1 Sigma_1, D V] share singular values and left vectors for orthogonal V.
  ``paper_literal=True`` instead truncates the new block to rank r through
  SVD(D^T D) as GET UPDATE does.
* With row sampling the new block's factor is D V~_r, with V~ from
  SVD(W^T W); the first round's orthonormalisation (QR of U~, SVD of R) is
  the merge into an empty basis.
* Convergence: sin(theta_i) are the singular values of U_E[k:, :k] (the part
  of the new top-k modes outside the old top-k span, in the basis [U Q]);
  cosines of the modes are |U_E[i, i]|.  The subspace criterion stops when
  max sin <= tol, the modes criterion when min |cos| >= tol.
* Singular values below max(m, n_c) * eps * sigma_1 count as zero when
  Algorithm 2 drops zero singular values.
* Mode signs: u_i^T z > 0 for z_i = int32(x0 of Philox(i, 0, 3, 0)) / 2^31.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# ----------------------------------------------------------------------------
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
# as 1, 2, 3", SC'11): two 32x32->64 multiplies per round, Weyl key schedule.
# ----------------------------------------------------------------------------
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

STREAM_COLS = 0
STREAM_ROWS = 1
STREAM_SIGN = 3


def philox4x32_10(x0, x1, x2, x3, k0, k1):
    """Ten Philox rounds on counter words x0..x3 (arrays of uint32 values)
    with key (k0, k1).  Returns the four output words as uint64 arrays."""
    x0 = np.asarray(x0, dtype=np.uint64) & MASK32
    x1 = np.asarray(x1, dtype=np.uint64) & MASK32
    x2 = np.asarray(x2, dtype=np.uint64) & MASK32
    x3 = np.asarray(x3, dtype=np.uint64) & MASK32
    k0 = np.uint64(k0 & MASK32)
    k1 = np.uint64(k1 & MASK32)
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    s32 = np.uint64(32)
    mask = np.uint64(MASK32)
    for _ in range(10):
        p0 = m0 * x0          # < 2^64, exact in uint64
        p1 = m1 * x2
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        k0 = np.uint64((int(k0) + PHILOX_W0) & MASK32)
        k1 = np.uint64((int(k1) + PHILOX_W1) & MASK32)
    return x0, x1, x2, x3


def seed_key(seed: int):
    return seed & MASK32, (seed >> 32) & MASK32


def uniform_u64(seed: int, t: int, stream: int, count: int) -> List[int]:
    """64-bit uniforms for draw indices j = 0..count-1 of iteration t."""
    k0, k1 = seed_key(seed)
    j = np.arange(count, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10(j, np.full(count, t), np.full(count, stream),
                                 np.zeros(count), k0, k1)
    return [(int(a) << 32) | int(b) for a, b in zip(x0, x1)]


def sign_reference(seed: int, m: int) -> np.ndarray:
    """z_i = int32(x0) / 2^31 from Philox(i, 0, STREAM_SIGN, 0)."""
    k0, k1 = seed_key(seed)
    i = np.arange(m, dtype=np.uint64)
    x0, _, _, _ = philox4x32_10(i, np.zeros(m), np.full(m, STREAM_SIGN),
                                np.zeros(m), k0, k1)
    return x0.astype(np.uint32).view(np.int32).astype(np.float64) / 2.0 ** 31


# ----------------------------------------------------------------------------
# Sample counts, Eq. 3 (columns, LTSVD) and Eq. 5 (columns = rows, CTSVD)
# ----------------------------------------------------------------------------
def columns_eq3(k: int, eps: float, delta: float) -> int:
    return int(math.ceil(4 * k * (1 + math.sqrt(8 * math.log(1 / delta))) ** 2 / eps ** 2))


def rows_eq5(k: int, eps: float, delta: float) -> int:
    return int(math.ceil(k * k * (1 + math.sqrt(math.log(2 / delta))) ** 2 / eps ** 4))


# ----------------------------------------------------------------------------
# Integer weights and draws (Algorithm 1, GET UPDATE first two steps)
# ----------------------------------------------------------------------------
def weight_bits(count: int) -> int:
    """L such that count * 2^L < 2^62."""
    return 62 - int(math.ceil(math.log2(count + 1)))


def quantize(values: np.ndarray, active: np.ndarray) -> np.ndarray:
    """w_j = floor(values_j / max_active * 2^L) on active entries, else 0."""
    values = np.asarray(values, dtype=np.float64)
    L = weight_bits(values.shape[0])
    w = np.zeros(values.shape[0], dtype=np.uint64)
    if not active.any():
        return w
    vmax = values[active].max()
    if not vmax > 0:
        return w
    q = np.floor(np.ldexp(values[active] / vmax, L))
    w[active] = q.astype(np.uint64)
    return w


def draw(weights: np.ndarray, count: int, seed: int, t: int, stream: int) -> np.ndarray:
    """Draw `count` indices with replacement, P[i] = w_i / sum(w)."""
    cdf = np.cumsum(weights.astype(np.uint64), dtype=np.uint64)
    total = int(cdf[-1])
    out = np.empty(count, dtype=np.int64)
    for j, u in enumerate(uniform_u64(seed, t, stream, count)):
        v = (u * total) >> 64
        out[j] = int(np.searchsorted(cdf, np.uint64(v), side="right"))
    return out


def column_values(strategy: str, t: int, s: np.ndarray, A: np.ndarray,
                  U: Optional[np.ndarray]) -> np.ndarray:
    """Unnormalised column probabilities for iteration t (Sec. 3.1).

    Round 0 is always L2N (p_i proportional to |a_i|^2, Eq. 2).  Afterwards:
    L2N keeps Eq. 2, UNF is uniform, ORT uses |a_i - U U^T a_i|^2 (Eq. 6)
    computed as max(0, |a_i|^2 - |U^T a_i|^2)."""
    if t == 0 or strategy == "l2n":
        return s
    if strategy == "unf":
        return np.ones_like(s)
    if strategy == "ort":
        proj = A.T @ U
        return np.maximum(0.0, s - np.sum(proj * proj, axis=1))
    raise ValueError(strategy)


def sample_columns(values: np.ndarray, in_S: np.ndarray, c: int, seed: int, t: int):
    """Draws c columns from S, returns sorted distinct I_c (Alg. 1, GET UPDATE)."""
    w = quantize(values, in_S)
    if int(w.sum()) == 0:
        w = in_S.astype(np.uint64)
    d = draw(w, c, seed, t, STREAM_COLS)
    return np.unique(d), w


# ----------------------------------------------------------------------------
# SAMPLE AND SCALE UNIQUE ROWS (Algorithm 1)
# ----------------------------------------------------------------------------
def sample_scale_rows(D: np.ndarray, row_values: np.ndarray, w: int, seed: int, t: int):
    """w row draws with probability q, distinct rows I_r with counts t_hat,
    each kept row scaled by sqrt(t_hat / (w q)).  q is the quantised
    probability actually used for drawing."""
    m = D.shape[0]
    wq = quantize(row_values, np.ones(m, dtype=bool))
    if int(wq.sum()) == 0:
        wq = np.ones(m, dtype=np.uint64)
    total = float(int(wq.astype(np.uint64).sum(dtype=np.uint64)))
    d = draw(wq, w, seed, t, STREAM_ROWS)
    rows, counts = np.unique(d, return_counts=True)
    q = wq[rows].astype(np.float64) / total
    scale = np.sqrt(counts / (w * q))
    W = D[rows, :] * scale[:, None]
    return W, rows, counts


def top_right_vectors_of_gram(W: np.ndarray, r: int) -> np.ndarray:
    """V~_r from SVD(W^T W) (Alg. 1 GET UPDATE)."""
    V, _, _ = np.linalg.svd(W.T @ W)
    return V[:, :r]


# ----------------------------------------------------------------------------
# BLOCK MERGE (Algorithm 2, Eqs. 8-9)
# ----------------------------------------------------------------------------
@dataclass
class MergeResult:
    U: np.ndarray
    sigma: np.ndarray
    UE: np.ndarray          # left singular vectors of the core E
    sigma_E: np.ndarray     # all singular values of E


def block_merge(U1: np.ndarray, s1: np.ndarray, C: np.ndarray, r: int) -> MergeResult:
    """Merge the rank-r factors (U1, s1) with a new block whose scaled left
    factor U_2 Sigma_2 is C.

    U_t = C - U1 (U1^T C) = U_o R (Householder QR); E = [[diag(s1), U1^T C],
    [0, R]]; E = U_E Sigma_E V_E^T; U = [U1 U_o] U_E, truncated to r and to
    the non-zero singular values."""
    m = C.shape[0]
    P = U1.T @ C
    Ut = C - U1 @ P
    Uo, R = np.linalg.qr(Ut, mode="reduced")
    r1, g = U1.shape[1], C.shape[1]
    E = np.zeros((r1 + g, r1 + g))
    E[:r1, :r1] = np.diag(s1)
    E[:r1, r1:] = P
    E[r1:, r1:] = R
    UE, sE, _ = np.linalg.svd(E)
    if sE.size == 0 or sE[0] == 0:
        keep = 0
    else:
        thresh = max(m, r1 + g) * np.finfo(np.float64).eps * sE[0]
        keep = min(r, int(np.count_nonzero(sE > thresh)))
    U = np.hstack([U1, Uo]) @ UE[:, :keep]
    return MergeResult(U=U, sigma=sE[:keep].copy(), UE=UE, sigma_E=sE)


def convergence_measures(UE: np.ndarray, k: int, r_prev: int):
    """(max sin, min |cos|) between the previous top-k modes and the merged
    top-k modes, read from the core's left singular vectors (basis [U Q]).

    sin(theta) = singular values of U_E[k:, :k]; mode cosines = |U_E[i, i]|.
    Meaningful only when the previous basis held at least k modes."""
    kk = min(k, UE.shape[1], r_prev)
    if kk < k or r_prev == 0:
        return 1.0, 0.0
    B = UE[k:, :k]
    sin_max = float(np.linalg.norm(B, 2)) if B.size else 0.0
    cos_min = float(np.min(np.abs(np.diag(UE[:k, :k]))))
    return sin_max, cos_min


# ----------------------------------------------------------------------------
# ISMA (Algorithm 1)
# ----------------------------------------------------------------------------
@dataclass
class Params:
    k: int
    c: int
    r: int = 0                      # carried rank; 0 -> k
    rows: int = 0                   # 1 = also sample rows (ICRS)
    w: int = 0                      # row draws; 0 -> Eq. 5 with eps = delta = 0.6, capped at m
    col_strategy: str = "unf"       # 'l2n' | 'unf' | 'ort' (round 0 is always L2N)
    row_strategy: str = "l2n"       # 'l2n' | 'ls'
    criterion: str = "subspace"     # 'subspace' | 'modes'
    tol: float = 1e-8               # subspace: stop at max sin <= tol; modes: stop at min |cos| >= tol
    max_iter: int = 1 << 30         # merges after round 0
    refine: bool = True
    seed: int = 0x5107
    paper_literal: bool = False
    replay: Optional[list] = None   # frozen column index sets per round

    def carried_rank(self) -> int:
        return self.r if self.r > 0 else self.k


@dataclass
class IterRecord:
    t: int
    idx: np.ndarray
    g: int
    remaining: int
    sin_max: float
    cos_min: float
    sigma: np.ndarray
    rows: Optional[np.ndarray] = None
    row_counts: Optional[np.ndarray] = None
    sigma_E: Optional[np.ndarray] = None   # every singular value of the merge core E


@dataclass
class Result:
    U: np.ndarray
    sigma: np.ndarray
    V: Optional[np.ndarray]
    trace: List[IterRecord] = field(default_factory=list)
    converged: bool = False
    sigma_all: Optional[np.ndarray] = None   # all r carried singular values

    @property
    def iterations(self) -> int:
        return len(self.trace)


def column_sq_norms(A: np.ndarray) -> np.ndarray:
    """s_j = sum_i a_ij^2 (numerator of Eq. 2)."""
    A = np.asarray(A, dtype=np.float64)
    return np.einsum("ij,ij->j", A, A)


def new_block(A: np.ndarray, idx: np.ndarray, p: Params, t: int, U: np.ndarray):
    """GET UPDATE: the new block's scaled factor U_2 Sigma_2."""
    D = A[:, idx]
    r = p.carried_rank()
    rec_rows = (None, None)
    if p.rows == 1:
        if p.row_strategy == "ls" and U.shape[1] > 0:
            Uk = U[:, : min(p.k, U.shape[1])]
            values = np.sum(Uk * Uk, axis=1) / Uk.shape[1]
        else:
            values = np.sum(D * D, axis=1)
        w = p.w if p.w > 0 else min(A.shape[0], rows_eq5(p.k, 0.6, 0.6))
        W, rows, counts = sample_scale_rows(D, values, w, p.seed, t)
        Vr = top_right_vectors_of_gram(W, r)
        return D @ Vr, (rows, counts)
    if p.paper_literal:
        Vr = top_right_vectors_of_gram(D, r)
        return D @ Vr, rec_rows
    return D, rec_rows


def fix_signs(U: np.ndarray, V: Optional[np.ndarray], seed: int):
    z = sign_reference(seed, U.shape[0])
    s = np.sign(U.T @ z)
    s[s == 0] = 1.0
    U = U * s
    if V is not None:
        V = V * s
    return U, V


def refine(A: np.ndarray, U: np.ndarray):
    """Closing step of Algorithm 1: QR(A^T U) = Q R, SVD(R) = U_R S_R V_R^T,
    U <- U V_R, sigma <- S_R, V <- Q U_R."""
    Y = np.asarray(A, dtype=np.float64).T @ U
    Q, R = np.linalg.qr(Y, mode="reduced")
    UR, SR, VRt = np.linalg.svd(R)
    return U @ VRt.T, SR, Q @ UR


def isma_steps(A: np.ndarray, p: Params):
    """Algorithm 1 of the paper, in FP64, with the readings listed above, as a
    generator that pauses after each unit of work: it yields ("norms", None)
    once the column norms exist, ("round", t) after each round t, and finally
    ("done", Result) after the refinement.  ``isma`` runs it to the end; the
    pauses only let a caller time the units one by one."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    r = p.carried_rank()
    s = column_sq_norms(A)
    yield "norms", None
    in_S = np.ones(n, dtype=bool)
    U = np.zeros((m, 0))
    sig = np.zeros(0)
    trace: List[IterRecord] = []
    converged = False
    t = 0
    while True:
        if p.replay is not None:
            if t >= len(p.replay):
                break
            idx = np.unique(np.asarray(p.replay[t], dtype=np.int64))
        else:
            vals = column_values(p.col_strategy, t, s, A, U)
            idx, _ = sample_columns(vals, in_S, p.c, p.seed, t)
        in_S[idx] = False
        C, (rows, counts) = new_block(A, idx, p, t, U)
        r_prev = U.shape[1]
        res = block_merge(U, sig, C, r)
        sin_max, cos_min = convergence_measures(res.UE, p.k, r_prev)
        U, sig = res.U, res.sigma
        trace.append(IterRecord(t=t, idx=idx, g=int(idx.size), remaining=int(in_S.sum()),
                                sin_max=sin_max, cos_min=cos_min, sigma=sig.copy(),
                                rows=rows, row_counts=counts, sigma_E=res.sigma_E.copy()))
        if t > 0 and r_prev >= p.k:
            if p.criterion == "subspace" and sin_max <= p.tol:
                converged = True
            if p.criterion == "modes" and cos_min >= p.tol:
                converged = True
        yield "round", t
        t += 1
        if converged or not in_S.any() or t > p.max_iter:
            break
    V = None
    if p.refine and U.shape[1] > 0:
        U, sig, V = refine(A, U)
    kk = min(p.k, U.shape[1])
    sig_all = sig.copy()
    U, V = U[:, :kk], (V[:, :kk] if V is not None else None)
    U, V = fix_signs(U, V, p.seed)
    yield "done", Result(U=U, sigma=sig[:kk], V=V, trace=trace, converged=converged, sigma_all=sig_all)


def isma(A: np.ndarray, p: Params) -> Result:
    """Algorithm 1 of the paper, in FP64, with the readings listed above."""
    for kind, val in isma_steps(A, p):
        if kind == "done":
            return val
    raise AssertionError("unreachable")


# ----------------------------------------------------------------------------
# Quality of the converged solution (Sec. 3.3, Eq. 7)
# ----------------------------------------------------------------------------
@dataclass
class Wedin:
    bound: float
    norm_R: float
    norm_S: float
    omega: float


def wedin_measure(A: np.ndarray, U: np.ndarray, sigma: np.ndarray, V: np.ndarray,
                  sigma_next: float) -> Wedin:
    """Right-hand side of Eq. 7 for the approximate top-k triplets
    (U, sigma, V): R = A V - U diag(sigma), S = A^T U - V diag(sigma), and
    omega estimated from the approximate singular values as
    min(|sigma_k - sigma_{k+1}|, sigma_k)."""
    A = np.asarray(A, dtype=np.float64)
    R = A @ V - U * sigma[None, :]
    S = A.T @ U - V * sigma[None, :]
    nR, nS = float(np.linalg.norm(R)), float(np.linalg.norm(S))
    sk = float(sigma[-1])
    omega = min(abs(sk - float(sigma_next)), sk)
    return Wedin(bound=math.sqrt(nR * nR + nS * nS) / omega, norm_R=nR, norm_S=nS, omega=omega)


# ----------------------------------------------------------------------------
# INCREMENTAL POD (Algorithm 3): ISMA per column block, merged with MAT
# ----------------------------------------------------------------------------
def incremental_pod(A: np.ndarray, blocks: int, p: Params) -> Result:
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    r = p.carried_rank()
    bounds = [(b * n) // blocks for b in range(blocks + 1)]
    U = np.zeros((A.shape[0], 0))
    sig = np.zeros(0)
    for b in range(blocks):
        sub = A[:, bounds[b]:bounds[b + 1]]
        pb = Params(**{**p.__dict__, "refine": False, "k": r})
        rb = isma(sub, pb)
        # rb.U carries r modes of the block with their singular values
        res = block_merge(U, sig, rb.U * rb.sigma, r)
        U, sig = res.U, res.sigma
    kk = min(p.k, U.shape[1])
    U, _ = fix_signs(U[:, :kk], None, p.seed)
    return Result(U=U, sigma=sig[:kk], V=None, trace=[], converged=True)


# ----------------------------------------------------------------------------
# Accuracy measures (Sec. 2): mode angles and principal angles
# ----------------------------------------------------------------------------
def sin_principal_max(U: np.ndarray, W: np.ndarray) -> float:
    """Largest sine of the principal angles between span(U) and span(W)
    (orthonormal columns, equal count): || (I - U U^T) W ||_2."""
    Ru = W - U @ (U.T @ W)
    return float(np.linalg.norm(Ru, 2))


def mode_angles(U: np.ndarray, W: np.ndarray) -> np.ndarray:
    """theta_i = acos(|u_i^T w_i|) in radians."""
    c = np.abs(np.sum(U * W, axis=0))
    return np.arccos(np.clip(c, 0.0, 1.0))
