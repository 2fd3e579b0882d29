"""GPU parity of ISMA with row sampling (ICRS, rows = 1): Algorithm 1's GET
UPDATE with rows and SAMPLE AND SCALE UNIQUE ROWS, Sec. 3.1 row strategies.

Row draws are integer work and compared bit-exactly with the oracle round by
round (distinct rows and their counts), like the column draws; the modes and
singular values within the floating-point tolerances of the ICS tests.
"""
import numpy as np
import pytest

from oracle import isma as O
from paper_1905_05107_gb300 import synth

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

pytestmark = pytest.mark.gpu

from paper_1905_05107_gb300 import build, pod  # noqa: E402

build.build()
DEV = torch.device("cuda:0")


def to_dev(A):
    t = torch.from_numpy(np.asfortranarray(A).T.copy()).to(DEV)
    return t.t()


def run_stepwise(A, k, c, **kw):
    """One pod_iterate step at a time, recording the column and row draws."""
    At = to_dev(A)
    ctx = pod.Context(At, k, c, rows=True, **kw)
    idx, rows, counts, meas = [], [], [], []
    t = 0
    while True:
        done, m_, steps = ctx.iterate(1)
        if steps == 0:
            break
        i, mm = ctx.trace(t)
        r, cnt = ctx.last_rows()
        idx.append(i)
        rows.append(r)
        counts.append(cnt)
        meas.append(mm)
        t += 1
        if done:
            break
    w = ctx.row_draws()
    U, s, _ = ctx.modes()
    torch.cuda.synchronize()
    out = dict(U=U.double().cpu().numpy(), sigma=s.cpu().numpy(), idx=idx, rows=rows, counts=counts,
               measure=meas, steps=t, w=w)
    ctx.close()
    return out


def check_trace(g, ref):
    assert g["steps"] == len(ref.trace)
    for t, rec in enumerate(ref.trace):
        assert np.array_equal(g["idx"][t], rec.idx), "columns, round %d" % t
        assert np.array_equal(g["rows"][t], rec.rows), "rows, round %d" % t
        assert np.array_equal(g["counts"][t], rec.row_counts), "row counts, round %d" % t
        assert int(g["counts"][t].sum()) == g["w"]


def oracle(A, k, c, **kw):
    kw.setdefault("seed", 0x5107)
    return O.isma(np.asarray(A, dtype=np.float64), O.Params(k=k, c=c, rows=1, **kw))


@pytest.mark.parametrize("m,k", [(20000, 1), (20000, 3), (20000, 10), (20000, 20), (3000, 20)])
def test_default_row_draws_eq5(m, k):
    """w = Eq. 5 with epsilon = delta = 0.6, capped at m."""
    A = synth.planted(m, 60, 0.8 ** np.arange(10), 1e-5, 3, np.float32)
    ctx = pod.Context(to_dev(A), k, 2 * k, rows=True)
    assert ctx.row_draws() == min(m, O.rows_eq5(k, 0.6, 0.6))
    ctx.close()


@pytest.mark.parametrize("row_strategy", ["l2n", "ls"])
def test_icrs_planted_f64_bit_exact_draws(row_strategy):
    """FP64 planted spectrum, to exhaustion of S: every round's columns, rows
    and row counts equal the oracle's; sigma and the subspace to 1e-9."""
    A = synth.planted(2500, 150, 0.8 ** np.arange(30), 1e-5, 21, np.float64)
    ref = oracle(A, 5, 12, row_strategy=row_strategy, tol=1e-8)
    g = run_stepwise(A, 5, 12, row_strategy=row_strategy, tol=1e-8)
    check_trace(g, ref)
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-9)
    assert O.sin_principal_max(ref.U, g["U"]) <= 1e-9


@pytest.mark.parametrize("kw", [dict(w=300), dict(w=5000, r=8), dict(col_strategy="l2n", max_iter=4),
                                dict(criterion="modes", tol=0.999)])
def test_icrs_options_f64(kw):
    A = synth.planted(1800, 120, 0.75 ** np.arange(25), 1e-5, 22, np.float64)
    okw = dict(kw)
    okw.setdefault("max_iter", 1 << 30)
    okw.setdefault("tol", 1e-8)
    ref = oracle(A, 4, 10, **okw)
    g = run_stepwise(A, 4, 10, **kw)
    check_trace(g, ref)
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-9)
    assert O.sin_principal_max(ref.U, g["U"]) <= 1e-9


def test_icrs_flow_f32_reduced():
    """Flow snapshots on a 60 x 60 grid, 300 snapshots, FP32, k = 20, c = 40:
    draws bit-exact, sigma and subspace within the FP32 tolerance 1e-5."""
    A = synth.make_flow_316(grid=60, n=300)
    ref = oracle(A, 20, 40, tol=1e-8)
    g = run_stepwise(A, 20, 40, tol=1e-8)
    check_trace(g, ref)
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-5)
    assert O.sin_principal_max(ref.U, g["U"]) <= 1e-5


def test_icrs_planted_f32_ragged():
    """FP32, m not a multiple of the row block (1024) or of 4."""
    A = synth.planted(5003, 90, 0.7 ** np.arange(20), 1e-4, 23, np.float32)
    ref = oracle(A, 4, 9, tol=1e-8)
    g = run_stepwise(A, 4, 9, tol=1e-8)
    check_trace(g, ref)
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-5)
    assert O.sin_principal_max(ref.U, g["U"]) <= 1e-5


def test_icrs_few_row_draws_degenerate():
    """w = 3 < g: W has rank <= 3 < r, so V_r holds null vectors of W and is
    not unique.  The draws still match the oracle; the run completes with
    orthonormal modes and finite singular values."""
    A = synth.planted(900, 60, 0.8 ** np.arange(12), 1e-5, 24, np.float64)
    ref = oracle(A, 4, 10, w=3, tol=1e-8, max_iter=3)
    g = run_stepwise(A, 4, 10, w=3, tol=1e-8, max_iter=3)
    check_trace(g, ref)
    U = g["U"]
    assert np.all(np.isfinite(g["sigma"]))
    np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-10)


def test_icrs_zero_matrix_uniform_rows():
    """All-zero data: every row weight is zero, rows are drawn uniformly
    (the fallback), and the run ends with zero singular values."""
    A = np.zeros((700, 30))
    ref = oracle(A, 2, 6, tol=1e-8, refine=False)
    g = run_stepwise(A, 2, 6, tol=1e-8, refine=False)
    check_trace(g, ref)
    assert np.all(g["sigma"] == 0.0)


def test_icrs_flow_f32_full_size():
    """The 316 x 316 x 2000 FP32 flow workload with rows (w = Eq. 5 default,
    13576 draws per round): all draws bit-exact, sigma and subspace 1e-5."""
    A = synth.make_flow_316()
    ref = oracle(A, 20, 40, tol=1e-8)
    g = run_stepwise(A, 20, 40, tol=1e-8)
    check_trace(g, ref)
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-5)
    assert O.sin_principal_max(ref.U, g["U"]) <= 1e-5


# ------------------------------------------------ literal GET UPDATE truncation
def run_literal(A, k, c, **kw):
    ctx = pod.Context(to_dev(A), k, c, block_trunc=True, **kw)
    done, meas, steps = ctx.iterate()
    idx = [ctx.trace(t)[0] for t in range(steps)]
    U, s, _ = ctx.modes()
    out = dict(U=U.double().cpu().numpy(), sigma=s.cpu().numpy(), idx=idx, steps=steps)
    ctx.close()
    return out


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-9), (np.float32, 1e-5)])
def test_block_truncation_matches_paper_literal_oracle(dtype, tol):
    """Algorithm 1 read literally: the new block is truncated to rank r by
    SVD(D^T D) before BLOCK MERGE (the oracle's paper_literal mode)."""
    A = synth.planted(3000, 160, 0.8 ** np.arange(40), 1e-5, 25, dtype)
    ref = O.isma(np.asarray(A, dtype=np.float64), O.Params(k=5, c=14, seed=0x5107, tol=1e-8, paper_literal=True))
    g = run_literal(A, 5, 14, tol=1e-8)
    assert g["steps"] == len(ref.trace)
    for t, rec in enumerate(ref.trace):
        assert np.array_equal(g["idx"][t], rec.idx)
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=tol)
    assert O.sin_principal_max(ref.U, g["U"]) <= tol


def _cut_floor(A, ref, r):
    """u_32 sigma_1 / (sigma_r - sigma_{r+1}) of the sampled blocks D, worst
    round: the accuracy to which FP32 arithmetic determines the truncated
    block's right vectors V_r (Davis-Kahan)."""
    f = 0.0
    for rec in ref.trace:
        s = np.linalg.svd(A[:, rec.idx], compute_uv=False)
        if s.size > r:
            f = max(f, 5.96e-8 * s[0] / (s[r - 1] - s[r]))
    return f


@pytest.mark.parametrize("core", ["f64", "auto"])
def test_block_truncation_flow_f32_reduced(core):
    """Flow snapshots (60 x 60 grid, 300 steps, FP32), k = r = 20, c = 40.
    Truncating a 40-column block at 20 cuts between nearly equal singular
    values in some rounds (relative gap 4e-4 of sigma_1), so the FP32 core's
    V_r is only determined to u_32 sigma_1 / gap (1.5e-4 here) in those
    rounds; with the FP64 core the result meets 1e-5, with the FP32 core a
    tenth of that floor."""
    A = synth.make_flow_316(grid=60, n=300)
    A64 = A.astype(np.float64)
    ref = O.isma(A64, O.Params(k=20, c=40, seed=0x5107, tol=1e-8, paper_literal=True))
    g = run_literal(A, 20, 40, tol=1e-8, core=core)
    assert g["steps"] == len(ref.trace)
    for t, rec in enumerate(ref.trace):
        assert np.array_equal(g["idx"][t], rec.idx)
    bar = 1e-5 if core == "f64" else max(1e-5, 0.1 * _cut_floor(A64, ref, 20))
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-5)
    assert O.sin_principal_max(ref.U, g["U"]) <= bar
