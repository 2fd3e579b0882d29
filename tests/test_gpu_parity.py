"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Bars (from the stated targets): sampled indices bit-exact; FP64 storage:
sigma and subspaces to 1e-10; FP32 storage: sigma relative error and sine
of the largest principal angle to the oracle subspace <= 1e-5."""
import numpy as np
import pytest

from oracle import isma as O
from paper_1905_05107_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_05107_gb300 import build, pod  # noqa: E402

build.build()
DEV = torch.device("cuda:0")


def to_dev(A):
    """Fortran-ordered (m, n) numpy array -> column-major CUDA tensor."""
    t = torch.from_numpy(np.asfortranarray(A).T.copy()).to(DEV)   # (n, m) row-major
    return t.t()


def oracle_params(k, c, **kw):
    kw.setdefault("seed", 0x5107)
    return O.Params(k=k, c=c, **kw)


def run_gpu(A, k, c, tol=1e-8, max_iter=0, refine=True, seed=0x5107, col_strategy="unf", r=0,
            criterion="subspace", core="auto", replay=None, with_v=False):
    At = to_dev(A)
    ctx = pod.Context(At, k, c, r=r, col_strategy=col_strategy, criterion=criterion, tol=tol,
                      max_iter=max_iter, refine=refine, seed=seed, core=core)
    if replay is not None:
        ctx.replay(replay)
    done, meas, steps = ctx.iterate()
    traces = [ctx.trace(t) for t in range(steps)]
    U, s, V = ctx.modes(with_v=with_v)
    torch.cuda.synchronize()
    out = dict(U=U.double().cpu().numpy(), sigma=s.cpu().numpy(), steps=steps, done=done,
               idx=[t[0] for t in traces], measure=[t[1] for t in traces],
               V=None if V is None else V.double().cpu().numpy())
    ctx.close()
    return out


def sin_max(U, W):
    return O.sin_principal_max(U, W)


# --------------------------------------------------------------------------- a0
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("m,n,pad", [(1, 1, 0), (1000, 37, 0), (4097, 65, 3), (100003, 9, 1)])
def test_colnorms(dtype, m, n, pad):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m + pad, n)).astype(dtype) * rng.random(n).astype(dtype) * 10
    At = to_dev(A)[:m, :]
    s = pod.colnorms(At).cpu().numpy()
    ref = O.column_sq_norms(A[:m, :])
    # FP32 data: each thread sums exact squares in a (hi, lo) float pair
    # (about 2^-44 per step over a few hundred steps), partials in FP64
    np.testing.assert_allclose(s, ref, rtol=2e-12 if dtype == np.float32 else 1e-13, atol=0)


# ----------------------------------------------------------------------- a1, a2
@pytest.mark.parametrize("n,c,t,stream_id", [(1, 1, 0, 0), (7, 20, 3, 0), (2000, 40, 5, 0),
                                             (4000, 100, 0, 1), (100003, 300, 11, 0)])
def test_sampler_bit_exact_shared_weights(n, c, t, stream_id):
    """Same integer weights and mask on both sides -> identical I_c and S."""
    rng = np.random.default_rng(n + c)
    vals = rng.random(n) ** 3
    vals[rng.random(n) < 0.1] = 0.0
    mask = rng.random(n) < 0.8
    mask[0] = True
    w = O.quantize(vals, mask)
    seed = 0xC0FFEE1234 + n
    # oracle: the draw rule of Algorithm 1's GET UPDATE over the same weights
    ww = w.copy()
    if int(ww.sum()) == 0:
        ww = mask.astype(np.uint64)
    ref = np.unique(O.draw(ww, c, seed, t, stream_id))
    wt = torch.from_numpy(w.view(np.int64)).to(DEV)
    mt = torch.from_numpy(mask.astype(np.uint8)).to(DEV)
    idx = pod.sample(wt, mt, c, seed, t, stream_id).cpu().numpy()
    assert np.array_equal(idx, ref)
    mask_after = mask.copy()
    mask_after[ref] = False
    assert np.array_equal(mt.cpu().numpy().astype(bool), mask_after)


def test_sampler_uniform_fallback_and_masking():
    n = 50
    mask = np.zeros(n, dtype=bool)
    mask[[4, 17, 33]] = True
    w = np.zeros(n, dtype=np.uint64)
    ref = np.unique(O.draw(mask.astype(np.uint64), 25, 9, 2, 0))
    idx = pod.sample(torch.from_numpy(w.view(np.int64)).to(DEV),
                     torch.from_numpy(mask.astype(np.uint8)).to(DEV), 25, 9, 2).cpu().numpy()
    assert np.array_equal(idx, ref)
    assert set(idx.tolist()) <= {4, 17, 33}


# ------------------------------------------------------------------- a4 .. a9
@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-11), (np.float32, 2e-6)])
@pytest.mark.parametrize("m,r1,g,r", [(300, 0, 7, 5), (513, 6, 9, 6), (4101, 10, 20, 10), (2000, 20, 40, 20),
                                      (777, 5, 3, 8), (3001, 12, 16, 4)])
def test_block_merge(dtype, tol, m, r1, g, r):
    rng = np.random.default_rng(m + r1 + g)
    X = rng.standard_normal((m, max(r1, 1) + 4)) * (0.7 ** np.arange(max(r1, 1) + 4))
    Ux, sx, _ = np.linalg.svd(X, full_matrices=False)
    U1, s1 = Ux[:, :r1], sx[:r1]
    C = rng.standard_normal((m, g)) * 0.3
    U1 = U1.astype(dtype).astype(np.float64)
    C = C.astype(dtype).astype(np.float64)
    ref = O.block_merge(U1, s1, C, r)
    U1t = to_dev(U1.astype(dtype)) if r1 else None
    s1t = torch.from_numpy(s1.copy()).to(DEV) if r1 else None
    Uo, so = pod.block_merge(U1t, s1t, to_dev(C.astype(dtype)), r)
    Uo = Uo.double().cpu().numpy()
    so = so.cpu().numpy()
    assert Uo.shape[1] == ref.U.shape[1]
    np.testing.assert_allclose(so, ref.sigma, rtol=tol)
    # The truncated subspace is determined only up to u sigma_1 / (sigma_r -
    # sigma_{r+1}) (Davis-Kahan / Wedin): the bar is the larger of 10 tol and
    # 10 times that floor for the storage precision u.
    sE = ref.sigma_E
    u = 5.96e-8 if dtype == np.float32 else 1.11e-16
    floor = u * sE[0] / (sE[r - 1] - sE[r]) if r < sE.size else 0.0
    assert sin_max(ref.U, Uo) < max(10 * tol, 10 * floor)
    assert np.abs(Uo.T @ Uo - np.eye(Uo.shape[1])).max() < 10 * tol


def test_block_merge_rank_deficient_block():
    """New columns inside span(U_1): Algorithm 2 keeps only the non-zero
    singular values."""
    rng = np.random.default_rng(3)
    m = 400
    X = rng.standard_normal((m, 4))
    Ux, sx, _ = np.linalg.svd(X, full_matrices=False)
    C = X @ rng.standard_normal((4, 6))
    Uo, so = pod.block_merge(to_dev(Ux), torch.from_numpy(sx.copy()).to(DEV), to_dev(C), 8)
    ref = O.block_merge(Ux, sx, C, 8)
    assert Uo.shape[1] == ref.U.shape[1] == 4
    np.testing.assert_allclose(so.cpu().numpy(), ref.sigma, rtol=1e-10)


# --------------------------------------------------------------- whole ISMA
def compare_runs(g, ref, sig_tol, sin_tol, k):
    assert g["steps"] == len(ref.trace)
    for t, rec in enumerate(ref.trace):
        assert np.array_equal(g["idx"][t], rec.idx), "round %d" % t
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=sig_tol)
    s = sin_max(ref.U, g["U"])
    assert s <= sin_tol, s


def test_isma_planted_small_f64():
    """2000 x 500 planted spectrum, FP64, k = 10, c = 20, loop until the
    subspace change is below 1e-8 or S is empty; refinement on."""
    A = synth.make_planted_small()
    ref = O.isma(A, oracle_params(10, 20, tol=1e-8))
    g = run_gpu(A, 10, 20, tol=1e-8)
    compare_runs(g, ref, 1e-10, 1e-10, 10)
    np.testing.assert_allclose(g["U"], ref.U, atol=1e-9)


def test_isma_planted_small_f32_copy():
    A = synth.make_planted_small(dtype=np.float32)
    A64 = A.astype(np.float64)
    ref = O.isma(A64, oracle_params(10, 20, tol=1e-8))
    g = run_gpu(A, 10, 20, tol=1e-8)
    compare_runs(g, ref, 1e-5, 1e-5, 10)


@pytest.mark.parametrize("grid,n", [(60, 300), (100, 600)])
def test_isma_flow_f32_reduced(grid, n):
    A = synth.make_flow_316(grid=grid, n=n)
    ref = O.isma(A.astype(np.float64), oracle_params(20, 40, tol=1e-8))
    g = run_gpu(A, 20, 40, tol=1e-8)
    compare_runs(g, ref, 1e-5, 1e-5, 20)


def test_isma_flow_f32_full_size():
    """The benchmark workload: 316 x 316 grid (m = 99856) x 2000 snapshots,
    FP32, k = 20, c = 40, run to the end, refinement on."""
    A = synth.make_flow_316()
    ref = O.isma(A.astype(np.float64), oracle_params(20, 40, tol=1e-8))
    g = run_gpu(A, 20, 40, tol=1e-8)
    compare_runs(g, ref, 1e-5, 1e-5, 20)


@pytest.mark.parametrize("kw", [dict(max_iter=3), dict(col_strategy="l2n"), dict(r=6, k=3),
                                dict(criterion="modes", tol=0.999), dict(c=1, k=1), dict(c=60, k=2)])
def test_isma_options_f64(kw):
    A = synth.planted(700, 160, 0.8 ** np.arange(30), 1e-5, 77, np.float64)
    k = kw.pop("k", 4)
    c = kw.pop("c", 12)
    okw = dict(kw)
    if "max_iter" not in okw:
        okw["max_iter"] = 1 << 30
    ref = O.isma(A, oracle_params(k, c, tol=kw.get("tol", 1e-8), **{x: v for x, v in okw.items() if x != "tol"}))
    g = run_gpu(A, k, c, **kw)
    compare_runs(g, ref, 1e-10, 1e-9, k)


def test_isma_ragged_and_padded_lda():
    rng = np.random.default_rng(5)
    m, n = 1237, 97
    A = synth.planted(m, n, 0.7 ** np.arange(20), 1e-4, 5, np.float32)
    pad = np.zeros((m + 5, n), dtype=np.float32, order="F")
    pad[:m] = A
    At = to_dev(pad)[:m, :]
    ctx = pod.Context(At, 5, 9, tol=1e-8)
    done, meas, steps = ctx.iterate()
    U, s, V = ctx.modes()
    ref = O.isma(A.astype(np.float64), oracle_params(5, 9, tol=1e-8))
    assert steps == len(ref.trace)
    np.testing.assert_allclose(s.cpu().numpy(), ref.sigma, rtol=1e-5)
    assert sin_max(ref.U, U.double().cpu().numpy()) < 1e-5
    ctx.close()


def test_refinement_right_vectors_f64():
    A = synth.planted(500, 120, 0.75 ** np.arange(25), 1e-5, 8, np.float64)
    ref = O.isma(A, oracle_params(5, 15, tol=1e-8))
    g = run_gpu(A, 5, 15, tol=1e-8, with_v=True)
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-10)
    np.testing.assert_allclose(g["U"], ref.U, atol=1e-9)
    np.testing.assert_allclose(g["V"], ref.V, atol=1e-9)


def test_replay_matches_oracle_replay():
    A = synth.planted(400, 90, 0.8 ** np.arange(20), 1e-4, 4, np.float64)
    rng = np.random.default_rng(0)
    sets = [np.sort(rng.choice(90, size=8, replace=False)) for _ in range(5)]
    ref = O.isma(A, oracle_params(4, 8, replay=sets, tol=0.0))
    g = run_gpu(A, 4, 8, tol=0.0, replay=sets)
    assert g["steps"] == 5
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-10)
    assert sin_max(ref.U, g["U"]) < 1e-10


# ----------------------------------------------------------------------- a9
U32 = 5.96e-8


def _measure_bar(ref, t, k, u):
    """Bar on |GPU measure - oracle measure| in round t: the top-k subspaces
    compared in that round are each fixed only to about u sigma_1 / gap_k of
    their merge cores (Davis-Kahan / Wedin), so 10 times the sum of the two
    floors, plus 1e-9 for the FP64 arithmetic of the measure itself."""
    def floor(rec):
        sE = rec.sigma_E
        if sE is None or sE.size <= k:
            return 0.0
        return u * sE[0] / max(sE[k - 1] - sE[k], 1e-300)
    prev = floor(ref.trace[t - 1]) if t > 0 else 0.0
    return 10.0 * (floor(ref.trace[t]) + prev) + 1e-9


@pytest.mark.parametrize("case", ["planted_f64", "planted_f32", "flow_f32"])
def test_convergence_measure_trace(case):
    """Alg. 1's convergence test, subspace form: the per-round max sin(theta)
    between the previous and the merged top-k modes, compared round by round
    with the oracle's (1.0 where no comparison exists yet).  FP64 data:
    within 1e-9; FP32 data: within the per-round floor of _measure_bar."""
    if case == "planted_f64":
        A, k, c, u = synth.make_planted_small(), 10, 20, 1.11e-16
    elif case == "planted_f32":
        A, k, c, u = synth.make_planted_small(dtype=np.float32), 10, 20, U32
    else:
        A, k, c, u = synth.make_flow_316(grid=100, n=600), 20, 40, U32
    ref = O.isma(A.astype(np.float64), oracle_params(k, c, tol=1e-8))
    g = run_gpu(A, k, c, tol=1e-8)
    assert g["steps"] == len(ref.trace)
    compared = 0
    for t, rec in enumerate(ref.trace):
        bar = 1e-9 if u < 1e-15 else _measure_bar(ref, t, k, u)
        assert abs(g["measure"][t] - rec.sin_max) <= bar, (t, g["measure"][t], rec.sin_max, bar)
        compared += rec.sin_max < 1.0
    assert compared >= len(ref.trace) - 2


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-8), (np.float32, 1e-4)])
def test_subspace_criterion_stops_before_s_is_empty(dtype, tol):
    """A noiseless planted matrix of rank k: once the sampled columns span its
    column space (round 2 with c = 2, k = 6) the next merge leaves the top-k
    subspace unchanged, max sin(theta) falls below tol and Alg. 1 stops with
    most columns unsampled.  Steps, the done flag, every draw and the final
    measure agree with the oracle."""
    k, c = 6, 2
    A = synth.planted(2000, 300, 0.7 ** np.arange(k), 0.0, 99, dtype)
    ref = O.isma(A.astype(np.float64), oracle_params(k, c, tol=tol))
    assert ref.converged and ref.trace[-1].remaining > 250 and len(ref.trace) == 4
    g = run_gpu(A, k, c, tol=tol)
    assert g["done"] and g["steps"] == len(ref.trace)
    for t, rec in enumerate(ref.trace):
        assert np.array_equal(g["idx"][t], rec.idx)
    assert g["measure"][-1] <= tol
    assert all(mv == 1.0 for mv in g["measure"][:-1])
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-10 if dtype == np.float64 else 1e-5)


def test_merge_core_cut_inside_degenerate_pair():
    """The flow snapshots' singular values come in exactly degenerate pairs
    (noise splits them by ~1e-3 of sigma_20 at most); with k = r = 21 every merge core is
    cut inside the eleventh pair, so the trailing rows of the core's Jacobi
    hold a direction as large as the last kept one and the Gershgorin guard
    of the skipped trailing pairs must send the sweeps back over every pair.
    Draws bit-exact; all 21 singular values and the well-separated top-20
    subspace (Alg. 2, SVD of the core) at the FP32 bar; sigma_21 and
    sigma_22 stay within the pair's noise split of the oracle."""
    A = synth.make_flow_316(grid=100, n=600)
    k, c = 21, 40
    ref = O.isma(A.astype(np.float64), oracle_params(k, c, tol=1e-8))
    g = run_gpu(A, k, c, tol=1e-8)
    assert g["steps"] == len(ref.trace)
    for t, rec in enumerate(ref.trace):
        assert np.array_equal(g["idx"][t], rec.idx), "round %d" % t
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-5)
    assert sin_max(ref.U[:, :20], g["U"][:, :20]) <= 1e-5
