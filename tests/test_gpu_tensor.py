"""The tcgen05 tensor-core contraction Y = A^T U (split-TF32 products) of the
closing refinement and the ORT weights, against the FP64 definition and the
FP32 SIMT kernel; and whole ISMA runs with it against the oracle."""
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
    return torch.from_numpy(np.asfortranarray(A).T.copy()).to(DEV).t()


def check_atu(m, n, r, precision, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)).astype(np.float32) * np.exp(rng.uniform(-3, 3, size=n)).astype(np.float32)
    U = rng.standard_normal((m, r)).astype(np.float32)
    Y = pod.atu(to_dev(A), to_dev(U), precision=precision).cpu().numpy()
    A64, U64 = A.astype(np.float64), U.astype(np.float64)
    ref = A64.T @ U64
    scale = np.abs(A64).T @ np.abs(U64)          # sum_i |a_ij| |u_il|
    err = np.max(np.abs(Y - ref) / scale)
    return err


@pytest.mark.parametrize("m,n,r", [(4096, 300, 20), (1000, 77, 1), (2048, 129, 33), (8192, 128, 64),
                                   (99856, 2000, 20)])
def test_atu_tensor_cores_vs_fp64(m, n, r):
    """Split-TF32 (3 TF32 products) with FP32 accumulation per 64 rows and
    double-float across: error below 2e-6 of sum |a_ij u_il| (TF32 split
    error ~2^-21 per product plus the tensor cores' FP32 group sums)."""
    err = check_atu(m, n, r, "tf32x3")
    assert err < 2e-6, err


@pytest.mark.parametrize("m,n,r", [(4096, 300, 20), (1000, 77, 1)])
def test_atu_simt_vs_fp64(m, n, r):
    assert check_atu(m, n, r, "f32") < 1e-5


def test_atu_tensor_cores_unsupported_shapes():
    A = torch.zeros((1002, 10), dtype=torch.float32, device=DEV).t().contiguous().t()
    U = torch.zeros((1002, 4), dtype=torch.float32, device=DEV).t().contiguous().t()
    with pytest.raises(pod.PodError) as e:
        pod.atu(A, U, precision="tf32x3")        # m not a multiple of 4
    assert e.value.status == pod.POD_EUNSUPPORTED
    A = torch.zeros((1000, 10), dtype=torch.float64, device=DEV).t().contiguous().t()
    U = torch.zeros((1000, 4), dtype=torch.float64, device=DEV).t().contiguous().t()
    with pytest.raises(pod.PodError) as e:
        pod.atu(A, U, precision="tf32x3")        # FP64 data
    assert e.value.status == pod.POD_EUNSUPPORTED


def run(A, k, c, **kw):
    ctx = pod.Context(to_dev(A), k, c, tol=1e-8, **kw)
    done, meas, steps = ctx.iterate()
    idx = [ctx.trace(t)[0] for t in range(steps)]
    U, s, V = ctx.modes(with_v=True)
    out = dict(U=U.double().cpu().numpy(), sigma=s.cpu().numpy(), V=V.double().cpu().numpy(), idx=idx)
    ctx.close()
    return out


def test_isma_flow_tensor_core_refinement():
    """FP32 flow snapshots with the refinement on the tensor cores: draws
    bit-exact, sigma and both subspaces within 1e-5."""
    A = synth.make_flow_316(grid=60, n=300)
    ref = O.isma(A.astype(np.float64), O.Params(k=20, c=40, seed=0x5107, tol=1e-8))
    g = run(A, 20, 40, precision="tf32x3")
    assert len(g["idx"]) == len(ref.trace)
    for t, rec in enumerate(ref.trace):
        assert np.array_equal(g["idx"][t], rec.idx)
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-5)
    assert O.sin_principal_max(ref.U, g["U"]) <= 1e-5
    assert O.sin_principal_max(ref.V, g["V"]) <= 1e-5


def test_isma_flow_ort_tensor_cores():
    """ORT weights (Eq. 6) from the tensor-core A^T U.  The weight
    s_j - |U^T a_j|^2 cancels for well-represented columns, so the FP32
    basis's difference from the FP64 oracle's (~1e-6) can move a quantised
    weight across a draw boundary after a few rounds; the first rounds' draws
    are compared bit-exactly, then the oracle's draws are replayed and the
    merges, refinement and the ORT path itself run to the end within 1e-5."""
    A = synth.make_flow_316(grid=100, n=600)
    A64 = A.astype(np.float64)
    ref = O.isma(A64, O.Params(k=20, c=40, seed=0x5107, tol=1e-8, col_strategy="ort"))
    ctx = pod.Context(to_dev(A), 20, 40, tol=1e-8, precision="tf32x3", col_strategy="ort")
    ctx.iterate(4)
    for t in range(4):
        assert np.array_equal(ctx.trace(t)[0], ref.trace[t].idx), t
    ctx.close()
    sets = [rec.idx for rec in ref.trace]
    rep = O.isma(A64, O.Params(k=20, c=40, seed=0x5107, tol=0.0, col_strategy="ort", replay=sets))
    ctx = pod.Context(to_dev(A), 20, 40, tol=0.0, precision="tf32x3", col_strategy="ort")
    ctx.replay(sets)
    done, meas, steps = ctx.iterate()
    assert steps == len(sets)
    U, s, V = ctx.modes(with_v=True)
    np.testing.assert_allclose(s.cpu().numpy(), rep.sigma, rtol=1e-5)
    assert O.sin_principal_max(rep.U, U.double().cpu().numpy()) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("strategy", ["ort", "l2n"])
def test_isma_planted_f64_strategies_bit_exact(strategy):
    """FP64 data (FP64 SIMT contractions): the ORT weights' cancellation
    stays far below a draw boundary, so every round's draws match."""
    A = synth.planted(3000, 200, 0.8 ** np.arange(40), 1e-6, 41, np.float64)
    ref = O.isma(A, O.Params(k=6, c=15, seed=0x5107, tol=1e-8, col_strategy=strategy))
    g = run(A, 6, 15, col_strategy=strategy)
    assert len(g["idx"]) == len(ref.trace)
    for t, rec in enumerate(ref.trace):
        assert np.array_equal(g["idx"][t], rec.idx), t
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-9)
    assert O.sin_principal_max(ref.U, g["U"]) <= 1e-9


def test_isma_flow_full_size_tensor_core_refinement():
    A = synth.make_flow_316()
    ref = O.isma(A.astype(np.float64), O.Params(k=20, c=40, seed=0x5107, tol=1e-8))
    g = run(A, 20, 40, precision="tf32x3")
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=1e-5)
    assert O.sin_principal_max(ref.U, g["U"]) <= 1e-5
    assert O.sin_principal_max(ref.V, g["V"]) <= 1e-5
