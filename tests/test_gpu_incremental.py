"""Algorithm 3 (incremental POD over column blocks streamed from host
memory) on the GPU against the oracle's incremental_pod."""
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


def host(A, pad=0):
    """Column-major pinned CPU tensor, optionally with a padded leading dimension."""
    m, n = A.shape
    buf = torch.zeros((n, m + pad), dtype=torch.float32 if A.dtype == np.float32 else torch.float64).pin_memory()
    buf[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T))
    return buf.t()[:m, :]


@pytest.mark.parametrize("blocks", [1, 4, 7])
def test_incremental_planted_f64(blocks):
    A = synth.make_planted_small()
    ref = O.incremental_pod(A, blocks, O.Params(k=10, c=20, seed=0x5107, tol=1e-8))
    U, s = pod.incremental(host(A), 10, 20, blocks, tol=1e-8)
    np.testing.assert_allclose(s.cpu().numpy(), ref.sigma, rtol=1e-10)
    np.testing.assert_allclose(U.cpu().numpy(), ref.U, atol=1e-9)


def test_incremental_padded_lda_and_uneven_blocks_f64():
    A = synth.planted(1203, 211, 0.8 ** np.arange(30), 1e-6, 61, np.float64)
    ref = O.incremental_pod(A, 5, O.Params(k=4, c=9, r=6, seed=0x5107, tol=1e-8))
    U, s = pod.incremental(host(A, pad=5), 4, 9, 5, r=6, tol=1e-8)
    np.testing.assert_allclose(s.cpu().numpy(), ref.sigma, rtol=1e-10)
    assert O.sin_principal_max(ref.U, U.cpu().numpy()) < 1e-9


def test_incremental_flow_f32():
    A = synth.make_flow_316(grid=100, n=600)
    ref = O.incremental_pod(A.astype(np.float64), 3, O.Params(k=20, c=40, seed=0x5107, tol=1e-8))
    U, s = pod.incremental(host(A), 20, 40, 3, tol=1e-8)
    np.testing.assert_allclose(s.cpu().numpy(), ref.sigma, rtol=1e-5)
    assert O.sin_principal_max(ref.U, U.double().cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-9), (np.float32, 5e-5)])
def test_incremental_wide_cores(dtype, tol):
    """k = 100, c = 200 (n_c = 300: wide tall passes, core SVD with its
    Jacobi arrays in global memory) on 4 column blocks.  FP32 bar: the cut
    at 100 of sigma_i = 0.97^i has a gap of 0.97^99 * 0.03 = 1.5e-3 of
    sigma_1, so FP32 determines the subspace to u sigma_1 / gap = 4e-5."""
    A = synth.planted(12000, 2400, 0.97 ** np.arange(400), 1e-6, 63, dtype)
    ref = O.incremental_pod(A.astype(np.float64), 4, O.Params(k=100, c=200, seed=0x5107, tol=1e-8))
    U, s = pod.incremental(host(A), 100, 200, 4, tol=1e-8)
    np.testing.assert_allclose(s.cpu().numpy(), ref.sigma, rtol=tol)
    assert O.sin_principal_max(ref.U, U.double().cpu().numpy()) <= tol
