"""Cores wider than shared memory (n_c = r + g beyond ~64 in FP32): the tall
passes keep their coefficient tiles and FP64 accumulators in global scratch,
the core SVD and the first CholeskyQR kernel their work arrays (the Jacobi
arrays stay in shared memory up to n_c ~ 160, then move to global memory
too).  Parity with the oracle as for the narrow path."""
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


def run(A, k, c, **kw):
    ctx = pod.Context(to_dev(A), k, c, **kw)
    done, meas, steps = ctx.iterate()
    idx = [ctx.trace(t)[0] for t in range(steps)]
    U, s, _ = ctx.modes()
    out = dict(U=U.double().cpu().numpy(), sigma=s.cpu().numpy(), idx=idx)
    ctx.close()
    return out


@pytest.mark.parametrize("m,n,k,c,dtype,tol", [
    (20000, 400, 20, 60, np.float32, 1e-5),     # previously beyond shared memory
    (30000, 800, 50, 100, np.float64, 1e-9),    # the precision configuration's k, c
    (30000, 800, 50, 100, np.float32, 1e-5),
    (20000, 1200, 100, 200, np.float64, 1e-9),  # the out-of-core configuration's k, c (n_c = 300)
])
def test_wide_planted(m, n, k, c, dtype, tol):
    sigma = 0.95 ** np.arange(min(n, 3 * k))
    A = synth.planted(m, n, sigma, 1e-6, 71, dtype)
    ref = O.isma(A.astype(np.float64), O.Params(k=k, c=c, seed=0x5107, tol=1e-8))
    g = run(A, k, c, tol=1e-8)
    assert len(g["idx"]) == len(ref.trace)
    for t, rec in enumerate(ref.trace):
        assert np.array_equal(g["idx"][t], rec.idx), t
    np.testing.assert_allclose(g["sigma"], ref.sigma, rtol=tol)
    assert O.sin_principal_max(ref.U, g["U"]) <= tol
