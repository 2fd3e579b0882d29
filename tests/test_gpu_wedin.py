"""GPU parity of the Eq. 7 quality measure (Sec. 3.3) against the oracle."""
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


def gpu_wedin(A, k, c, r, **kw):
    ctx = pod.Context(to_dev(A), k, c, r=r, tol=1e-8, **kw)
    ctx.iterate()
    U, s, V = ctx.modes(with_v=True)
    w = ctx.wedin()
    ctx.close()
    return w, s.cpu().numpy()


def oracle_wedin(A, k, c, r):
    res = O.isma(np.asarray(A, dtype=np.float64), O.Params(k=k, c=c, r=r, seed=0x5107, tol=1e-8))
    return O.wedin_measure(np.asarray(A, dtype=np.float64), res.U, res.sigma, res.V, res.sigma_all[k])


def test_wedin_planted_f64():
    A = synth.make_planted_small()
    w, _ = gpu_wedin(A, 10, 20, 12)
    ref = oracle_wedin(A, 10, 20, 12)
    np.testing.assert_allclose(w["norm_R"], ref.norm_R, rtol=1e-6)
    np.testing.assert_allclose(w["omega"], ref.omega, rtol=1e-9)
    np.testing.assert_allclose(w["bound"], ref.bound, rtol=1e-6)
    assert w["norm_S"] <= 1e-12 * np.sqrt(np.sum(A * A))


def test_wedin_flow_f32_reduced():
    """FP32: |R| is a residual of the converged FP32 subspace; it agrees with
    the oracle's to the subspace accuracy (sin 1e-5 of sigma_1 ~ 1e2 at this
    size) and S vanishes to the FP32 refinement rounding."""
    A = synth.make_flow_316(grid=60, n=300)
    w, s = gpu_wedin(A, 20, 40, 22)
    ref = oracle_wedin(A, 20, 40, 22)
    sigma1 = float(s[0])
    assert abs(w["norm_R"] - ref.norm_R) <= 1e-4 * sigma1 + 1e-2 * ref.norm_R
    np.testing.assert_allclose(w["omega"], ref.omega, rtol=1e-3)
    assert w["norm_S"] <= 1e-5 * sigma1


def test_wedin_needs_refinement_and_spare_mode():
    A = synth.planted(500, 60, 0.8 ** np.arange(20), 1e-6, 31, np.float64)
    ctx = pod.Context(to_dev(A), 4, 8, r=4, tol=1e-8)
    ctx.iterate()
    with pytest.raises(pod.PodError) as e:
        ctx.wedin()
    assert e.value.status == pod.POD_ESTATE
    ctx.modes()
    with pytest.raises(pod.PodError) as e:
        ctx.wedin()
    assert e.value.status == pod.POD_EUNSUPPORTED
    ctx.close()
