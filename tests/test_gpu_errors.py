"""Error paths of the C ABI on the GPU: a non-finite value in A (POD_ENAN)
and a tensor-core wait that runs out (POD_ETIMEOUT).  Both leave the context
poisoned (POD_ESTATE afterwards) and the CUDA context usable: a new problem
runs correctly after them.  No test makes the GPU fault, trap or hang: the
timeout comes from a small poll bound set through pod_set_wait_limit, and
the kernel that gives up still waits (with the default bound) for its own
copies and tensor-core operations before it returns."""
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
    return torch.from_numpy(np.asfortranarray(A).T.copy()).to(DEV).t()


def healthy_run():
    """A small problem after an error: the device and the library still work."""
    A = synth.planted(1200, 96, 0.8 ** np.arange(20), 1e-5, 3, np.float32)
    res = pod.pod(to_dev(A), k=4, c=8, tol=1e-8)
    torch.cuda.synchronize()
    ref = O.isma(A.astype(np.float64), O.Params(k=4, c=8, tol=1e-8))
    np.testing.assert_allclose(res.sigma.cpu().numpy(), ref.sigma, rtol=1e-5)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("where", ["nan", "inf"])
def test_non_finite_input_gives_enan_and_poisons(dtype, where):
    A = synth.planted(2000, 120, 0.8 ** np.arange(20), 1e-5, 5, dtype)
    A = np.asfortranarray(A)
    A[17, :] = np.nan if where == "nan" else np.inf   # every column holds it
    ctx = pod.Context(to_dev(A), 5, 10, tol=1e-8)
    with pytest.raises(pod.PodError) as e:
        ctx.iterate()
    assert e.value.status == pod.POD_ENAN
    with pytest.raises(pod.PodError) as e2:
        ctx.modes()
    assert e2.value.status == pod.POD_ESTATE
    with pytest.raises(pod.PodError) as e3:
        ctx.iterate()
    assert e3.value.status == pod.POD_ESTATE
    ctx.close()
    healthy_run()


def test_tensor_core_wait_timeout_is_reported_and_recovers():
    """The refinement's A^T U runs on the tensor cores (split TF32); with a
    pipeline-wait bound of one poll its first wait runs out: pod_modes
    returns POD_ETIMEOUT, the context is poisoned, and the GPU keeps working."""
    A = synth.planted(4096, 256, 0.8 ** np.arange(20), 1e-5, 7, np.float32)
    ctx = pod.Context(to_dev(A), 4, 16, tol=1e-8, precision="tf32x3")
    ctx.iterate()
    ctx.set_wait_limit(1)
    with pytest.raises(pod.PodError) as e:
        ctx.modes()
    assert e.value.status == pod.POD_ETIMEOUT
    with pytest.raises(pod.PodError) as e2:
        ctx.modes()
    assert e2.value.status == pod.POD_ESTATE
    with pytest.raises(pod.PodError):
        ctx.set_wait_limit(0)
    ctx.close()
    torch.cuda.synchronize()
    healthy_run()


def test_default_wait_limit_restored_runs_clean():
    """Setting the bound back to the default before any launch leaves the
    result unchanged."""
    A = synth.planted(4096, 256, 0.8 ** np.arange(20), 1e-5, 7, np.float32)
    ctx = pod.Context(to_dev(A), 4, 16, tol=1e-8, precision="tf32x3")
    ctx.set_wait_limit(1)
    ctx.set_wait_limit(0)
    ctx.iterate()
    U, s, _ = ctx.modes()
    ref = O.isma(A.astype(np.float64), O.Params(k=4, c=16, tol=1e-8))
    np.testing.assert_allclose(s.cpu().numpy(), ref.sigma, rtol=1e-5)
    ctx.close()
