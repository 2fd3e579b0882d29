"""GPU adjoint of the truncated POD (pod_backward) against the FP64
PyTorch-autograd reference of the same frozen-draw forward (oracle/grad.py),
and against central finite differences of the NumPy oracle."""
import numpy as np
import pytest

from oracle import grad as Gd
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


def gpu_grad(A, k, c, w, g, ws=None, **kw):
    """GPU forward with a tape, the loss gradient in U (and sigma) formed on
    the GPU, pod_backward -> dL/dA; also returns the forward's draws."""
    At = to_dev(A)
    ctx = pod.Context(At, k, c, keep_tape=True, tol=1e-8, **kw)
    done, meas, steps = ctx.iterate()
    sets = [ctx.trace(t)[0] for t in range(steps)]
    U, s, _ = ctx.modes()
    gt = torch.as_tensor(g, dtype=U.dtype, device=DEV)
    wt = torch.as_tensor(w, dtype=torch.float64, device=DEV)
    proj = (U.t().double() @ gt.double())                         # u_i^T g
    dU = (gt.double()[:, None] * (2.0 * wt * proj)[None, :]).to(U.dtype)
    ds = None if ws is None else torch.as_tensor(ws, dtype=torch.float64, device=DEV)
    dA = ctx.backward(dU, ds)
    out = dA.double().cpu().numpy()
    ctx.close()
    return out, sets


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("refine,with_sigma", [(True, False), (True, True), (False, False), (False, True)])
def test_backward_planted_f64_matches_autograd(refine, with_sigma):
    A = synth.planted(700, 90, 1.0 - 0.03 * np.arange(30), 1e-7, 51, np.float64)
    k, c, r = 4, 10, 6
    w, g = synth.diff_loss_weights(k, A.shape[0])
    ws = np.linspace(0.7, 1.3, k) if with_sigma else None
    G, sets = gpu_grad(A, k, c, w, g, ws, r=r, refine=refine)
    R, _ = Gd.gradient(A, sets, k, r, w, g, ws, refine=refine)
    assert rel(G, R) < 1e-8, rel(G, R)


def test_backward_planted_f32_matches_autograd():
    A = synth.make_diff_c4(m=20_000, n=200)
    k, c = 16, 32
    w, g = synth.diff_loss_weights(k, A.shape[0])
    G, sets = gpu_grad(A, k, c, w, g)
    R, _ = Gd.gradient(A.astype(np.float64), sets, k, k, w, g)
    assert rel(G, R) < 1e-4, rel(G, R)


def _fd_check(A, G, sets, k, c, w, g, directions, seed):
    """Central differences (h = 1e-3) of the FP64 oracle's loss with the run's
    draws frozen, along `directions` random unit directions D (Frobenius
    norm 1): |FD - <dL/dA, D>| <= 1e-3 |dL/dA|_F."""
    A64 = A.astype(np.float64)
    rng = np.random.default_rng(seed)
    h = 1e-3

    def L(X):
        res = O.isma(X, O.Params(k=k, c=c, seed=0x5107, tol=0.0, replay=sets))
        return float(np.sum(w * (res.U.T @ g) ** 2))

    gnorm = np.linalg.norm(G)
    worst = 0.0
    for _ in range(directions):
        D = rng.standard_normal(A.shape)
        D /= np.linalg.norm(D)
        fd = (L(A64 + h * D) - L(A64 - h * D)) / (2 * h)
        err = abs(fd - np.sum(G * D))
        worst = max(worst, err / gnorm)
        assert err <= 1e-3 * gnorm, (fd, np.sum(G * D))
    return worst


def test_backward_fd_64_directions_reduced():
    """The differentiation workload's spectrum and loss at m = 20000,
    n = 200 (k = 16, c = 32, FP32): the GPU adjoint against central finite
    differences of the FP64 oracle along 64 random directions."""
    A = synth.make_diff_c4(m=20_000, n=200)
    k, c = 16, 32
    w, g = synth.diff_loss_weights(k, A.shape[0])
    G, sets = gpu_grad(A, k, c, w, g)
    _fd_check(A, G, sets, k, c, w, g, 64, 11)


def test_backward_differentiation_workload_full_size():
    """m = 200000, n = 1000, k = 16, c = 32 (FP32): the GPU adjoint against
    the FP64 autograd reference of the same frozen draws, and against central
    finite differences (h = 1e-3) of the FP64 oracle along random unit
    directions: |FD - <dL/dA, D>| <= 1e-3 |dL/dA|_F."""
    A = synth.make_diff_c4()
    k, c = 16, 32
    w, g = synth.diff_loss_weights(k, A.shape[0])
    G, sets = gpu_grad(A, k, c, w, g)
    A64 = A.astype(np.float64)
    R, _ = Gd.gradient(A64, sets, k, k, w, g)
    assert rel(G, R) < 1e-4, rel(G, R)
    _fd_check(A, G, sets, k, c, w, g, 4, 7)
