"""The precision forms of the dense contractions on the tcgen05 tensor cores:
split-TF32 (POD_PREC_TF32X3), split-BF16 (POD_PREC_BF16X3) and BF16
(POD_PREC_BF16) products for A^T U (the refinement's QR(A^T U), the ORT
weights of Eq. 6) and U^T C (BLOCK MERGE's projection, Algorithm 2), checked
against the FP64 definition and, through whole ISMA runs, against the FP64
oracle.

Per-entry bars for A^T U follow the arithmetic: each product carries a
relative error of about 2^-21 (TF32X3), 2^-16 (BF16X3) or 2^-8 (BF16), and
the tensor cores accumulate 64 rows in FP32, so |Y - Y_64| <= c u_eff
(|A|^T |U|) with u_eff = 2^-19, 2^-15, 2^-7.  Whole runs: the benchmark spec's
BF16-split tolerances (sigma relative and sin(theta) <= 1e-3); the BF16
form is held to 1e-2."""
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
U_EFF = {"tf32x3": 2.0 ** -19, "bf16x3": 2.0 ** -15, "bf16": 2.0 ** -7}


def to_dev(A):
    return torch.from_numpy(np.asfortranarray(A).T.copy()).to(DEV).t()


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "bf16"])
@pytest.mark.parametrize("m,n,r", [(1028, 300, 20), (4096, 128, 64), (65540, 1000, 50), (200, 7, 1), (33000, 2, 33)])
def test_atu_tensor_core_forms(prec, m, n, r):
    """Ragged m (a partial last slab), several ragged M-tiles of 128 columns,
    r from 1 to 64, work ranges that cross M-tile boundaries."""
    rng = np.random.default_rng(m + n + r)
    A = (rng.standard_normal((m, n)) * rng.random(n) * 3).astype(np.float32)
    U = rng.standard_normal((m, r)).astype(np.float32)
    Y = pod.atu(to_dev(A), to_dev(U), precision=prec).cpu().numpy()
    A64, U64 = A.astype(np.float64), U.astype(np.float64)
    ref = A64.T @ U64
    scale = np.abs(A64).T @ np.abs(U64)
    err = np.abs(Y - ref) / scale
    assert err.max() <= 4 * U_EFF[prec], (prec, err.max())


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "bf16"])
def test_atu_tensor_core_forms_repeatable(prec):
    """Fixed-order sums: two calls give bit-identical results."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((8192, 640)).astype(np.float32)
    U = rng.standard_normal((8192, 40)).astype(np.float32)
    Ad, Ud = to_dev(A), to_dev(U)
    Y1 = pod.atu(Ad, Ud, precision=prec).cpu().numpy()
    Y2 = pod.atu(Ad, Ud, precision=prec).cpu().numpy()
    assert np.array_equal(Y1, Y2)


def run(A, k, c, prec, **kw):
    ctx = pod.Context(to_dev(A), k, c, tol=1e-8, precision=prec, **kw)
    done, meas, steps = ctx.iterate()
    idx = [ctx.trace(t)[0] for t in range(steps)]
    U, s, _ = ctx.modes()
    torch.cuda.synchronize()
    out = dict(U=U.double().cpu().numpy(), sigma=s.cpu().numpy(), steps=steps, idx=idx)
    ctx.close()
    return out


@pytest.mark.parametrize("prec,bar", [("bf16x3", 1e-3), ("bf16", 1e-2), ("tf32x3", 1e-5)])
@pytest.mark.parametrize("case", ["flow", "planted"])
def test_isma_precision_forms_against_oracle(prec, bar, case):
    """Whole ISMA runs (U^T C and A^T U in the given form, the Grams, core SVD
    and convergence test at FP32 / FP64 level): every draw identical, sigma
    and the k-subspace within the form's bar of the FP64 oracle."""
    if case == "flow":
        A, k, c = synth.make_flow_316(grid=100, n=600), 20, 40
    else:
        A, k, c = synth.planted(8192, 400, np.exp(-np.arange(60) / 15.0), 1e-4, 23, np.float32), 10, 24
    ref = O.isma(A.astype(np.float64), O.Params(k=k, c=c, tol=1e-8, seed=0x5107))
    g = run(A, k, c, prec)
    assert g["steps"] == len(ref.trace)
    for t, rec in enumerate(ref.trace):
        assert np.array_equal(g["idx"][t], rec.idx), t
    rel = np.max(np.abs(g["sigma"] - ref.sigma) / ref.sigma)
    sin = O.sin_principal_max(ref.U, g["U"])
    assert rel <= bar and sin <= bar, (prec, rel, sin)


def test_ort_draws_with_bf16x3_weights_follow_the_oracle_first_rounds():
    """ORT weights from A^T U in split BF16: the first rounds' draws match the
    oracle's (later rounds may move a quantised weight across a draw
    boundary, as with FP32 data)."""
    A = synth.planted(4096, 300, 0.85 ** np.arange(40), 1e-5, 31, np.float32)
    k, c = 6, 12
    ref = O.isma(A.astype(np.float64), O.Params(k=k, c=c, tol=1e-8, col_strategy="ort", max_iter=2))
    g = run(A, k, c, "bf16x3", col_strategy="ort", max_iter=2)
    assert g["steps"] == len(ref.trace) == 3
    assert np.array_equal(g["idx"][0], ref.trace[0].idx)
    assert np.array_equal(g["idx"][1], ref.trace[1].idx)
