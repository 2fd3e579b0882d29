"""Pins of the FP64 reference gradient (oracle/grad.py): its forward equals
the NumPy oracle's ISMA with replayed draws, and its autograd gradient equals
central finite differences of the NumPy oracle (an independent forward:
Householder QR + LAPACK SVD merges).  CPU only."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grad as Gd  # noqa: E402
from oracle import isma as O  # noqa: E402
from paper_1905_05107_gb300 import synth  # noqa: E402


def _case(seed=3, m=300, n=60, rank=20):
    A = synth.planted(m, n, 1.0 - 0.04 * np.arange(rank), 0.0, seed, np.float64)
    rng = np.random.default_rng(seed)
    sets = [np.sort(rng.choice(n, size=9, replace=False))]
    rest = np.setdiff1d(np.arange(n), sets[0])
    rng.shuffle(rest)
    for i in range(0, rest.size, 9):
        sets.append(np.sort(rest[i:i + 9]))
    return A, sets


def _oracle_loss(A, sets, k, r, w, g, ws):
    res = O.isma(A, O.Params(k=k, c=9, r=r, seed=0x5107, tol=0.0, replay=sets))
    val = float(np.sum(w * (res.U.T @ g) ** 2))
    if ws is not None:
        val += float(np.sum(ws * res.sigma))
    return val


def test_reference_forward_matches_oracle():
    A, sets = _case()
    U, s = Gd.forward(torch.tensor(A), sets, 4, 6)
    res = O.isma(A, O.Params(k=4, c=9, r=6, seed=0x5107, tol=0.0, replay=sets))
    np.testing.assert_allclose(s.numpy(), res.sigma, rtol=1e-12)
    assert O.sin_principal_max(res.U, U.numpy()) < 1e-11


@pytest.mark.parametrize("with_sigma", [False, True])
def test_reference_gradient_matches_oracle_finite_differences(with_sigma):
    A, sets = _case()
    k, r = 4, 6
    rng = np.random.default_rng(11)
    w = rng.uniform(0.5, 1.5, k)
    g = rng.standard_normal(A.shape[0])
    ws = rng.uniform(0.5, 1.5, k) if with_sigma else None
    G, L = Gd.gradient(A, sets, k, r, w, g, ws)
    assert abs(L - _oracle_loss(A, sets, k, r, w, g, ws)) <= 1e-10 * abs(L)
    h = 1e-6
    for _ in range(4):
        D = rng.standard_normal(A.shape)
        D /= np.linalg.norm(D)
        fd = (_oracle_loss(A + h * D, sets, k, r, w, g, ws) - _oracle_loss(A - h * D, sets, k, r, w, g, ws)) / (2 * h)
        assert abs(fd - np.sum(G * D)) <= 1e-6 * np.linalg.norm(G), (fd, np.sum(G * D))
