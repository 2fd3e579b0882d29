"""Pins of the oracle's quality measure (Sec. 3.3, Eq. 7, Wedin's bound)
against closed forms and the theorem itself.  CPU only."""
import numpy as np

from oracle import isma as O
from paper_1905_05107_gb300 import synth


def _exact(A, k):
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    return U, s, Vt.T


def _sin_fro(X, Y):
    """|sin Theta|_F between the column spans of orthonormal X and Y."""
    c = np.linalg.svd(X.T @ Y, compute_uv=False)
    return float(np.sqrt(np.sum(np.maximum(0.0, 1.0 - c * c))))


def test_exact_triplets_give_zero_residuals():
    A = synth.planted(300, 80, 0.8 ** np.arange(30), 0.0, 91, np.float64)
    U, s, V = _exact(A, 6)
    w = O.wedin_measure(A, U[:, :6], s[:6], V[:, :6], s[6])
    assert w.norm_R <= 1e-12 * s[0] and w.norm_S <= 1e-12 * s[0]
    assert w.bound <= 1e-10


def test_scaled_singular_values_closed_form():
    """Exact vectors, sigma scaled by (1 + d): R = -d U S and S = -d V S, so
    |R| = |S| = d |sigma| and the bound is sqrt(2) d |sigma| / omega with
    omega = min(|sigma_k (1 + d) - sigma_{k+1}|, sigma_k (1 + d))."""
    A = synth.planted(250, 60, 0.7 ** np.arange(25), 0.0, 92, np.float64)
    U, s, V = _exact(A, 5)
    d = 1e-3
    st = s[:5] * (1 + d)
    w = O.wedin_measure(A, U[:, :5], st, V[:, :5], s[5])
    ref = d * np.linalg.norm(s[:5])
    assert abs(w.norm_R - ref) <= 1e-12 * s[0] and abs(w.norm_S - ref) <= 1e-12 * s[0]
    omega = min(abs(st[-1] - s[5]), st[-1])
    assert abs(w.omega - omega) <= 1e-15
    assert abs(w.bound - np.sqrt(2) * ref / omega) <= 1e-9 * w.bound


def test_bound_holds_for_perturbed_subspaces():
    """Wedin's theorem: sqrt(|sin Theta|^2 + |sin Phi|^2) <= sqrt(|R|^2 + |S|^2)
    / omega, omega from the true spectrum, for rotated approximate bases."""
    rng = np.random.default_rng(7)
    A = synth.planted(400, 120, 0.75 ** np.arange(40), 1e-6, 93, np.float64)
    Ue, s, Ve = _exact(A, 8)
    k = 8
    for eps in (1e-6, 1e-4, 1e-2):
        Ut, _ = np.linalg.qr(Ue[:, :k] + eps * rng.standard_normal((A.shape[0], k)))
        Vt, _ = np.linalg.qr(Ve[:, :k] + eps * rng.standard_normal((A.shape[1], k)))
        Ut = Ut * np.sign(np.diag(Ue[:, :k].T @ Ut))[None, :]   # QR may flip columns
        Vt = Vt * np.sign(np.diag(Ve[:, :k].T @ Vt))[None, :]
        sig = np.diag(Ut.T @ A @ Vt).copy()
        w = O.wedin_measure(A, Ut, sig, Vt, s[k])
        omega_true = min(np.min(np.abs(sig[-1] - s[k:])), sig[-1])
        lhs = np.hypot(_sin_fro(Ue[:, :k], Ut), _sin_fro(Ve[:, :k], Vt))
        rhs = np.hypot(w.norm_R, w.norm_S) / omega_true
        assert lhs <= rhs * (1 + 1e-9), (eps, lhs, rhs)
        assert rhs < 50 * lhs + 1e-12   # not vacuous


def test_isma_result_is_within_its_measure():
    """The planted FP64 workload after ISMA and refinement (r = k + 2 so that
    sigma_{k+1} exists): the true principal-angle error is below the Eq. 7
    measure, which is far below the sqrt(2k) that Sec. 3.3 names as the sign of
    an unconverged or ill-separated result."""
    A = synth.make_planted_small()
    k = 10
    res = O.isma(A, O.Params(k=k, c=20, r=k + 2, seed=0x5107, tol=1e-8))
    w = O.wedin_measure(A, res.U, res.sigma, res.V, res.sigma_all[k])
    Ue, s, Ve = _exact(A, k)
    lhs = np.hypot(_sin_fro(Ue[:, :k], res.U), _sin_fro(Ve[:, :k], res.V))
    assert lhs <= w.bound
    assert w.bound < 0.05 * np.sqrt(2 * k)
    assert w.norm_S <= 1e-10 * res.sigma[0]   # A^T U = V Sigma after the refinement
