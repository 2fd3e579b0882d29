"""Pins for the oracle's BLOCK MERGE (Algorithm 2, Eqs. 8-9), the ISMA loop
(Algorithm 1), the closing refinement and Algorithm 3, against LAPACK's SVD
of the whole matrix, planted and closed-form spectra, and invariants.
CPU only."""
import numpy as np
import pytest

from oracle import isma as O
from paper_1905_05107_gb300 import synth


def _svd(X):
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    return U, s, Vt.T


def _sin(U, W):
    return O.sin_principal_max(U, W)


@pytest.mark.parametrize("m,n1,n2", [(60, 7, 5), (40, 12, 30), (25, 3, 1)])
def test_merge_of_exact_factors_is_svd_of_concatenation(m, n1, n2):
    """Eqs. 8-9: merging the exact SVD of X with a block Y, untruncated,
    reproduces the SVD of [X Y]."""
    rng = np.random.default_rng(m + n1 + n2)
    X = rng.standard_normal((m, n1))
    Y = rng.standard_normal((m, n2))
    Ux, sx, _ = _svd(X)
    res = O.block_merge(Ux, sx, Y, r=n1 + n2)
    Ur, sr, _ = _svd(np.hstack([X, Y]))
    np.testing.assert_allclose(res.sigma, sr, rtol=1e-12)
    assert _sin(Ur, res.U) < 1e-12
    # the merged factors reproduce the concatenation's column space energy
    np.testing.assert_allclose(res.U.T @ res.U, np.eye(res.U.shape[1]), atol=1e-13)


def test_merge_block_given_as_scaled_factor():
    """Passing the new block as U_2 Sigma_2 or as Y itself (Y = U_2 Sigma_2 V_2^T,
    V_2 square) gives the same merged factors (Eq. 8's E differs only by V_2)."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((50, 6))
    Y = rng.standard_normal((50, 4))
    Ux, sx, _ = _svd(X)
    Uy, sy, _ = _svd(Y)
    a = O.block_merge(Ux, sx, Y, r=10)
    b = O.block_merge(Ux, sx, Uy * sy, r=10)
    np.testing.assert_allclose(a.sigma, b.sigma, rtol=1e-12)
    assert _sin(a.U, b.U) < 1e-12


def test_merge_into_empty_basis_is_svd():
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((30, 8))
    res = O.block_merge(np.zeros((30, 0)), np.zeros(0), Y, r=5)
    Uy, sy, _ = _svd(Y)
    np.testing.assert_allclose(res.sigma, sy[:5], rtol=1e-12)
    assert _sin(Uy[:, :5], res.U) < 1e-12


def test_merge_drops_zero_singular_values():
    """Algorithm 2 keeps min(r, number of non-zero sigma)."""
    rng = np.random.default_rng(2)
    X = rng.standard_normal((40, 3))
    Ux, sx, _ = _svd(X)
    Y = X @ rng.standard_normal((3, 4))     # inside span(X)
    res = O.block_merge(Ux, sx, Y, r=6)
    assert res.U.shape[1] == 3


def test_merge_truncation_is_best_rank_r_of_merged_factors():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((70, 9))
    Y = rng.standard_normal((70, 6))
    Ux, sx, _ = _svd(X)
    res = O.block_merge(Ux, sx, Y, r=4)
    Ur, sr, _ = _svd(np.hstack([X, Y]))
    np.testing.assert_allclose(res.sigma, sr[:4], rtol=1e-12)
    assert _sin(Ur[:, :4], res.U) < 1e-11


def test_mat_error_bound_sequence():
    """Sec. 3.2.1: after a series of MAT operations over P partitions,
    ||X - Z_r||_2 <= (2^(P+1) - 3) sigma_{r+1}(X); the projection of X on the
    merged modes is at least as good as Z_r."""
    rng = np.random.default_rng(8)
    m, r = 80, 5
    s_true = 0.7 ** np.arange(40)
    X = (synth.haar(rng, m, 40) * s_true) @ synth.haar(rng, 48, 40).T
    X += 1e-3 * rng.standard_normal(X.shape)
    sigma_X = np.linalg.svd(X, compute_uv=False)
    for P in (2, 3, 4, 6):
        parts = np.array_split(np.arange(48), P)
        U, s = np.zeros((m, 0)), np.zeros(0)
        for cols in parts:
            Ub, sb, _ = _svd(X[:, cols])
            res = O.block_merge(U, s, Ub[:, :r] * sb[:r], r)
            U, s = res.U, res.sigma
        err = np.linalg.norm(X - U @ (U.T @ X), 2)
        assert err <= (2 ** (P + 1) - 3) * sigma_X[r] * (1 + 1e-12)


def test_convergence_measure_matches_principal_angles():
    """sin(theta) read from U_E[k:, :k] equals the principal angles between
    the old and the merged top-k modes computed in R^m."""
    rng = np.random.default_rng(12)
    m, k = 90, 4
    X = rng.standard_normal((m, 10)) * (0.8 ** np.arange(10))
    U1, s1, _ = _svd(X)
    U1, s1 = U1[:, :k], s1[:k]
    C = rng.standard_normal((m, 6)) * 0.5
    res = O.block_merge(U1, s1, C, r=k)
    sin_max, cos_min = O.convergence_measures(res.UE, k, k)
    assert abs(sin_max - _sin(U1, res.U[:, :k])) < 1e-12
    cosines = np.abs(np.sum(U1 * res.U[:, :k], axis=0))
    assert abs(cos_min - cosines.min()) < 1e-12


def _params(**kw):
    base = dict(k=3, c=6, tol=0.0, refine=False, seed=17)
    base.update(kw)
    return O.Params(**base)


def test_isma_full_rank_carried_equals_lapack_svd():
    """With r >= rank and the loop run until S is empty, ISMA is the exact
    truncated SVD (every column has been merged without loss)."""
    rng = np.random.default_rng(21)
    A = rng.standard_normal((120, 30))
    A -= A.mean(axis=1, keepdims=True)
    res = O.isma(A, _params(k=5, r=30, c=7))
    assert res.trace[-1].remaining == 0
    U, s, _ = _svd(A)
    np.testing.assert_allclose(res.sigma, s[:5], rtol=1e-12)
    assert _sin(U[:, :5], res.U) < 1e-11
    for i in range(5):
        assert abs(abs(U[:, i] @ res.U[:, i]) - 1) < 1e-12


def test_isma_planted_noiseless_exact():
    """A = U diag(sigma) V^T of rank 6 with r = 6: once the draws span
    col(A) the modes and sigma are exact (closed form)."""
    Ut, st, Vt = synth.planted_factors(200, 60, [5, 4, 3, 2, 1, 0.5], 3)
    A = (Ut * st) @ Vt.T
    res = O.isma(A, _params(k=4, r=6, c=10, refine=False))
    np.testing.assert_allclose(res.sigma, st[:4], rtol=1e-12)
    assert _sin(Ut[:, :4], res.U) < 1e-12


def test_isma_flow_closed_form_spectrum():
    """Separable travelling waves on an integer grid are exactly orthogonal:
    sigma = amp_j sqrt(m n / 8), each twice (noiseless, uncentred)."""
    grid, n, modes = 20, 48, 5
    A = synth.flow(grid, n, modes, 0.0, 7, dtype=np.float64, center=False, max_k=8, max_omega=20)
    expect = synth.flow_spectrum(grid, n, modes, 7, max_k=8, max_omega=20)
    res = O.isma(A, _params(k=10, r=10, c=9, refine=True))
    np.testing.assert_allclose(res.sigma, expect, rtol=1e-11)
    # pairs are degenerate: compare the subspaces of whole pairs only
    Ua, _, _ = _svd(A)
    assert _sin(Ua[:, :10], res.U) < 1e-10


def test_isma_orthonormal_and_deterministic():
    A = synth.planted(150, 80, 0.8 ** np.arange(20), 1e-4, 4, np.float64)
    p = _params(k=4, r=4, c=8, col_strategy="unf")
    a = O.isma(A, p)
    b = O.isma(A, p)
    np.testing.assert_allclose(a.U.T @ a.U, np.eye(4), atol=1e-13)
    assert [t.idx.tolist() for t in a.trace] == [t.idx.tolist() for t in b.trace]
    assert np.array_equal(a.U, b.U)


def test_isma_trace_partitions_columns():
    """Every round draws only from S and S shrinks by exactly I_c."""
    A = synth.planted(100, 70, 0.9 ** np.arange(15), 1e-3, 6, np.float64)
    res = O.isma(A, _params(k=3, c=9))
    seen = set()
    for rec in res.trace:
        assert not (set(rec.idx.tolist()) & seen)
        seen |= set(rec.idx.tolist())
        assert rec.remaining == 70 - len(seen)
    assert res.trace[-1].remaining == 0


def test_first_round_is_column_norm_sampling():
    """Round 0 uses Eq. 2 (a zero column is never drawn in round 0)."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((30, 40))
    A[:, 5] = 0.0
    A[:, 11] = 0.0
    for seed in range(20):
        res = O.isma(A, _params(k=2, c=10, seed=seed, max_iter=0))
        assert 5 not in res.trace[0].idx and 11 not in res.trace[0].idx


def test_ort_weights_are_residual_norms():
    """Eq. 6: |a_i - U U^T a_i|^2 by explicit projection."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((25, 12))
    U, _ = np.linalg.qr(rng.standard_normal((25, 3)))
    s = O.column_sq_norms(A)
    vals = O.column_values("ort", 1, s, A, U)
    direct = np.array([np.sum((A[:, j] - U @ (U.T @ A[:, j])) ** 2) for j in range(12)])
    np.testing.assert_allclose(vals, direct, rtol=1e-10, atol=1e-12)


def test_refinement_sigma_and_right_vectors():
    """QR(A^T U), SVD(R): sigma are the singular values of U^T A and
    U^T A = Sigma V^T."""
    A = synth.planted(120, 50, 0.7 ** np.arange(12), 1e-3, 9, np.float64)
    res = O.isma(A, _params(k=4, r=4, c=8, refine=True))
    s_proj = np.linalg.svd(res.U.T @ A, compute_uv=False)
    np.testing.assert_allclose(res.sigma, s_proj, rtol=1e-12)
    np.testing.assert_allclose(res.U.T @ A, np.diag(res.sigma) @ res.V.T, atol=1e-12)
    np.testing.assert_allclose(res.V.T @ res.V, np.eye(4), atol=1e-13)


def test_signs_follow_reference_vector():
    A = synth.planted(80, 30, 0.6 ** np.arange(8), 1e-4, 2, np.float64)
    res = O.isma(A, _params(k=3, r=3, c=6, refine=True))
    z = O.sign_reference(17, 80)
    assert np.all(res.U.T @ z > 0)


def test_paper_literal_equals_direct_when_block_untruncated():
    """With r >= g the rank-r truncation of GET UPDATE keeps the whole block."""
    A = synth.planted(90, 40, 0.8 ** np.arange(10), 1e-3, 5, np.float64)
    a = O.isma(A, _params(k=3, r=8, c=6))
    b = O.isma(A, _params(k=3, r=8, c=6, paper_literal=True))
    np.testing.assert_allclose(a.sigma, b.sigma, rtol=1e-10)
    assert _sin(a.U, b.U) < 1e-10


def test_icrs_first_round_orthonormal_and_converges_to_svd_on_low_rank():
    """ICRS (rows = 1): the merged modes are orthonormal, and on an exactly
    rank-r matrix every round's D V~_r lies in col(A), so the final modes
    span col(A)."""
    Ut, st, Vt = synth.planted_factors(300, 60, [3, 2, 1], 8)
    A = (Ut * st) @ Vt.T
    res = O.isma(A, _params(k=3, r=3, c=12, rows=1, w=150, refine=True))
    np.testing.assert_allclose(res.U.T @ res.U, np.eye(3), atol=1e-12)
    assert _sin(Ut, res.U) < 1e-10
    np.testing.assert_allclose(res.sigma, st, rtol=1e-10)


def test_replay_reproduces_sampled_run():
    A = synth.planted(100, 50, 0.8 ** np.arange(10), 1e-3, 3, np.float64)
    a = O.isma(A, _params(k=3, c=7))
    b = O.isma(A, _params(k=3, c=7, replay=[t.idx for t in a.trace]))
    assert np.array_equal(a.U, b.U)


def test_incremental_pod_exact_on_low_rank():
    """Algorithm 3 with r >= rank: one pass over 4 blocks recovers the SVD."""
    Ut, st, Vt = synth.planted_factors(150, 80, [4, 3, 2, 1], 13)
    A = (Ut * st) @ Vt.T
    res = O.incremental_pod(A, 4, _params(k=3, r=4, c=8))
    np.testing.assert_allclose(res.sigma, st[:3], rtol=1e-11)
    assert _sin(Ut[:, :3], res.U) < 1e-10


def test_modes_criterion_stops_early_on_exact_low_rank():
    Ut, st, Vt = synth.planted_factors(120, 90, [5, 3, 1], 6)
    A = (Ut * st) @ Vt.T
    res = O.isma(A, _params(k=2, r=3, c=10, criterion="modes", tol=0.999))
    assert res.converged and res.trace[-1].remaining > 0
