"""Pins for the oracle's random draws: Philox4x32-10, integer weights, the
selection rule, and the row scaling of SAMPLE AND SCALE UNIQUE ROWS
(Algorithm 1).  CPU only."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

from oracle import isma as O


def _curand():
    for name in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if name and (os.path.exists(name) or not name.startswith("/")):
            try:
                return ctypes.CDLL(name)
            except OSError:
                pass
    return None


PHILOX_HOST = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10


def _curand_block(lib, seed, offset, words):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX_HOST) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(words, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(words)) == 0
        return out
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 0x5107, 0xDEADBEEF12345678, (1 << 64) - 1])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host-side Philox4_32_10 generator is an independent
    implementation.  Its output block b at offset o (in 32-bit words) is
    Philox(counter = (B mod 2^32, B >> 32, b mod 65536, 0)) with
    B = (o/4 + b) >> 16, key = (seed low, seed high): this covers every
    counter word the sampler uses (j, t, stream) and both key words."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    k0, k1 = O.seed_key(seed)
    for base_block in [0, 3 << 16, (5 << 16) + 7, ((1 << 32) + 2) << 16]:
        out = _curand_block(lib, seed, 4 * base_block, 64).reshape(-1, 4)
        for b in range(out.shape[0]):
            blk = base_block + b
            hi = blk >> 16
            x = O.philox4x32_10([hi & O.MASK32], [hi >> 32], [blk & 0xFFFF], [0], k0, k1)
            got = [int(v[0]) for v in x]
            assert got == [int(v) for v in out[b]], (seed, blk)


def test_uniform_u64_layout():
    """u = (x0 << 32) | x1 of Philox(j, t, stream, 0)."""
    k0, k1 = O.seed_key(0x1234)
    u = O.uniform_u64(0x1234, 7, 1, 5)
    for j in range(5):
        x = O.philox4x32_10([j], [7], [1], [0], k0, k1)
        assert u[j] == (int(x[0][0]) << 32) | int(x[1][0])


def _select_brute(weights, v):
    acc = 0
    for i, w in enumerate(weights):
        acc += int(w)
        if acc > v:
            return i
    raise AssertionError("v beyond total")


def test_selection_rule_exhaustive():
    """Every v in [0, W) maps to the smallest i with prefix_i > v; zero
    weights are never chosen (brute force over small weight vectors)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        w = rng.integers(0, 4, size=rng.integers(1, 9)).astype(np.uint64)
        if int(w.sum()) == 0:
            continue
        cdf = np.cumsum(w, dtype=np.uint64)
        for v in range(int(w.sum())):
            i = int(np.searchsorted(cdf, np.uint64(v), side="right"))
            assert i == _select_brute(w, v)
            assert w[i] > 0


def test_mulhi_range():
    """v = floor(u W / 2^64) spans exactly [0, W)."""
    W = (1 << 61) + 12345
    assert (0 * W) >> 64 == 0
    assert (((1 << 64) - 1) * W) >> 64 == W - 1


def test_quantize_bounds_and_masking():
    s = np.array([4.0, 1.0, 0.0, 2.0, 8.0])
    active = np.array([True, True, True, True, False])
    w = O.quantize(s, active)
    L = O.weight_bits(5)
    assert int(w[0]) == 1 << L          # the active maximum maps to 2^L
    assert int(w[1]) == 1 << (L - 2)
    assert int(w[2]) == 0 and int(w[4]) == 0
    assert int(w.sum()) < (1 << 62)


def test_draw_frequencies_chi_square():
    """20000 draws follow the weights (chi-square, 5 dof, p > 1e-4)."""
    w = np.array([1, 0, 3, 6, 0, 2, 8], dtype=np.uint64) << np.uint64(40)
    d = O.draw(w, 20000, 99, 0, O.STREAM_COLS)
    counts = np.bincount(d, minlength=w.size)
    assert counts[1] == 0 and counts[4] == 0
    p = w.astype(np.float64) / float(w.sum())
    nz = p > 0
    expected = 20000 * p[nz]
    chi2 = float(((counts[nz] - expected) ** 2 / expected).sum())
    assert chi2 < 25.7  # chi-square 5 dof, upper tail 1e-4


def test_sample_columns_only_from_S_sorted_distinct():
    n = 300
    s = np.random.default_rng(1).random(n)
    in_S = np.ones(n, dtype=bool)
    in_S[::3] = False
    idx, _ = O.sample_columns(s, in_S, 50, 7, 2)
    assert np.all(in_S[idx])
    assert np.all(np.diff(idx) > 0)


def test_sample_columns_uniform_fallback_when_weights_vanish():
    n = 40
    in_S = np.zeros(n, dtype=bool)
    in_S[[3, 9, 17]] = True
    idx, _ = O.sample_columns(np.zeros(n), in_S, 30, 5, 1)
    assert set(idx.tolist()) <= {3, 9, 17} and len(idx) > 0


def test_row_scaling_matches_duplicates():
    """Dedupe + sqrt(t_hat/(w q)) scaling gives the same W^T W as keeping
    every drawn row with scale 1/sqrt(w q) (Sec. 3.1, row sampling)."""
    rng = np.random.default_rng(11)
    D = rng.standard_normal((40, 6))
    vals = np.sum(D * D, axis=1)
    w = 200
    W, rows, counts = O.sample_scale_rows(D, vals, w, 21, 3)
    assert counts.sum() == w and len(rows) < w
    wq = O.quantize(vals, np.ones(40, dtype=bool))
    q = wq.astype(np.float64) / float(int(wq.sum(dtype=np.uint64)))
    draws = O.draw(wq, w, 21, 3, O.STREAM_ROWS)
    Wdup = np.stack([D[i] / np.sqrt(w * q[i]) for i in draws])
    np.testing.assert_allclose(W.T @ W, Wdup.T @ Wdup, rtol=1e-12, atol=1e-12)


def test_sign_reference_range():
    z = O.sign_reference(5, 1000)
    assert z.min() >= -1.0 and z.max() < 1.0
    assert abs(z.mean()) < 0.1


def test_eq5_row_count_hand_computed():
    """Eq. 5, c = w = k^2 (1 + sqrt(log(2 / delta)))^2 / epsilon^4 (natural
    log), worked by hand for epsilon = delta = 0.6 (the YF row of the paper's
    parameter table):
      log(2 / 0.6) = 1.2039728, sqrt = 1.0972569, (1 + 1.0972569)^2 = 4.3984866,
      0.6^4 = 0.1296;
      k = 5 : 25 * 4.3984866 / 0.1296 = 848.47  -> 849
      k = 20: 400 * 4.3984866 / 0.1296 = 13575.6 -> 13576
      k = 2 : 4 * 4.3984866 / 0.1296 = 135.76   -> 136."""
    assert O.rows_eq5(5, 0.6, 0.6) == 849
    assert O.rows_eq5(20, 0.6, 0.6) == 13576
    assert O.rows_eq5(2, 0.6, 0.6) == 136


def test_eq3_column_count_hand_computed():
    """Eq. 3, c = 4 k (1 + sqrt(8 log(1 / delta)))^2 / epsilon^2, by hand for
    k = 5, epsilon = delta = 0.6: log(1 / 0.6) = 0.5108256, 8x = 4.0866049,
    sqrt = 2.0215353, (1 + 2.0215353)^2 = 9.1296759, 20 * 9.1296759 / 0.36 =
    507.20 -> 508."""
    assert O.columns_eq3(5, 0.6, 0.6) == 508


def _capture_row_values(monkeypatch):
    seen = {}
    real = O.sample_scale_rows

    def spy(D, row_values, w, seed, t):
        seen["values"] = np.array(row_values, copy=True)
        out = real(D, row_values, w, seed, t)
        seen["rows"], seen["counts"] = out[1], out[2]
        return out

    monkeypatch.setattr(O, "sample_scale_rows", spy)
    return seen


def test_leverage_row_values_closed_form(monkeypatch):
    """Leverage-score row probabilities (Sec. 3.1, Table 2: q_i = |u^i|^2 / k
    over the first k current modes).  U carries r = 4 > k = 2 modes: its
    first two columns live on rows 0..3 as the orthonormal pair
    (1, 1, 1, 1) / 2 and (1, -1, 1, -1) / 2, so each of those rows has
    |u^i|^2 = 1/4 + 1/4 and q_i = 1/4; the extra modes live on rows 10 and
    11 and must not count.  D is zero on rows 0..3 and large elsewhere, so
    row values taken from D, or from all r columns of U, would differ."""
    m, n = 40, 12
    rng = np.random.default_rng(3)
    A = rng.standard_normal((m, n))
    A[0:4, :] = 0.0
    U = np.zeros((m, 4))
    U[0:4, 0] = 0.5
    U[0:4, 1] = [0.5, -0.5, 0.5, -0.5]
    U[10, 2] = 1.0
    U[11, 3] = 1.0
    seen = _capture_row_values(monkeypatch)
    p = O.Params(k=2, c=3, r=4, rows=1, w=64, row_strategy="ls")
    O.new_block(A, np.array([1, 5, 7]), p, 1, U)
    want = np.zeros(m)
    want[0:4] = 0.25
    np.testing.assert_array_equal(seen["values"], want)
    # all draws on rows 0..3; the four weights are equal, so draw j picks
    # support row floor(u_j * 4 / 2^64) (the selection rule on equal weights)
    us = O.uniform_u64(p.seed, 1, O.STREAM_ROWS, p.w)
    expect = np.bincount([(u * 4) >> 64 for u in us], minlength=4)
    np.testing.assert_array_equal(seen["rows"], np.flatnonzero(expect))
    np.testing.assert_array_equal(seen["counts"], expect[expect > 0])


def test_leverage_rows_fall_back_to_d_norms_without_modes(monkeypatch):
    """Round 0 has no modes: the LS strategy takes the L2 norms of D's rows
    (Alg. 1, GET UPDATE with rows), here a closed form for a D with two
    non-zero rows."""
    m, n = 30, 6
    A = np.zeros((m, n))
    A[4, :] = 2.0
    A[9, :] = [1.0, 0, 0, 3.0, 0, 0]
    seen = _capture_row_values(monkeypatch)
    p = O.Params(k=2, c=2, rows=1, w=16, row_strategy="ls")
    O.new_block(A, np.array([0, 3]), p, 0, np.zeros((m, 0)))
    want = np.zeros(m)
    want[4] = 8.0
    want[9] = 10.0
    np.testing.assert_array_equal(seen["values"], want)
    assert set(seen["rows"].tolist()) <= {4, 9}
