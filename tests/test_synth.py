"""The seeded synthetic inputs match the recipes they stand for (the shapes,
value distributions and structure of the paper's large sparse experiments),
checked on the CPU: row lengths, distinct sorted columns, value ranges and
rounding, exact consistency of b, symmetry of the Laplacian, the request
trace's statistics, and determinism per seed."""
import math

import numpy as np

from paper_2207_07615_gb300 import synth


def _rows(A):
    rp = np.asarray(A.row_ptr)
    ci = np.asarray(A.col_idx)
    return rp, ci


def _distinct_sorted(A):
    rp, ci = _rows(A)
    d = np.diff(ci.astype(np.int64))
    row_start = np.zeros(len(ci), dtype=bool)
    row_start[rp[:-1][np.diff(rp) > 0]] = True
    # within a row every step is strictly increasing
    assert np.all(d[~row_start[1:]] > 0)
    assert ci.min(initial=0) >= 0 and ci.max(initial=-1) < A.n


def test_square_diag_dominant_recipe():
    """C1: n x n, `per_row` distinct off-diagonal columns, diagonal 1 + abs
    row sum of the off-diagonals (strictly dominant), b = A x*."""
    A, b, xs = synth.square_diag_dominant(n=300, per_row=10, seed=0)
    assert (A.m, A.n, A.nnz) == (300, 300, 300 * 11)
    _distinct_sorted(A)
    D = A.to_dense()
    off = D - np.diag(np.diag(D))
    assert np.all((off != 0).sum(axis=1) == 10)
    np.testing.assert_allclose(np.diag(D), 1.0 + np.abs(off).sum(axis=1), rtol=1e-15)
    np.testing.assert_allclose(D @ xs, b, rtol=1e-12, atol=1e-12)


def test_overdetermined_scaled_recipe():
    """C2 (reduced): 8 distinct uniform columns a row, values z c_j with
    column scales 10^U(-2, 2), rounded to FP32 once, b = A x* in FP64 from
    the rounded values (the FP32 system is exactly consistent)."""
    m, n = 20000, 4000
    A, b, xs = synth.overdetermined_scaled(m=m, n=n, per_row=8, seed=1)
    assert (A.m, A.n, A.nnz) == (m, n, 8 * m)
    assert np.asarray(A.val).dtype == np.float32
    _distinct_sorted(A)
    assert np.all(np.diff(np.asarray(A.row_ptr)) == 8)
    # column scales: per column, |values| / |z| spans 10^-2 .. 10^2; the
    # largest magnitude in a column is at most a few sigma times 100
    v = np.abs(np.asarray(A.val, dtype=np.float64))
    assert v.max() < 100 * 8 and v[v > 0].min() < 1e-2
    # exactly consistent in FP64 from the FP32 values
    Ad = A.astype(np.float64).scipy()
    np.testing.assert_allclose(Ad @ xs, b, rtol=1e-13, atol=1e-13)
    # columns drawn uniformly: every column count is near the mean (8m/n = 40)
    counts = np.bincount(np.asarray(A.col_idx), minlength=n)
    assert abs(counts.mean() - 40.0) < 1e-9 and counts.std() < 10


def test_powerlaw_rows_recipe():
    """C3 (reduced): truncated Zipf row lengths on [1, max_len] with mean
    20, distinct columns, U(-1, 1) values rounded to FP32."""
    s = synth.zipf_exponent(20.0, 5000)
    assert 1.6 < s < 1.8                                  # s ~ 1.70 for mean 20 on [1, 5000]
    l = np.arange(1, 5001, dtype=np.float64)
    w = l ** -s
    assert abs((l * w).sum() / w.sum() - 20.0) < 1e-6
    A, b, xs = synth.powerlaw_underdetermined(m=20000, n=200000, mean_len=20.0, max_len=5000, seed=2)
    lengths = np.diff(np.asarray(A.row_ptr))
    assert lengths.min() >= 1 and lengths.max() <= 5000
    assert abs(lengths.mean() - 20.0) < 3.0               # heavy tail: the sample mean moves
    assert np.median(lengths) <= 5                        # most rows are short
    _distinct_sorted(A)
    v = np.asarray(A.val)
    assert v.dtype == np.float32 and np.all(np.abs(v) <= 1.0)


def test_batched_systems_recipe():
    """C4a (a few systems): m log-uniform in [1e3, 2e5], n = m or m // 2,
    row lengths U{5..50} capped at n, FP32 values, b = A x*."""
    out = synth.batched_systems(nsys=6, seed0=1000)
    assert len(out) == 6
    for A, b, xs in out:
        assert 1000 <= A.m <= 200000 and A.n in (A.m, max(1, A.m // 2))
        lengths = np.diff(np.asarray(A.row_ptr))
        assert lengths.min() >= min(5, A.n) and lengths.max() <= min(50, A.n)
        assert np.asarray(A.val).dtype == np.float32
        _distinct_sorted(A)
        np.testing.assert_allclose(A.astype(np.float64).scipy() @ xs, b, rtol=1e-12, atol=1e-10)


def test_laplacian_recipe():
    """C4b (N = 6 instead of 126): 7-point stencil, Dirichlet, diagonal 6,
    neighbours -1, nnz = 7 N^3 - 6 N^2, symmetric."""
    N = 6
    A = synth.laplacian7(N)
    assert A.m == A.n == N ** 3 and A.nnz == 7 * N ** 3 - 6 * N ** 2
    D = A.to_dense()
    np.testing.assert_array_equal(D, D.T)
    assert np.all(np.diag(D) == 6.0)
    off = D - np.diag(np.diag(D))
    assert set(np.unique(off)) <= {0.0, -1.0}
    assert synth.laplacian7(126, dtype=np.float32).nnz == 13_907_376   # the configuration's count
    B, X = synth.laplacian_rhs(A, nrhs=4, seed0=2000)
    np.testing.assert_allclose(D @ X, B, rtol=1e-12, atol=1e-12)


def test_serving_trace_recipe():
    """C5: Poisson arrivals at the given rate (exponential gaps), pool ids
    uniform, pool matrices with m log-uniform in [1e3, 1e6], aspect n/m in
    {0.5, 1, 2}, row lengths U{8..32}."""
    arr, ids, mats = synth.serving_trace(nreq=20000, rate=2000.0, pool=8, m_lo=1e3, m_hi=2e4, seed=3000)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - 1.0 / 2000.0) < 0.05 / 2000.0
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05       # exponential: cv = 1
    assert ids.min() >= 0 and ids.max() < 8
    for A in mats:
        assert 1000 <= A.m <= 20000
        assert any(abs(A.n - A.m * a) <= 1 for a in (0.5, 1.0, 2.0))
        lengths = np.diff(np.asarray(A.row_ptr))
        assert lengths.min() >= min(8, A.n) and lengths.max() <= 32
        _distinct_sorted(A)


def test_generators_are_deterministic_per_seed():
    a = synth.overdetermined_scaled(m=2000, n=400, seed=5)
    b = synth.overdetermined_scaled(m=2000, n=400, seed=5)
    c = synth.overdetermined_scaled(m=2000, n=400, seed=6)
    np.testing.assert_array_equal(np.asarray(a[0].col_idx), np.asarray(b[0].col_idx))
    np.testing.assert_array_equal(np.asarray(a[0].val), np.asarray(b[0].val))
    np.testing.assert_array_equal(a[1], b[1])
    assert not np.array_equal(np.asarray(a[0].col_idx), np.asarray(c[0].col_idx))
    assert math.isclose(float(np.linalg.norm(a[2])), float(np.linalg.norm(b[2])))
