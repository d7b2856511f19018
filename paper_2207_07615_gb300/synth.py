"""Seeded synthetic inputs for PLSS (consistent sparse systems A x = b).

This module builds inputs only: sparse matrices in CSR form, exact solutions
x*, right-hand sides b = A x*, request traces. It holds none of the solver's
arithmetic, so both the CUDA path and the CPU oracle may take their inputs
from here.

The paper measures on SuiteSparse / LIBSVM matrices (Sec. 8, Experiments
I-V), which are not available; these generators stand in for them with the
shapes of the paper's large sparse experiments (Experiment III runs to 1e6-1e7
rows at densities 1e-5..1e-6). Every generator draws from
numpy.random.Generator(PCG64(seed)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CSR", "rng_for", "distinct_columns", "from_dense", "rhs",
    "square_diag_dominant", "overdetermined_scaled", "powerlaw_underdetermined",
    "batched_systems", "laplacian7", "laplacian_rhs", "serving_trace",
    "zipf_exponent", "dense_rank_deficient",
]


@dataclasses.dataclass
class CSR:
    """Compressed sparse row matrix: row_ptr int64[m+1], col_idx int32[nnz]
    (sorted and distinct within each row), val float64 or float32 [nnz]."""
    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def astype(self, dtype) -> "CSR":
        return CSR(self.m, self.n, self.row_ptr, self.col_idx, self.val.astype(dtype))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.m, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        d[rows, self.col_idx] = self.val
        return d

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val.astype(np.float64), self.col_idx, self.row_ptr),
                             shape=(self.m, self.n))


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def distinct_columns(rng: np.random.Generator, lengths: np.ndarray, n: int,
                     exclude_diag: bool = False) -> np.ndarray:
    """Uniform random column indices, distinct within each row, sorted per row.

    lengths[i] columns are drawn for row i (lengths must be <= n, or <= n-1
    when the diagonal is excluded). Duplicates are redrawn until none remain.
    """
    lengths = np.asarray(lengths, dtype=np.int64)
    m = lengths.shape[0]
    total = int(lengths.sum())
    row = np.repeat(np.arange(m, dtype=np.int64), lengths)
    span = n - 1 if exclude_diag else n

    def draw(k, rows):
        c = rng.integers(0, span, size=k, dtype=np.int64)
        if exclude_diag:
            c = c + (c >= rows)
        return c

    col = draw(total, row)
    while True:
        key = row * n + col
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(total, dtype=bool)
        dup[order[1:]] = ks[1:] == ks[:-1]
        nd = int(dup.sum())
        if nd == 0:
            break
        col[dup] = draw(nd, row[dup])
    key = row * n + col
    order = np.argsort(key, kind="stable")
    return col[order].astype(np.int32)


def _ptr(lengths: np.ndarray) -> np.ndarray:
    p = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=p[1:])
    return p


def from_dense(d: np.ndarray) -> CSR:
    d = np.asarray(d, dtype=np.float64)
    m, n = d.shape
    mask = d != 0
    lengths = mask.sum(axis=1)
    rows, cols = np.nonzero(mask)
    return CSR(m, n, _ptr(lengths), cols.astype(np.int32), d[rows, cols].copy())


def rhs(A: CSR, xstar: np.ndarray) -> np.ndarray:
    """b = A x* in FP64 (A's stored values promoted to FP64)."""
    return np.asarray(A.scipy() @ np.asarray(xstar, dtype=np.float64), dtype=np.float64)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def square_diag_dominant(n: int = 2000, per_row: int = 10, seed: int = 0):
    """Square n x n system: per row `per_row` distinct uniform off-diagonal
    columns with N(0,1) values, diagonal 1 + (row abs-sum of off-diagonals).
    x* ~ N(0,1), b = A x*, FP64. Returns (A, b, x*)."""
    rng = rng_for(seed)
    lengths = np.full(n, per_row, dtype=np.int64)
    cols = distinct_columns(rng, lengths, n, exclude_diag=True)
    offv = rng.standard_normal(n * per_row)
    rows = np.repeat(np.arange(n), per_row)
    diag = 1.0 + np.bincount(rows, weights=np.abs(offv), minlength=n)
    # merge the diagonal into each sorted row
    all_rows = np.concatenate([rows, np.arange(n)])
    all_cols = np.concatenate([cols.astype(np.int64), np.arange(n)])
    all_vals = np.concatenate([offv, diag])
    order = np.lexsort((all_cols, all_rows))
    A = CSR(n, n, _ptr(lengths + 1), all_cols[order].astype(np.int32), all_vals[order])
    xstar = rng.standard_normal(n)
    return A, rhs(A, xstar), xstar


def overdetermined_scaled(m: int = 1_000_000, n: int = 200_000, per_row: int = 8,
                          seed: int = 1, scale_decades: float = 2.0):
    """Overdetermined consistent system: per row `per_row` distinct uniform
    columns, A_ij = z * c_j with z ~ N(0,1) and column scales
    c_j = 10**U(-scale_decades, scale_decades). Values are rounded to FP32 once;
    the returned A carries float32 values and b = A x* is formed in FP64 from
    those rounded values, so the FP32 system is exactly consistent.
    Returns (A[f32 values], b, x*)."""
    rng = rng_for(seed)
    lengths = np.full(m, per_row, dtype=np.int64)
    cols = distinct_columns(rng, lengths, n)
    c = 10.0 ** rng.uniform(-scale_decades, scale_decades, size=n)
    z = rng.standard_normal(m * per_row)
    val = (z * c[cols]).astype(np.float32)
    A = CSR(m, n, _ptr(lengths), cols, val)
    xstar = rng.standard_normal(n)
    return A, rhs(A, xstar), xstar


def zipf_exponent(mean: float = 20.0, lmax: int = 5000) -> float:
    """Exponent s of P(L = l) proportional to l**-s on [1, lmax] with the given mean."""
    l = np.arange(1, lmax + 1, dtype=np.float64)
    lo, hi = 0.5, 4.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        w = l ** (-mid)
        if (l * w).sum() / w.sum() > mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def powerlaw_underdetermined(m: int = 100_000, n: int = 1_000_000, mean_len: float = 20.0,
                             max_len: int = 5000, seed: int = 2):
    """Underdetermined system with power-law row lengths (truncated Zipf on
    [1, max_len] with the given mean), distinct uniform columns, values
    U(-1,1) rounded to FP32. Returns (A[f32 values], b, x*)."""
    rng = rng_for(seed)
    max_len = min(max_len, n)
    s = zipf_exponent(mean_len, max_len)
    l = np.arange(1, max_len + 1, dtype=np.float64)
    pr = l ** (-s)
    pr /= pr.sum()
    lengths = rng.choice(np.arange(1, max_len + 1), size=m, p=pr).astype(np.int64)
    cols = distinct_columns(rng, lengths, n)
    val = rng.uniform(-1.0, 1.0, size=int(lengths.sum())).astype(np.float32)
    A = CSR(m, n, _ptr(lengths), cols, val)
    xstar = rng.standard_normal(n)
    return A, rhs(A, xstar), xstar


def batched_systems(nsys: int = 256, m_lo: float = 1e3, m_hi: float = 2e5,
                    len_lo: int = 5, len_hi: int = 50, seed0: int = 1000):
    """Independent systems of uneven size. System s (seed seed0+s):
    m = round(exp U(ln m_lo, ln m_hi)), n = m or m//2 by a fair coin, row
    lengths U{len_lo..len_hi} capped at n, values N(0,1) rounded to FP32,
    b = A x*. Returns a list of (A, b, x*)."""
    out = []
    for s in range(nsys):
        rng = rng_for(seed0 + s)
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        n = m if rng.integers(0, 2) == 0 else max(1, m // 2)
        lengths = np.minimum(rng.integers(len_lo, len_hi + 1, size=m), n).astype(np.int64)
        cols = distinct_columns(rng, lengths, n)
        val = rng.standard_normal(int(lengths.sum())).astype(np.float32)
        A = CSR(m, n, _ptr(lengths), cols, val)
        xstar = rng.standard_normal(n)
        out.append((A, rhs(A, xstar), xstar))
    return out


def laplacian7(N: int = 126, dtype=np.float32) -> CSR:
    """7-point 3-D Laplacian on an N^3 grid, Dirichlet boundary (no wrap):
    diagonal 6, neighbours -1. Symmetric positive definite."""
    nn = N * N * N
    idx = np.arange(nn, dtype=np.int64)
    i = idx // (N * N)
    j = (idx // N) % N
    k = idx % N
    cols = []
    vals = []
    # neighbours in ascending column order: -N^2, -N, -1, 0, +1, +N, +N^2
    for off, ok in ((-N * N, i > 0), (-N, j > 0), (-1, k > 0), (0, None),
                    (1, k < N - 1), (N, j < N - 1), (N * N, i < N - 1)):
        c = idx + off
        if ok is None:
            cols.append(c)
            vals.append(np.full(nn, 6.0))
        else:
            cols.append(np.where(ok, c, -1))
            vals.append(np.where(ok, -1.0, 0.0))
    C = np.stack(cols, axis=1)
    V = np.stack(vals, axis=1)
    mask = C >= 0
    lengths = mask.sum(axis=1)
    return CSR(nn, nn, _ptr(lengths), C[mask].astype(np.int32), V[mask].astype(dtype))


def laplacian_rhs(A: CSR, nrhs: int = 32, seed0: int = 2000):
    """Right-hand sides b_j = A x*_j with x*_j ~ N(0,1) from seed seed0+j.
    Returns (B, X*) as (m x nrhs) and (n x nrhs) row-major FP64 arrays."""
    Xs = np.stack([rng_for(seed0 + j).standard_normal(A.n) for j in range(nrhs)], axis=1)
    B = np.asarray(A.scipy() @ Xs, dtype=np.float64)
    return np.ascontiguousarray(B), np.ascontiguousarray(Xs)


def serving_trace(nreq: int = 10_000, rate: float = 2000.0, pool: int = 256,
                  m_lo: float = 1e3, m_hi: float = 1e6, len_lo: int = 8, len_hi: int = 32,
                  seed: int = 3000, build_pool: bool = True):
    """Open-loop Poisson request trace. Returns (arrivals[s], pool_ids, pool)
    where pool is a list of matrices (A, n) with m log-uniform in [m_lo, m_hi],
    aspect n/m in {0.5, 1, 2}, row lengths U{len_lo..len_hi}, values N(0,1)
    rounded to FP32. Each request draws a pool matrix; its x* comes from
    seed + 1_000_000 + request id."""
    rng = rng_for(seed)
    gaps = rng.exponential(1.0 / rate, size=nreq)
    arrivals = np.cumsum(gaps)
    pool_ids = rng.integers(0, pool, size=nreq)
    mats = []
    if build_pool:
        for p in range(pool):
            r = rng_for(seed + 1 + p)
            m = int(round(math.exp(r.uniform(math.log(m_lo), math.log(m_hi)))))
            aspect = (0.5, 1.0, 2.0)[int(r.integers(0, 3))]
            n = max(1, int(round(m * aspect)))
            lengths = np.minimum(r.integers(len_lo, len_hi + 1, size=m), n).astype(np.int64)
            cols = distinct_columns(r, lengths, n)
            val = r.standard_normal(int(lengths.sum())).astype(np.float32)
            mats.append(CSR(m, n, _ptr(lengths), cols, val))
    return arrivals, pool_ids, mats


def dense_rank_deficient(rng: np.random.Generator, m: int, n: int, rank: int) -> np.ndarray:
    """Dense m x n matrix of the given rank with O(1) singular values
    (for small exact-arithmetic-like checks)."""
    U, _ = np.linalg.qr(rng.standard_normal((m, rank)))
    V, _ = np.linalg.qr(rng.standard_normal((n, rank)))
    s = rng.uniform(1.0, 3.0, size=rank)
    return (U * s) @ V.T
