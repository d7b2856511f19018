"""Pins of the oracle's general sketch (Sec. 2.4: Theorem 2.1 and
Corollary 2.2, with random sign sketch columns).

References, none of them the oracle: the published first outputs of the
SplitMix64 stream, the sketch columns drawn again by an implementation of
SplitMix64 written here from its definition, eq:pkLong evaluated densely
with S_k = [s_1 ... s_k] (pseudo-inverse), finite termination at the
pseudo-inverse solution, and the orthogonality of Sec. 2.1.
"""
import numpy as np
import pytest

import oracle
from paper_2207_07615_gb300 import synth
from tests import _pins

M64 = (1 << 64) - 1


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def splitmix_out(seed, j):
    """Output j (0-based) of SplitMix64 seeded with `seed`, from its
    definition: the state after j + 1 additions of the golden gamma, mixed."""
    z = (seed + (j + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def sketch(seed, m, k):
    """Sketch column k: entry i is -1 where bit 63 of output k*m + i is set."""
    return np.array([-1.0 if splitmix_out(seed, k * m + i) >> 63 else 1.0 for i in range(m)])


def read_hex_golden(name):
    import os
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (t.strip() for t in line.split("="))
                out[k] = int(v, 16)
    return out


def test_splitmix_published_outputs():
    """The generator behind the sketch columns reproduces SplitMix64's
    published outputs, and the oracle's sketch entries are their sign bits."""
    g = read_hex_golden("splitmix64_seed0.txt")
    assert [splitmix_out(0, j) for j in range(3)] == [g["out0"], g["out1"], g["out2"]]
    got = [oracle.sketch_entry(0, 3, 0, i) for i in range(3)]
    assert got == [-1.0, 1.0, 1.0]          # bit 63 of out0 set, of out1 and out2 clear
    for seed, m, k in ((5, 7, 0), (5, 7, 3), (2**63 + 11, 40, 9)):
        np.testing.assert_array_equal([oracle.sketch_entry(seed, m, k, i) for i in range(m)],
                                      sketch(seed, m, k))


def _dense_reference(D, b, seed, steps, K=None):
    """eq:pkLong with S_k = the sketch columns of the current history
    (all columns so far, or the last window of K), x0 = 0."""
    m, n = D.shape
    x = np.zeros(n)
    cols, xs = [], []
    for k in range(steps):
        if K and len(cols) == K:
            cols = []
        s = sketch(seed, m, k)
        cols.append(s)
        S = np.stack(cols, axis=1)
        r = b - D @ x
        x = x + _pins.pk_long(D, np.ones(n), S, r)
        xs.append(x.copy())
    return xs


def _cases():
    rng = synth.rng_for(71)
    out = []
    for (m, n, rank) in [(6, 6, 6), (9, 5, 5), (5, 9, 5), (8, 8, 5)]:
        D = synth.dense_rank_deficient(rng, m, n, rank)
        out.append((D, D @ rng.standard_normal(n), rank))
    return out


CASES = _cases()


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_general_equals_pklong(ci):
    """Theorem 2.1 / Corollary 2.2 reproduce eq:pkLong with S_k = [s_1 ... s_k]
    for every k up to rank(A)."""
    D, b, rank = CASES[ci]
    A = synth.from_dense(D)
    seed = 1000 + ci
    out = oracle.general(A, b, tol=0.0, maxit=rank, K=64, seed=seed, hist=rank)
    ref = _dense_reference(D, b, seed, rank)
    for k in range(rank):
        assert rel(out["hist_x"][k], ref[k]) < 1e-9, k


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_general_terminates_at_the_limit(ci):
    """After rank(A) full-rank sketch columns the iterate is the limit
    x0 + A^T (A A^T)^+ (b - A x0) (updates lie in range(A^T), Corollary 3.3);
    further columns add nothing (delta at rounding level: skipped)."""
    D, b, rank = CASES[ci]
    A = synth.from_dense(D)
    out = oracle.general(A, b, tol=0.0, maxit=rank + 3, K=64, seed=2000 + ci)
    assert rel(out["x"], _pins.limit_solution(D, b, np.zeros(D.shape[1]))) < 1e-9
    assert out["relres_true"] < 1e-10
    assert out["skipped"] >= 1


def test_general_orthogonality():
    """Sec. 2.1: previous sketch columns are orthogonal to the next residual
    (s_j^T r_k = 0, j <= k), and the updates are mutually orthogonal."""
    D, b, rank = CASES[1]
    A = synth.from_dense(D)
    seed = 3001
    out = oracle.general(A, b, tol=0.0, maxit=rank - 1, K=64, seed=seed, hist=rank - 1)
    X = np.vstack([np.zeros(D.shape[1]), out["hist_x"]])
    P = np.diff(X, axis=0)
    G = P @ P.T
    sc = np.sqrt(np.outer(np.diag(G), np.diag(G)))
    off = ~np.eye(len(P), dtype=bool)
    assert np.max(np.abs(G[off]) / sc[off]) < 1e-9
    for k in range(1, len(X)):
        r = b - D @ X[k]
        for j in range(k):
            s = sketch(seed, D.shape[0], j)
            assert abs(s @ r) <= 1e-9 * np.linalg.norm(s) * np.linalg.norm(b)


def test_general_window():
    """A history of at most K = 3 columns, emptied when full: every step
    equals eq:pkLong with S = the current window's columns."""
    rng = synth.rng_for(72)
    D = rng.standard_normal((14, 10))
    b = D @ rng.standard_normal(10)
    A = synth.from_dense(D)
    out = oracle.general(A, b, tol=0.0, maxit=9, K=3, seed=77, hist=9)
    ref = _dense_reference(D, b, 77, 9, K=3)
    for k in range(9):
        assert rel(out["hist_x"][k], ref[k]) < 1e-9, k


def test_planted_N_update_is_caught():
    """Leaving the rank-one term t t^T / delta out of eq:Nkrec breaks the
    agreement with eq:pkLong from the third column on."""
    D, b, rank = CASES[0]
    A = synth.from_dense(D)
    bad = oracle.general(A, b, tol=0.0, maxit=rank, K=64, seed=1000, hist=rank, plant=1)
    ref = _dense_reference(D, b, 1000, rank)
    assert max(rel(bad["hist_x"][k], ref[k]) for k in range(rank)) > 1e-3
