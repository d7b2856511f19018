"""GPU parity of the general sketch (Sec. 2.4: random sign sketch columns,
Corollary 2.2) against the CPU oracle, through the C ABI.

Both sides draw the same sketch columns (SplitMix64 outputs by index). The
oracle follows Theorem 2.1's update of N = (Y^T Y)^{-1}; the GPU keeps the
same projector as orthogonal directions. Tolerance: 1e-10 relative on x, or
the parity margin times the oracle's own rounding spread (the oracle run
again on b (1 + 2^-50)) where that is larger.
"""
import numpy as np
import pytest

import oracle
from paper_2207_07615_gb300 import synth
from tests import _parity

pytestmark = pytest.mark.gpu

F = 1.0 + 2.0 ** -50


@pytest.fixture(scope="module")
def plss():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2207_07615_gb300 import plss as P
    return P


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def oracle_with_bar(A, b, x0=None, **kw):
    r1 = oracle.general(A, b, x0=x0, **kw)
    r2 = oracle.general(A, b * F, x0=None if x0 is None else x0 * F, **kw)
    spread = rel(r2["x"] / F, r1["x"])
    return r1, max(_parity.FLOOR, _parity.MARGIN * spread)


@pytest.mark.parametrize("K", [0, 3, 64])
def test_parity_rectangular(plss, K):
    """An overdetermined and an underdetermined sparse system, a few steps
    and many (history emptied when full)."""
    for A, b in (synth.overdetermined_scaled(m=3000, n=400, per_row=6, seed=31, scale_decades=0.5)[:2],
                 synth.powerlaw_underdetermined(m=300, n=2000, mean_len=10, max_len=200, seed=32)[:2]):
        A = A.astype(np.float64)
        with plss.Context(A) as ctx:
            for maxit, seed in ((1, 5), (9, 5), (150, 6)):
                ref, bar = oracle_with_bar(A, b, tol=0.0, maxit=maxit, K=K, seed=seed)
                x, r = ctx.solve(b, sketch="general", kacz_hist=K, seed=seed, tol=0.0, maxit=maxit)
                assert r["iters"] == ref["iters"] == maxit
                assert rel(x, ref["x"]) <= bar, (K, maxit, rel(x, ref["x"]), bar)


def test_full_row_rank_reaches_pinv(plss):
    """A wide full-row-rank A: after m sketch columns (history kept) x = A^+ b
    (updates lie in range(A^T), Corollary 3.3), on the GPU as in the oracle."""
    rng = synth.rng_for(33)
    m, n = 120, 300
    D = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.05)
    D[np.arange(m), np.arange(m)] += 2.0
    A = synth.from_dense(D)
    b = D @ rng.standard_normal(n)
    ref, bar = oracle_with_bar(A, b, tol=0.0, maxit=m, K=m, seed=8)
    with plss.Context(A) as ctx:
        x, r = ctx.solve(b, sketch="general", kacz_hist=m, seed=8, tol=0.0, maxit=m)
    assert rel(x, ref["x"]) <= bar
    assert rel(x, np.linalg.pinv(D) @ b) < 1e-8


def test_tall_system_converges_in_n_columns(plss):
    """A consistent tall system with full column rank: with the history kept
    the method stops within n sketch columns (the oracle too) at x*."""
    A, b, xs = synth.overdetermined_scaled(m=2000, n=150, per_row=6, seed=34, scale_decades=0.3)
    A = A.astype(np.float64)
    ref = oracle.general(A, b, tol=1e-10, maxit=400, K=400, seed=3)
    with plss.Context(A) as ctx:
        x, r = ctx.solve(b, sketch="general", kacz_hist=400, seed=3, tol=1e-10, maxit=400)
    assert ref["status"] == "converged" and r["status"] == "converged"
    assert r["iters"] <= A.n + 2 and abs(r["iters"] - ref["iters"]) <= 2
    assert r["relres_true"] <= 1e-10
    assert rel(x, xs) < 1e-7


def test_fp32_storage(plss):
    """FP32 storage of A: the oracle on the same float-rounded values (the
    sketch algebra is in double on both sides)."""
    A, b, _ = synth.overdetermined_scaled(m=2500, n=300, per_row=6, seed=35, scale_decades=0.5)
    A32 = A.astype(np.float32)
    ref, bar = oracle_with_bar(A32.astype(np.float64), b, tol=0.0, maxit=60, K=20, seed=4)
    with plss.Context(A32, precision="fp32") as ctx:
        x, r = ctx.solve(b, sketch="general", kacz_hist=20, seed=4, tol=0.0, maxit=60)
    assert rel(x, ref["x"]) <= bar


def test_options_rejected(plss):
    A, b, _ = synth.overdetermined_scaled(m=300, n=50, per_row=4, seed=36)
    A = A.astype(np.float64)
    with plss.Context(A) as ctx:
        with pytest.raises(plss.PlssError):
            ctx.solve(b, sketch="general", kacz_hist=1025, tol=0.0, maxit=5)
        with pytest.raises(plss.PlssError):
            ctx.solve(b, sketch="general", w_mode=1, tol=0.0, maxit=5)


def test_zero_rhs_and_start_vector(plss):
    """b = 0 returns x0 at once (converged, no column drawn); a nonzero start
    vector follows the oracle."""
    A, b, _ = synth.overdetermined_scaled(m=2000, n=300, per_row=6, seed=37, scale_decades=0.5)
    A = A.astype(np.float64)
    x0 = synth.rng_for(5).standard_normal(A.n)
    with plss.Context(A) as ctx:
        x, r = ctx.solve(np.zeros(A.m), x0, sketch="general", kacz_hist=8, tol=1e-8, maxit=50)
        assert r["status"] == "converged" and r["iters"] == 0
        np.testing.assert_array_equal(x, x0)
        ref, bar = oracle_with_bar(A, b, x0=x0, tol=0.0, maxit=40, K=8, seed=6)
        x, r = ctx.solve(b, x0, sketch="general", kacz_hist=8, seed=6, tol=0.0, maxit=40)
    assert rel(x, ref["x"]) <= bar
