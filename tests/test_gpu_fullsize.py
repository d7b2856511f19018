"""Parity at the benchmark sizes, in the configuration bench.py times
(default layout and schedule): the leading updates of each workload against
the oracle, sampled where the oracle would be too slow in full.

* C2, 1,000,000 x 200,000 (the headline): the first 12 updates' scalars and
  x_12 in FP64 (calibrated bar, at least 8 updates at the plain 1e-10), and
  the first updates of FP32 storage against the oracle's FP32 emulation.
* C3, 100,000 x 1,000,000 power-law rows: 10 updates of the residual sketch,
  3,000 rows of the identity sketch (K = 0 and K = 8) and 120 rows with a
  window of 256 (the whole-GPU form).
* The general sketch on C2: the first 8 sketch columns, history 64.
* C4b, the 126^3 Laplacian with 32 right-hand sides (SpMM sweeps): 6
  updates, columns 0 and 31 against single-right-hand-side oracle solves.
* C4a-shaped batch: the first 24 of the 256 systems (seeds 1000..1023) in one
  batched context, 10 updates each against the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2207_07615_gb300 import synth
from tests import _parity

pytestmark = pytest.mark.gpu


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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def c2():
    A, b, xs = synth.overdetermined_scaled()
    return A, b


def test_c2_fp64_first_updates(plss, c2):
    A, b = c2
    A64 = A.astype(np.float64)
    K = 12
    ref = _parity.reference(A64, b, K)
    with plss.Context(A64) as ctx:
        lay = ctx.layout()
        assert lay["row_sliced"] == lay["row_tiles"] and lay["col_sliced"] == lay["col_tiles"]
        x, res, hist = ctx.solve(b, tol=0.0, maxit=K, hist=K)
    assert res["iters"] == K
    _parity.check_scalars(hist, ref, min_strict=8)
    _parity.check_x(x, ref, K)


def test_c2_fp32_first_updates(plss, c2):
    A, b = c2
    K = 6
    emu = oracle.residual(A, b, tol=0.0, maxit=K, prec=1, stop_on_true=True, hist=K)
    with plss.Context(A, precision="fp32") as ctx:
        x, res, hist = ctx.solve(b, tol=0.0, maxit=K, hist=K)
    assert _parity.rel_rows(hist[:K], emu["hist_s"][:K]).max() < 1e-4
    assert rel(x, emu["x"]) < 1e-4


@pytest.fixture(scope="module")
def c3():
    A, b, xs = synth.powerlaw_underdetermined()
    return A.astype(np.float64), b


def test_c3_residual_first_updates(plss, c3):
    A, b = c3
    K = 10
    ref = _parity.reference(A, b, K)
    with plss.Context(A) as ctx:
        x, res, hist = ctx.solve(b, tol=0.0, maxit=K, hist=K)
    _parity.check_scalars(hist, ref, min_strict=6)
    _parity.check_x(x, ref, K)


@pytest.mark.parametrize("K,rows", [(0, 3000), (8, 3000), (256, 120)])
def test_c3_identity_rows(plss, c3, K, rows):
    A, b = c3
    seed = 11
    r1 = oracle.kaczmarz(A, b, tol=0.0, maxit=rows, K=K, seed=seed)
    r2 = oracle.kaczmarz(A, b * _parity.F, tol=0.0, maxit=rows, K=K, seed=seed)
    bar = max(_parity.FLOOR, _parity.MARGIN * rel(r2["x"] / _parity.F, r1["x"]))
    with plss.Context(A) as ctx:
        x, res = ctx.solve(b, sketch="identity", kacz_hist=K, seed=seed, tol=0.0, maxit=rows)
    assert res["iters"] == rows
    assert rel(x, r1["x"]) <= bar


def test_c4b_spmm_sampled_columns(plss):
    A = synth.laplacian7(dtype=np.float64)
    B, Xs = synth.laplacian_rhs(A)
    K = 6
    with plss.Context(A, symmetric=True) as ctx:
        X, rs = ctx.solve_rhs(B, tol=0.0, maxit=K)
    assert all(r["iters"] == K for r in rs)
    for j in (0, 31):
        ref = _parity.reference(A, B[:, j].copy(), K)
        _parity.check_x(X[:, j], ref, K)


def test_c4a_batched_first_systems(plss):
    systems = synth.batched_systems(nsys=24)
    As = [A.astype(np.float64) for A, _, _ in systems]
    bs = [b for _, b, _ in systems]
    K = 10
    with plss.Context(As) as ctx:
        xs, rs = ctx.solve_batched(bs, tol=0.0, maxit=K, w_mode=2)
    for A, b, x, r in zip(As, bs, xs, rs):
        assert r["iters"] == K
        ref = _parity.reference(A, b, K, w=oracle.colweights(A, 2))
        _parity.check_x(x, ref, K)


def test_c2_general_first_columns(plss, c2):
    """The general sketch (Sec. 2.4) on the headline system: 8 random sign
    columns with a history of 64, against the oracle's Theorem 2.1."""
    A, b = c2
    A64 = A.astype(np.float64)
    cols, seed = 8, 21
    r1 = oracle.general(A64, b, tol=0.0, maxit=cols, K=64, seed=seed)
    r2 = oracle.general(A64, b * _parity.F, tol=0.0, maxit=cols, K=64, seed=seed)
    bar = max(_parity.FLOOR, _parity.MARGIN * rel(r2["x"] / _parity.F, r1["x"]))
    with plss.Context(A64) as ctx:
        x, res = ctx.solve(b, sketch="general", kacz_hist=64, seed=seed, tol=0.0, maxit=cols)
    assert res["iters"] == cols
    assert rel(x, r1["x"]) <= bar
