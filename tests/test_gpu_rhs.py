"""GPU parity of the many-right-hand-side form (SpMM sweeps): every column
of a block solve follows the oracle's single-right-hand-side run of
Algorithm 1 on that column (calibrated bar of tests/_parity.py) and stops on
its own."""
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def test_laplacian_block_matches_columns(plss):
    """7-point Laplacian (symmetric: A^T r reuses the CSR), 5 right-hand sides."""
    A = synth.laplacian7(12, dtype=np.float64)
    B, Xs = synth.laplacian_rhs(A, nrhs=5, seed0=2000)
    K = 30
    with plss.Context(A, symmetric=True) as ctx:
        X, rs = ctx.solve_rhs(B, tol=0.0, maxit=K, hist=K)
        for j in range(5):
            ref = _parity.reference(A, B[:, j].copy(), K)
            assert rs[j]["iters"] == K
            _parity.check_x(X[:, j], ref, K)
        X, rs = ctx.solve_rhs(B, tol=1e-10, maxit=5000)
    for j in range(5):
        fin = oracle.residual(A, B[:, j].copy(), tol=1e-10, maxit=5000)
        assert rs[j]["status"] == "converged" and rs[j]["relres_true"] <= 2e-10
        assert abs(rs[j]["iters"] - fin["iters"]) <= 2
        assert rel(X[:, j], Xs[:, j]) < 1e-8


def test_nonsymmetric_block_with_x0_and_hist(plss):
    A, _, _ = synth.overdetermined_scaled(m=6000, n=1500, per_row=8, seed=31, scale_decades=0.5)
    A = A.astype(np.float64)
    rng = synth.rng_for(5)
    Xs = rng.standard_normal((A.n, 3))
    B = np.ascontiguousarray(A.scipy() @ Xs)
    X0 = np.ascontiguousarray(rng.standard_normal((A.n, 3)))
    K = 40
    with plss.Context(A) as ctx:
        X, rs = ctx.solve_rhs(B, X0, tol=0.0, maxit=K, hist=K)
    for j in range(3):
        ref = _parity.reference(A, B[:, j].copy(), K, x0=X0[:, j].copy())
        _parity.check_x(X[:, j], ref, K)


def test_columns_stop_independently_fp32(plss):
    """FP32 storage with FP64 refinement; one column starts at its solution."""
    A = synth.laplacian7(10, dtype=np.float32)
    B, Xs = synth.laplacian_rhs(A, nrhs=4, seed0=7)
    X0 = np.zeros_like(Xs)
    X0[:, 2] = Xs[:, 2]
    with plss.Context(A, precision="fp32", symmetric=True) as ctx:
        X, rs = ctx.solve_rhs(B, np.ascontiguousarray(X0), tol=1e-8, maxit=5000)
    assert rs[2]["iters"] == 0
    for j in range(4):
        assert rs[j]["status"] == "converged" and rs[j]["relres_true"] <= 1e-8
        assert rel(X[:, j], Xs[:, j]) < 1e-6
