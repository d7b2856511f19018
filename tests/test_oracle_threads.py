"""The OpenMP build of the oracle (the all-cores CPU baseline of the
benchmark) runs the same method as the plain build: the same source with
its row, column and vector loops split over the host cores, so only the
order of the partial sums of rho, phi and theta changes. Checked on the
CPU against the plain build's scalars, update by update, and against x*
of a nonsingular system (Theorem 3.1: the limit is the unique solution)."""
import numpy as np
import pytest

import oracle
from paper_2207_07615_gb300 import synth
from tests import _parity


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()
    try:
        oracle._load_omp()
    except RuntimeError as e:   # gcc without OpenMP support
        pytest.skip(str(e))


def test_threaded_build_follows_the_plain_one():
    """Update by update, within the bar the GPU parity tests use: 1e-10
    while the recursion is at rounding level, then the plain build's own
    rounding sensitivity (its run on b (1 + 2^-50)) times the margin. Like
    every Lanczos-type recursion, reordered sums drift apart once the
    residuals lose orthogonality: after 40 updates x differs in the fifth
    digit while the scalars still agree to 1e-11. (OpenMP combines the
    threads' partial sums in the order they finish, so the threaded
    trajectory itself varies a little from run to run.)"""
    A, b, xs = synth.overdetermined_scaled(m=20000, n=4000, per_row=8, seed=11, scale_decades=1.0)
    A = A.astype(np.float64)
    H = 40
    ref = _parity.reference(A, b, H)
    many = oracle.residual(A, b, tol=0.0, maxit=H, hist=H, threads=True)
    assert many["iters"] == ref["iters"] == H
    assert _parity.check_scalars(many["hist_s"], ref) >= 10
    for k in range(1, H + 1):
        _parity.check_x(many["hist_x"][k - 1], ref, k)


def test_threaded_build_solves_the_square_system():
    A, b, xs = synth.square_diag_dominant()
    out = oracle.residual(A, b, tol=1e-10, maxit=2000, threads=True)
    assert out["status"] == "converged" and out["relres_true"] < 2e-10
    assert np.linalg.norm(out["x"] - xs) / np.linalg.norm(xs) < 1e-8
