"""Pins of the oracle's restart schedules: the identity sketch's history
window (Sec. 7, eq:pkKacz) and the residual sketch's refinement restarts
(the FP32-storage extension, which the paper does not have).

The references are independent of the oracle: exact rational projections
onto the window's hyperplanes (eq:pkLong with identity columns), a 3x3 case
worked by hand, and eq:pkLong evaluated densely with a residual sketch that
starts afresh where the restart rule, applied to the dense run's own
residuals, says so. Each pin is also run against a planted defect in the
oracle (a wrong window reset, a wrong restart threshold) and must reject it.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2207_07615_gb300 import synth
from tests import _pins


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _seed_for_order(order):
    m = len(order)
    for seed in range(5000):
        perm, _ = oracle.permutation(seed, m)
        if tuple(perm) == tuple(order):
            return seed
    raise AssertionError("no seed gives that order")


# ------------------------------------------------- identity-sketch window

@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_window_3x3_worked_by_hand(K):
    """eq:pkKacz with a window of K directions on the 3x3 case worked by
    hand (tests/golden/kaczmarz_window_3x3_hand.txt)."""
    g = _pins.load_golden("kaczmarz_window_3x3_hand.txt")
    A = synth.from_dense(g["A"])
    seed = _seed_for_order((0, 1, 2))
    tag = {0: "k0", 1: "k0", 2: "k2", 3: "k3"}[K]
    xs = [g["x1"], g[tag + "_x2"] if tag != "k0" else g["k0_x2"], g[tag + "_x3"]]
    for k in (1, 2, 3):
        out = oracle.kaczmarz(A, g["b"], tol=0.0, maxit=k, K=K, seed=seed)
        assert out["skipped"] == 0
        np.testing.assert_allclose(out["x"], xs[k - 1], rtol=1e-14, atol=1e-15)


def _window_case(K, m=10, n=16, passes=2):
    """A random integer m x n matrix (full row rank) and two row passes whose
    windows of K rows never hold a row twice (so no row is dependent on its
    window); returns (D, b, seed, order)."""
    rng = np.random.default_rng(40 + K)
    D = rng.integers(-3, 4, size=(m, n)).astype(np.float64)
    D[np.arange(m), np.arange(m)] += 5.0
    xs = rng.integers(-4, 5, size=n).astype(np.float64)
    b = D @ xs
    for seed in range(1, 5000):
        st, order = seed, []
        for _ in range(passes):
            perm, st = oracle.permutation(st, m)
            order.extend(int(i) for i in perm)
        if K == 0:
            return D, b, seed, order
        wins = [order[i:i + K] for i in range(0, len(order), K)]
        if all(len(set(w)) == len(w) for w in wins):
            return D, b, seed, order
    raise AssertionError("no suitable seed")


@pytest.mark.parametrize("K", [1, 2, 3, 4, 7])
def test_window_equals_exact_projection(K):
    """Every step of the windowed identity sketch, over two passes (windows
    that straddle the passes' boundary included), equals the exact
    projection of x onto the hyperplanes of the current window's rows --
    eq:pkLong with S = the identity columns of the window only."""
    D, b, seed, order = _window_case(K)
    A = synth.from_dense(D)
    ref = _pins.window_projection_exact(D.astype(np.int64), b.astype(np.int64), order, K)
    for k in range(1, len(order) + 1):
        out = oracle.kaczmarz(A, b, tol=0.0, maxit=k, K=K, seed=seed)
        assert out["skipped"] == 0
        xr = np.array([float(v) for v in ref[k - 1]])
        assert rel(out["x"], xr) < 1e-12, (K, k)


@pytest.mark.parametrize("plant", [1, 2, 3])
def test_planted_window_reset_is_caught(plant):
    """A window emptied one row late, one row early or never breaks the
    agreement with the exact windowed projection."""
    K = 3
    D, b, seed, order = _window_case(K)
    A = synth.from_dense(D)
    ref = _pins.window_projection_exact(D.astype(np.int64), b.astype(np.int64), order, K)
    worst = 0.0
    for k in range(1, len(order) + 1):
        out = oracle.kaczmarz(A, b, tol=0.0, maxit=k, K=K, seed=seed, plant=plant)
        xr = np.array([float(v) for v in ref[k - 1]])
        worst = max(worst, rel(out["x"], xr))
    assert worst > 1e-3


def test_window_of_whole_pass_matches_full_history():
    """With K = m the first pass never empties the window: the identity
    sketch then reaches A^+ b on a wide full-row-rank A (Corollary 3.3),
    and the exact projection agrees step by step."""
    D, b, seed, order = _window_case(10)
    A = synth.from_dense(D)
    out = oracle.kaczmarz(A, b, tol=0.0, maxit=10, K=10, seed=seed)
    assert rel(out["x"], np.linalg.pinv(D) @ b) < 1e-10


# ---------------------------------------------- residual-sketch restarts

def _drift(rho, rho_s, since):
    return rho > 4.0 * rho_s


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("a,c,fires", [(4.0, 0.25, False), (5.0, 0.2, True), (10.0, 0.1, True)])
def test_drift_restart(prec, a, c, fires):
    """A = diag(1, a), b = (1, c): after the first update rho_1/rho_0 =
    rho_0 ||A y||^2/||y||^4 - 1 (y = A^T b) is 3.52, 5.76 and 24.5 for the
    three cases. The drift restart (rho above 4x its value at the last
    start) must fire exactly when that ratio exceeds 4; without a restart
    the second update solves the 2x2 system (Theorem 3.1), with one the
    second update is a fresh first step from b - A x_1."""
    D = np.diag([1.0, a])
    b = np.array([1.0, c])
    A = synth.from_dense(D)
    y = D.T @ b
    ratio = (b @ b) * np.sum((D @ y) ** 2) / (y @ y) ** 2 - 1.0
    assert (ratio > 4.0) == fires
    xs, rhos, restarts = _pins.projection_run_restarted(D, b, np.zeros(2), np.ones(2), 2, _drift)
    assert restarts[:1] == ([1] if fires else [])
    out = oracle.residual(A, b, tol=0.0, maxit=2, prec=prec, inner_tol=1e-150, hist=2)
    betas = out["hist_s"][:, 2]
    assert (betas[1] == 0.0) == fires
    tol = 1e-13 if prec == 0 else 1e-6
    for k in range(2):
        assert rel(out["hist_x"][k], xs[k]) < tol, k
    if not fires:
        assert rel(out["hist_x"][1], np.linalg.solve(D, b)) < tol


def test_planted_drift_threshold_is_caught():
    """A drift restart at 2x instead of 4x fires on the ratio-3.52 case and
    no longer solves the 2x2 system in two updates."""
    D = np.diag([1.0, 4.0])
    b = np.array([1.0, 0.25])
    A = synth.from_dense(D)
    bad = oracle.residual(A, b, tol=0.0, maxit=2, inner_tol=1e-150, hist=2, plant=2)
    assert rel(bad["hist_x"][1], np.linalg.solve(D, b)) > 1e-3


def _restart_case():
    rng = synth.rng_for(123)
    D = rng.standard_normal((40, 24)).astype(np.float32).astype(np.float64)
    b = D @ rng.standard_normal(24)
    return D, b


def _inner_rule(tau):
    def rule(rho, rho_s, since):
        return rho <= tau * tau * rho_s or rho > 4.0 * rho_s
    return rule


@pytest.mark.parametrize("prec", [0, 1])
def test_inner_restart_schedule(prec):
    """Restart of the inner solve once rho has fallen by inner_tol^2 since the
    last start: the restart indices and iterates equal those of eq:pkLong
    evaluated densely with a residual sketch that starts afresh where the
    rule, applied to the dense run's own ||b - A x_k||^2, fires. The rule's
    thresholds are crossed with a clear margin, so rounding cannot move a
    restart."""
    D, b = _restart_case()
    A = synth.from_dense(D)
    tau, K = 0.25, 16
    xs, rhos, restarts = _pins.projection_run_restarted(D, b, np.zeros(24), np.ones(24), K,
                                                       _inner_rule(tau))
    assert len(restarts) >= 3
    # margins: no rho within 5 % of a threshold
    rho_s, s = float(b @ b), 0
    for k, rho in enumerate(rhos, start=1):
        for thr in (tau * tau * rho_s, 4.0 * rho_s):
            assert abs(np.log(rho / thr)) > 0.05, (k, rho, thr)
        if k in restarts:
            rho_s = rho
    out = oracle.residual(A, b, tol=0.0, maxit=K, prec=prec, inner_tol=tau, hist=K)
    starts = [k for k in range(K) if out["hist_s"][k, 2] == 0.0]
    assert starts == [0] + restarts
    tol = 1e-9 if prec == 0 else 1e-4
    for k in range(K):
        assert rel(out["hist_x"][k], xs[k]) < tol, k


def test_planted_inner_threshold_is_caught():
    """Restarting once rho has fallen by inner_tol (instead of inner_tol^2)
    moves the restarts off the dense reference's indices."""
    D, b = _restart_case()
    A = synth.from_dense(D)
    tau, K = 0.25, 16
    _, _, restarts = _pins.projection_run_restarted(D, b, np.zeros(24), np.ones(24), K,
                                                   _inner_rule(tau))
    bad = oracle.residual(A, b, tol=0.0, maxit=K, inner_tol=tau, hist=K, plant=3)
    starts = [k for k in range(K) if bad["hist_s"][k, 2] == 0.0]
    assert starts != [0] + restarts


def test_refine_period():
    """FP32 storage with a restart every R = 3 updates: the restarts fall
    after updates 3, 6, 9, ... and the iterates follow eq:pkLong with the
    sketch started afresh at those updates."""
    D, b = _restart_case()
    A = synth.from_dense(D)
    K, R = 12, 3
    xs, _, restarts = _pins.projection_run_restarted(D, b, np.zeros(24), np.ones(24), K,
                                                    lambda rho, rho_s, since: since == R)
    assert restarts == [3, 6, 9, 12]
    out = oracle.residual(A, b, tol=0.0, maxit=K, prec=1, refine=R, hist=K)
    starts = [k for k in range(K) if out["hist_s"][k, 2] == 0.0]
    assert starts == [0, 3, 6, 9]
    for k in range(K):
        assert rel(out["hist_x"][k], xs[k]) < 1e-4, k


# ------------------------------------------------ residual replacement

@pytest.mark.parametrize("ci", range(5))
def test_replacement_leaves_fp64_iterates_unchanged(ci):
    """Residual replacement (refinement mode `replace`): every 2 updates the
    residual is recomputed as b - A x and replaces the recursive one while
    the recursion goes on. In exact arithmetic the two residuals are equal,
    so the iterates are those of eq:pkLong with the full residual sketch
    (no restart) for every k up to rank(A) -- to the same bar as the plain
    recursion's pin (test_oracle_pins.test_recursion_equals_pklong), on the
    same systems."""
    from tests.test_oracle_pins import CASES
    D, b, rank = CASES[ci]
    A = synth.from_dense(D)
    n = D.shape[1]
    x0 = synth.rng_for(11 + ci).standard_normal(n)
    xs, ps, _ = _pins.projection_run(D, b, x0, np.ones(n), rank, "residual")
    out = oracle.residual(A, b, x0=x0, tol=0.0, maxit=rank, refine=2, replace=True, hist=rank)
    assert all(out["hist_s"][k, 2] != 0.0 for k in range(1, rank))   # no restart after the first update
    for k in range(rank):
        assert rel(out["hist_x"][k], xs[k]) < 1e-10, k


def test_replacement_refreshes_the_fp32_residual():
    """FP32 storage with replacement every 3 updates: after updates 3, 6, 9
    the residual the recursion continues from is b - A x recomputed in double
    and rounded to float (and nothing restarts), while a restart of the same
    schedule begins a new recursion (beta = 0) at those updates."""
    D, b = _restart_case()
    A = synth.from_dense(D)
    K, R = 10, 3
    out = oracle.residual(A, b, tol=0.0, maxit=K, prec=1, refine=R, replace=True, hist=K)
    assert all(out["hist_s"][k, 2] != 0.0 for k in range(1, K))
    for k in (3, 6, 9):
        r_true = (b - D @ out["hist_x"][k - 1]).astype(np.float32).astype(np.float64)
        np.testing.assert_array_equal(out["hist_r"][k], r_true)
    rst = oracle.residual(A, b, tol=0.0, maxit=K, prec=1, refine=R, hist=K)
    assert [k for k in range(K) if rst["hist_s"][k, 2] == 0.0] == [0, 3, 6, 9]
