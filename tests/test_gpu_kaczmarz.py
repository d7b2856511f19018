"""GPU parity of the identity sketch (PLSS Kaczmarz, eq:pkKacz, Sec. 7)
against the CPU oracle, through the C ABI.

Both sides draw the same row order (SplitMix64 stream + Fisher-Yates
shuffle per pass from the same seed). Tolerance: 1e-10 relative on x, or
the parity margin times the oracle's own rounding spread (the oracle run
again on b (1 + 2^-50)) where that is larger. Windows of up to 64
directions run one CTA per system; larger ones (one system) run on the
whole GPU with grid barriers between a row's two phases.
"""
import numpy as np
import pytest

import oracle
from paper_2207_07615_gb300 import synth
from tests import _parity, _pins

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


def oracle_with_bar(A, b, maxit, K, seed, x0=None):
    r1 = oracle.kaczmarz(A, b, x0=x0, tol=0.0, maxit=maxit, K=K, seed=seed)
    r2 = oracle.kaczmarz(A, b * F, x0=None if x0 is None else x0 * F, tol=0.0, maxit=maxit, K=K, seed=seed)
    spread = rel(r2["x"] / F, r1["x"])
    return r1, max(_parity.FLOOR, _parity.MARGIN * spread)


def test_golden_2x2(plss):
    """The 2x2 system worked by hand (eq:pkKacz) in both row orders."""
    g = _pins.load_golden("plss_2x2_hand.txt")
    A = synth.from_dense(g["A"])
    seeds = {}
    for seed in range(200):
        perm, _ = oracle.permutation(seed, 2)
        seeds.setdefault(tuple(perm), seed)
    with plss.Context(A) as ctx:
        for order, tag in (((0, 1), "kz01"), ((1, 0), "kz10")):
            s = seeds[order]
            x1, _ = ctx.solve(g["b"], sketch="identity", kacz_hist=4, seed=s, tol=0.0, maxit=1)
            x2, _ = ctx.solve(g["b"], sketch="identity", kacz_hist=4, seed=s, tol=0.0, maxit=2)
            np.testing.assert_allclose(x1, g[tag + "_x1"], rtol=1e-15)
            np.testing.assert_allclose(x2, g[tag + "_x2"], rtol=1e-14)
        x2k0, _ = ctx.solve(g["b"], sketch="identity", kacz_hist=0, seed=seeds[(0, 1)], tol=0.0, maxit=2)
        np.testing.assert_allclose(x2k0, g["kz01_k0_x2"], rtol=1e-14)


@pytest.mark.parametrize("K", [0, 1, 4, 16, 17, 64])
def test_parity_powerlaw_rows(plss, K):
    """Underdetermined power-law rows (some longer than the CTA), several
    passes with restarts of the window, up to the one-CTA kernel's largest
    window."""
    A, b, xs = synth.powerlaw_underdetermined(m=600, n=6000, mean_len=20, max_len=1500, seed=21)
    A = A.astype(np.float64)
    with plss.Context(A) as ctx:
        for maxit, seed in ((1, 3), (7, 3), (600, 5), (2500, 5)):
            ref, bar = oracle_with_bar(A, b, maxit, K, seed)
            x, r = ctx.solve(b, sketch="identity", kacz_hist=K, seed=seed, tol=0.0, maxit=maxit)
            assert r["iters"] == maxit
            assert rel(x, ref["x"]) <= bar, (K, maxit, rel(x, ref["x"]), bar)


def test_converges_and_matches(plss):
    """A rank-deficient underdetermined power-law system (some rows repeat a
    single column): the window of 32 reaches 1e-8 where plain Kaczmarz
    stalls; both sides converge within a few passes of each other to the
    same limit."""
    A, b, xs = synth.powerlaw_underdetermined(m=400, n=4000, mean_len=12, max_len=600, seed=22)
    A = A.astype(np.float64)
    ref = oracle.kaczmarz(A, b, tol=1e-8, maxit=400 * 300, K=32, seed=9)
    with plss.Context(A) as ctx:
        x, r = ctx.solve(b, sketch="identity", kacz_hist=32, seed=9, tol=1e-8, maxit=400 * 300)
    assert ref["status"] == "converged"
    assert r["status"] == "converged" and r["relres_true"] <= 1e-8
    assert abs(r["iters"] - ref["iters"]) <= 0.25 * ref["iters"] + 400
    assert rel(x, ref["x"]) < 1e-4


def test_square_overdetermined_and_x0(plss):
    A, b, xs = synth.square_diag_dominant(n=300, per_row=5, seed=23)
    x0 = synth.rng_for(2).standard_normal(300)
    ref = oracle.kaczmarz(A, b, x0=x0, tol=0.0, maxit=900, K=3, seed=1)
    with plss.Context(A) as ctx:
        x, r = ctx.solve(b, x0, sketch="identity", kacz_hist=3, seed=1, tol=0.0, maxit=900)
    assert rel(x, ref["x"]) < 1e-9


@pytest.mark.parametrize("K,nsys", [(6, 11), (24, 4)])
def test_batched_identity(plss, K, nsys):
    """One CTA per system (eleven systems with a window of 6, four with 24);
    system s uses the row stream seeded seed + s."""
    systems = [synth.powerlaw_underdetermined(m=100 + 37 * s, n=900 + 100 * s, mean_len=8,
                                              max_len=120, seed=40 + s) for s in range(nsys)]
    As = [A.astype(np.float64) for A, _, _ in systems]
    bs = [b for _, b, _ in systems]
    with plss.Context(As) as ctx:
        xs, rs = ctx.solve_batched(bs, sketch="identity", kacz_hist=K, seed=100, tol=0.0, maxit=500)
    for s, (A, b, x, r) in enumerate(zip(As, bs, xs, rs)):
        ref, bar = oracle_with_bar(A, b, 500, K, 100 + s)
        assert r["iters"] == 500
        assert rel(x, ref["x"]) <= bar


@pytest.mark.parametrize("K", [65, 128, 512])
def test_wide_window_parity_powerlaw(plss, K):
    """Windows above 64 directions (the whole-GPU form): parity with the
    oracle after one row, part of a pass, and over several passes whose
    window resets straddle the passes."""
    A, b, xs = synth.powerlaw_underdetermined(m=600, n=6000, mean_len=20, max_len=1500, seed=21)
    A = A.astype(np.float64)
    with plss.Context(A) as ctx:
        for maxit, seed in ((1, 3), (70, 3), (1100, 5)):
            ref, bar = oracle_with_bar(A, b, maxit, K, seed)
            x, r = ctx.solve(b, sketch="identity", kacz_hist=K, seed=seed, tol=0.0, maxit=maxit)
            assert r["iters"] == maxit
            assert rel(x, ref["x"]) <= bar, (K, maxit, rel(x, ref["x"]), bar)


def test_wide_window_full_history_reaches_pinv(plss):
    """A window as long as a pass (K = m = 300 > 64) on a wide full-row-rank
    A: after the m rows of the first pass x solves A x = b with the least
    norm, x = A^+ b (Corollary 3.3), on the GPU as in the oracle."""
    rng = synth.rng_for(61)
    m, n = 300, 900
    D = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.02)
    D[np.arange(m), np.arange(m)] += 2.0
    A = synth.from_dense(D)
    b = D @ rng.standard_normal(n)
    ref, bar = oracle_with_bar(A, b, m, m, 7)
    with plss.Context(A) as ctx:
        x, r = ctx.solve(b, sketch="identity", kacz_hist=m, seed=7, tol=0.0, maxit=m)
    assert rel(x, ref["x"]) <= bar
    assert rel(x, np.linalg.pinv(D) @ b) < 1e-9


@pytest.mark.parametrize("K", [8, 40, 96])
def test_window_fp32_storage(plss, K):
    """FP32 storage of A with the one-CTA window (K = 8, 40) and the
    whole-GPU window (K = 96): the oracle on the same float-rounded values
    (the window algebra is in double on both sides)."""
    A, b, xs = synth.powerlaw_underdetermined(m=500, n=5000, mean_len=16, max_len=800, seed=24)
    A32 = A.astype(np.float32)
    A64 = A32.astype(np.float64)
    ref, bar = oracle_with_bar(A64, b, 900, K, 2)
    with plss.Context(A32, precision="fp32") as ctx:
        x, r = ctx.solve(b, sketch="identity", kacz_hist=K, seed=2, tol=0.0, maxit=900)
    assert rel(x, ref["x"]) <= bar


def test_window_limits_rejected(plss):
    """A window above 4,096 directions, or above 64 on a batched context,
    is refused before anything runs."""
    A, b, _ = synth.powerlaw_underdetermined(m=100, n=900, mean_len=8, max_len=60, seed=25)
    A = A.astype(np.float64)
    with plss.Context(A) as ctx:
        with pytest.raises(plss.PlssError):
            ctx.solve(b, sketch="identity", kacz_hist=4097, tol=0.0, maxit=10)
    with plss.Context([A, A]) as ctx:
        with pytest.raises(plss.PlssError):
            ctx.solve_batched([b, b], sketch="identity", kacz_hist=65, tol=0.0, maxit=10)


def test_wide_window_largest_cap_and_start_vector(plss):
    """The largest window (4,096 directions) on a small system with a start
    vector, against the oracle; and a system with a row longer than the
    8,192 entries a CTA holds is refused for windows above 64."""
    A, b, _ = synth.powerlaw_underdetermined(m=300, n=3000, mean_len=12, max_len=200, seed=26)
    A = A.astype(np.float64)
    x0 = synth.rng_for(8).standard_normal(A.n)
    ref, bar = oracle_with_bar(A, b, 700, 4096, 4, x0=x0)
    with plss.Context(A) as ctx:
        x, r = ctx.solve(b, x0, sketch="identity", kacz_hist=4096, seed=4, tol=0.0, maxit=700)
    assert rel(x, ref["x"]) <= bar
    m, n = 2, 9000
    rp = np.array([0, 8300, 8302], dtype=np.int64)
    ci = np.concatenate([np.arange(8300), [0, 1]]).astype(np.int32)
    Along = synth.CSR(m, n, rp, ci, np.ones(8302))
    with plss.Context(Along) as ctx:
        with pytest.raises(plss.PlssError):
            ctx.solve(np.ones(2), sketch="identity", kacz_hist=65, tol=0.0, maxit=2)
