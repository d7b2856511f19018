"""plss_tune: the measured choice of the sweep plan. Every candidate is
measured, the answer is the fastest of them, and a context built with the
chosen plan solves to the oracle's iterates (the plan changes tile shapes
and schedules, never the arithmetic's result beyond summation order)."""
import numpy as np
import pytest

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


def _check_table(best, table, small_possible):
    shapes = {(e["layout"], e["tile_shift"]) for e in table}
    assert shapes == {(lay, s) for lay in ("auto", "csr") for s in (-1, 0, 1)}
    assert all(e["status"] == "ok" and e["us_per_update"] > 0 for e in table)
    assert {e["schedule"] for e in table} == ({"grid", "small"} if small_possible else {"grid"})
    win = min(table, key=lambda e: e["us_per_update"])
    assert best == {k: win[k] for k in ("layout", "tile_shift", "schedule")}


def test_tune_batched_and_solve_with_the_choice(plss):
    systems = synth.batched_systems(nsys=5, m_lo=300, m_hi=3000, len_lo=5, len_hi=20, seed0=70)
    As = [A.astype(np.float64) for A, _, _ in systems]
    bs = [b for _, b, _ in systems]
    best, table = plss.tune(As, updates=8)
    _check_table(best, table, small_possible=True)
    K = 30
    with plss.Context(As, layout=best["layout"], tile_shift=best["tile_shift"]) as ctx:
        xs, rs = ctx.solve_batched(bs, tol=0.0, maxit=K, schedule=best["schedule"])
    for A, b, x, r in zip(As, bs, xs, rs):
        assert r["iters"] == K
        _parity.check_x(x, _parity.reference(A, b, K), K)


@pytest.mark.parametrize("shift", [-2, 2])
def test_tile_shift_extremes_keep_parity(plss, shift):
    A, b, _ = synth.powerlaw_underdetermined(m=3000, n=9000, mean_len=12, max_len=400, seed=5)
    A = A.astype(np.float64)
    K = 25
    ref = _parity.reference(A, b, K)
    for layout in ("auto", "csr"):
        with plss.Context(A, layout=layout, tile_shift=shift) as ctx:
            x, res, hist = ctx.solve(b, tol=0.0, maxit=K, hist=K, schedule="grid")
        assert res["iters"] == ref["iters"]
        _parity.check_scalars(hist, ref, min_strict=1)
        _parity.check_x(x, ref, res["iters"])


def test_tune_fp32_single_system(plss):
    A, b, _ = synth.overdetermined_scaled(m=40_000, n=8_000, per_row=8, seed=9, scale_decades=1.0)
    best, table = plss.tune(A, updates=10, precision="fp32", w_mode=2)
    _check_table(best, table, small_possible=True)
