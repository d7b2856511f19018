"""Checkpoint and resume of the residual sketch (plss_resume,
plss_state_save / plss_state_load), through the C ABI.

A solve stopped by its update cap and resumed must give the iterates of the
uninterrupted solve bit for bit: every reduction runs in a fixed order and
the stopping rule keeps the transition the recursion was about to take.
Compared: x, the update count, and the scalars of Algorithm 1 for the
updates after the stop (the history rows). The resumed answer is also
checked against the CPU oracle at the parity bar of the other GPU tests.
"""
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


def _system(seed=3, m=20000, n=4000, decades=2.0):
    A, b, xs = synth.overdetermined_scaled(m=m, n=n, per_row=8, seed=seed, scale_decades=decades)
    return A, b


def _same(x1, x2):
    assert np.array_equal(np.asarray(x1), np.asarray(x2)), float(np.max(np.abs(np.asarray(x1) - np.asarray(x2))))


@pytest.mark.parametrize("schedule", ["grid", "small"])
def test_resume_reproduces_the_uninterrupted_solve(plss, schedule):
    """FP64: 700 updates at once against 260 + (resume to) 700."""
    A, b = _system(m=6000, n=1500) if schedule == "small" else _system()
    A = A.astype(np.float64)
    N, N1 = 700, 260
    with plss.Context(A) as ctx:
        x_full, r_full, h_full = ctx.solve(b, tol=0.0, maxit=N, hist=N, schedule=schedule)
        x1, r1 = ctx.solve(b, tol=0.0, maxit=N1, schedule=schedule)
        assert r1["status"] == "not_converged" and r1["iters"] == N1
        xs, rs, h = ctx.resume(tol=0.0, maxit=N, hist=N, schedule=schedule)
    assert rs[0]["iters"] == r_full["iters"] == N
    _same(xs[0], x_full)
    assert np.array_equal(h[N1:N], h_full[N1:N])


def test_state_moves_between_contexts(plss):
    """Save after the stop, load into a second context of the same matrix,
    resume there: the same iterates; the answer agrees with the oracle."""
    A, b = _system(seed=4)
    A = A.astype(np.float64)
    N, N1 = 900, 333
    with plss.Context(A) as ctx:
        x_full, r_full = ctx.solve(b, tol=0.0, maxit=N)
        ctx.solve(b, tol=0.0, maxit=N1)
        blob = ctx.state_save()
    with plss.Context(A) as ctx2:
        ctx2.state_load(blob)
        xs, rs = ctx2.resume(tol=0.0, maxit=N)
    _same(xs[0], x_full)
    assert rs[0]["iters"] == N
    ref = _parity.reference(A, b, N)
    _parity.check_x(xs[0], ref, N)


@pytest.mark.parametrize("mode", ["restart", "replace"])
def test_fp32_refinement_resumes_mid_period(plss, mode):
    """FP32 storage with refinement every 50 updates, stopped at 437 (inside a
    period) and resumed to 900, against 900 at once; then, with W =
    diag(1/||A_j||), stopped at 300 and resumed to the tolerance."""
    A, b = _system(seed=5)
    A32 = A.astype(np.float32)
    kw = dict(refine_period=50, refine_mode=mode)
    with plss.Context(A32, precision="fp32") as ctx:
        x_full, r_full = ctx.solve(b, tol=0.0, maxit=900, **kw)
        ctx.solve(b, tol=0.0, maxit=437, **kw)
        xs, rs = ctx.resume(tol=0.0, maxit=900, **kw)
        _same(xs[0], x_full)
        assert rs[0]["iters"] == r_full["iters"]
        # to a tolerance (with column weights, which this scaling needs in FP32)
        x_tol, r_tol = ctx.solve(b, tol=1e-6, maxit=20000, w_mode=1, **kw)
        ctx.solve(b, tol=1e-6, maxit=300, w_mode=1, **kw)
        xs2, rs2 = ctx.resume(tol=1e-6, maxit=20000, w_mode=1, **kw)
    assert r_tol["status"] == "converged" and rs2[0]["status"] == "converged"
    assert rs2[0]["iters"] == r_tol["iters"]
    _same(xs2[0], x_tol)


def test_batched_systems_resume_independently(plss):
    """Three systems; a tolerance the first reaches before the stop: it stays
    converged, the others go on, all as in the uninterrupted batched solve."""
    systems = [_system(seed=10 + s, m=3000 + 500 * s, n=700 + 100 * s, decades=0.5) for s in range(3)]
    As = [A.astype(np.float64) for A, _ in systems]
    bs = [b for _, b in systems]
    with plss.Context(As) as ctx:
        xf, rf = ctx.solve_batched(bs, tol=1e-9, maxit=5000)
        assert all(r["status"] == "converged" for r in rf), rf
        cut = min(r["iters"] for r in rf) + 5            # the first has converged, the others not
        assert sum(r["iters"] > cut for r in rf) >= 1, rf
        x1, r1 = ctx.solve_batched(bs, tol=1e-9, maxit=cut)
        xs, rs = ctx.resume(tol=1e-9, maxit=5000)
    for s in range(3):
        assert rs[s]["status"] == rf[s]["status"] and rs[s]["iters"] == rf[s]["iters"], (s, rs[s], rf[s])
        _same(xs[s], xf[s])


def test_resume_of_a_converged_solve_changes_nothing(plss):
    A, b = _system(seed=6, m=5000, n=1000, decades=0.5)
    A = A.astype(np.float64)
    with plss.Context(A) as ctx:
        x, r = ctx.solve(b, tol=1e-8, maxit=20000)
        assert r["status"] == "converged"
        xs, rs = ctx.resume(tol=1e-8, maxit=20000)
    assert rs[0]["status"] == "converged" and rs[0]["iters"] == r["iters"]
    _same(xs[0], x)


def test_resume_and_load_refusals(plss):
    A, b = _system(seed=7, m=5000, n=1000)
    B, _ = _system(seed=8, m=5200, n=1000)
    A = A.astype(np.float64)
    B = B.astype(np.float64)
    with plss.Context(A) as ctx:
        with pytest.raises(plss.PlssError, match="no residual-sketch state"):
            ctx.resume(tol=0.0, maxit=10)
        ctx.solve(b, tol=0.0, maxit=20)
        blob = ctx.state_save()
        with pytest.raises(plss.PlssError, match="bytes"):
            ctx.state_load(blob[: len(blob) // 2])
        with pytest.raises(plss.PlssError, match="version"):
            ctx.state_load(b"X" + blob[1:])
        # the scalars of system 0 start after the 48-byte header; its update
        # count is at +64 (after eight doubles), its phase at +128
        import struct
        for fmt, off, val in (("<q", 48 + 64, -1), ("<i", 48 + 128, 1)):
            bad = bytearray(blob)
            struct.pack_into(fmt, bad, off, val)
            with pytest.raises(plss.PlssError, match="not those of a finished solve"):
                ctx.state_load(bytes(bad))
        ctx.state_load(blob)                                  # the intact state still loads
        xs, rs = ctx.resume(tol=0.0, maxit=30)
        assert rs[0]["iters"] == 30
        ctx.solve(b, sketch="identity", tol=0.0, maxit=10)   # overwrites x and b
        with pytest.raises(plss.PlssError, match="no residual-sketch state"):
            ctx.resume(tol=0.0, maxit=30)
    with plss.Context(B) as ctx2:
        with pytest.raises(plss.PlssError, match="other sizes"):
            ctx2.state_load(blob)
