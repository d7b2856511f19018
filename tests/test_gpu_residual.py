"""GPU parity of the residual-sketch path (Algorithm 1) against the CPU oracle.

All solves go through the C ABI (libplss.so) via the thin Python binding.
Tolerance: FP64 mode, the per-update scalars (rho, phi, beta, gamma, theta)
and the iterates x_k agree with the oracle to 1e-10 relative (the parity bar
for double precision; the two sides differ only in summation order).
"""
import numpy as np
import pytest

import oracle
from paper_2207_07615_gb300 import synth
from tests import _parity

pytestmark = pytest.mark.gpu

RTOL = 1e-10


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


def scal_rel(h_gpu, h_ref):
    """Max relative difference of the per-update scalars, column by column."""
    k = min(len(h_gpu), len(h_ref))
    g, r = np.asarray(h_gpu[:k]), np.asarray(h_ref[:k])
    d = np.abs(g - r) / np.maximum(np.abs(r), 1e-300)
    d[:, 2][r[:, 2] == 0] = np.abs(g[:, 2])[r[:, 2] == 0]   # beta = 0 on the first update
    return float(d.max()) if d.size else 0.0


def test_smoke():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.smoke()


@pytest.mark.parametrize("schedule", ["small", "grid"])
def test_square_2000_every_iterate(plss, schedule):
    """The 2,000 x 2,000 diagonally dominant system, tol 1e-10: every update's
    scalars (rho, phi, beta, gamma, theta) and sampled iterates x_k against the
    oracle, at 1e-10 while the recursion's own rounding sensitivity allows it
    and within the calibrated bar after; same final answer."""
    A, b, xs = synth.square_diag_dominant()
    ref = _parity.reference(A, b, 2000)
    fin = oracle.residual(A, b, tol=1e-10, maxit=2000)
    with plss.Context(A) as ctx:
        x, res, hist = ctx.solve(b, tol=1e-10, maxit=2000, hist=2000, schedule=schedule)
        assert res["status"] == "converged"
        assert abs(res["iters"] - fin["iters"]) <= 2
        strict = _parity.check_scalars(hist, ref, min_strict=20)
        assert res["relres_true"] <= 2e-10
        assert rel(x, fin["x"]) < 1e-8
        for k in (1, 2, 3, 7, 15, strict, strict + 5, res["iters"]):
            xk, rk = ctx.solve(b, tol=0.0, maxit=k, schedule=schedule)
            assert rk["iters"] == k and rk["status"] == "not_converged"
            _parity.check_x(xk, ref, k)


def test_device_io_matches_host_io(plss):
    import torch
    A, b, xs = synth.square_diag_dominant(n=1500, per_row=8, seed=3)
    x0 = synth.rng_for(4).standard_normal(A.n)
    with plss.Context(A) as ctx:
        xh, rh = ctx.solve(b, x0, tol=1e-9)
        xd, rd = ctx.solve(torch.from_numpy(b).cuda(), torch.from_numpy(x0).cuda(), tol=1e-9)
        torch.cuda.synchronize()
    assert rh["iters"] == rd["iters"]
    np.testing.assert_array_equal(xh, xd.cpu().numpy())   # same kernels, same order


def test_determinism(plss):
    A, b, xs = synth.overdetermined_scaled(m=20000, n=4000, per_row=8, seed=5, scale_decades=1.0)
    with plss.Context(A.astype(np.float64)) as ctx:
        x1, r1 = ctx.solve(b, tol=1e-9, maxit=500)
        x2, r2 = ctx.solve(b, tol=1e-9, maxit=500)
    assert r1["iters"] == r2["iters"]
    np.testing.assert_array_equal(x1, x2)


def _shape(shape):
    if shape == "tall":
        return synth.overdetermined_scaled(m=30000, n=6000, per_row=8, seed=7, scale_decades=1.0)
    if shape == "wide":
        return synth.overdetermined_scaled(m=3000, n=9000, per_row=12, seed=8, scale_decades=0.5)
    return synth.powerlaw_underdetermined(m=4000, n=40000, mean_len=20, max_len=5000, seed=9)


_ORACLE_CACHE = {}


def _oracle_once(key, fn):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = fn()
    return _ORACLE_CACHE[key]


SCHEDULES = [("auto", "small"), ("auto", "grid"), ("csr", "grid")]


@pytest.mark.parametrize("layout,schedule", SCHEDULES)
@pytest.mark.parametrize("shape", ["tall", "wide", "powerlaw"])
def test_parity_shapes(plss, shape, layout, schedule):
    """Overdetermined with column scales, underdetermined, and power-law rows
    (rows longer than a tile run one CTA per row), with the sliced tiles
    (auto) and with the CSR/CSC only: 80 updates against the oracle
    (calibrated bar), then the solve to 1e-8 reaches the oracle's limit
    x0 + A^T (A A^T)^+ (b - A x0) within the accuracy the tolerance allows."""
    A, b, xs = _shape(shape)
    A = A.astype(np.float64)
    K = 80
    ref = _oracle_once((shape, "ref"), lambda: _parity.reference(A, b, K))
    with plss.Context(A, layout=layout) as ctx:
        lay = ctx.layout()
        if layout == "csr":
            assert lay["row_sliced"] == 0 and lay["col_sliced"] == 0
        elif shape == "powerlaw":
            # power-law rows pad slices too much and stay in the CSR; the
            # short columns are sliced
            assert lay["row_sliced"] < lay["row_tiles"] and lay["col_sliced"] > 0
        else:
            assert lay["row_sliced"] > 0 and lay["col_sliced"] > 0
        x, res, hist = ctx.solve(b, tol=0.0, maxit=K, hist=K, schedule=schedule)
        assert res["iters"] == K
        _parity.check_scalars(hist, ref, min_strict=10)
        _parity.check_x(x, ref, K)
        x, res = ctx.solve(b, tol=1e-8, maxit=200000, stop_on_true=1, schedule=schedule)
    assert res["status"] == "converged" and res["relres_true"] <= 1e-8
    if shape != "powerlaw":   # the oracle needs ~80k updates (a minute) there
        fin = _oracle_once((shape, "fin"),
                           lambda: oracle.residual(A, b, tol=1e-8, maxit=200000, stop_on_true=True))
        assert fin["status"] == "converged"
        assert rel(x, fin["x"]) < 1e-4


@pytest.mark.parametrize("w_mode", [1, 2])
def test_weighted_parity(plss, w_mode):
    """PLSS W (Sec. 4.1) with W = diag(1/||A_j||) or diag(1/||A_j||^2)."""
    A, b, xs = synth.overdetermined_scaled(m=20000, n=3000, per_row=8, seed=11, scale_decades=1.5)
    A = A.astype(np.float64)
    w = oracle.colweights(A, w_mode)
    K = 80
    ref = _parity.reference(A, b, K, w=w)
    with plss.Context(A) as ctx:
        x, res, hist = ctx.solve(b, tol=0.0, maxit=K, hist=K, w_mode=w_mode)
        _parity.check_scalars(hist, ref, min_strict=10)
        _parity.check_x(x, ref, K)
        x, res = ctx.solve(b, tol=1e-9, maxit=100000, w_mode=w_mode, stop_on_true=1)
    assert res["status"] == "converged" and res["relres_true"] <= 1e-9
    assert rel(x, xs) < 1e-5     # full column rank: the solution is x*


@pytest.mark.parametrize("layout", ["auto", "csr"])
def test_fp32_storage_parity_and_accuracy(plss, layout):
    """FP32 storage, FP64 scalars and refinement: early scalars follow the
    oracle's FP32 emulation to float rounding; with W = diag(1/||A_j||^2) the
    answer reaches the FP64 tolerance on b - A x and the FP64 oracle's x."""
    A, b, xs = synth.overdetermined_scaled(m=40000, n=8000, per_row=8, seed=12, scale_decades=1.0)
    emu = oracle.residual(A, b, tol=0.0, maxit=20, prec=1, stop_on_true=True, hist=20)
    w = oracle.colweights(A, 2)
    ref = oracle.residual(A, b, w=w, tol=1e-11, maxit=5000)
    with plss.Context(A, precision="fp32", layout=layout) as ctx:
        assert (ctx.layout()["row_sliced"] > 0) == (layout == "auto")
        _, _, hist = ctx.solve(b, tol=0.0, maxit=20, hist=20)
        assert _parity.rel_rows(hist[:8], emu["hist_s"][:8]).max() < 1e-4
        x, res = ctx.solve(b, tol=1e-8, maxit=5000, w_mode=2)
    assert res["status"] == "converged"
    assert res["relres_true"] <= 1e-8
    assert rel(x, ref["x"]) < 1e-6


def test_spmv_primitives(plss):
    A, b, xs = synth.powerlaw_underdetermined(m=3000, n=20000, mean_len=20, max_len=5000, seed=13)
    A = A.astype(np.float64)
    v = synth.rng_for(1).standard_normal(A.n)
    r = synth.rng_for(2).standard_normal(A.m)
    with plss.Context(A) as ctx:
        np.testing.assert_allclose(ctx.spmv(v), oracle.spmv(A, v), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(ctx.spmv(r, transpose=True), oracle.spmvt(A, r), rtol=1e-12, atol=1e-12)


def test_edge_cases(plss):
    A, b, xs = synth.square_diag_dominant(n=300, per_row=4, seed=2)
    x0 = np.linspace(-1, 1, 300)
    with plss.Context(A) as ctx:
        x, r = ctx.solve(np.zeros(300), x0, tol=1e-10)          # ||b|| = 0: x0 back at once
        assert r["status"] == "converged" and r["iters"] == 0
        np.testing.assert_array_equal(x, x0)
        x, r = ctx.solve(b, xs, tol=1e-10)                       # exact start
        assert r["iters"] == 0 and r["status"] == "converged"
        x, r = ctx.solve(b, tol=1e-12, maxit=0)                  # no update allowed
        assert r["iters"] == 0 and r["status"] == "not_converged"
        np.testing.assert_array_equal(x, np.zeros(300))
    # b outside range(A): A^T r0 = 0 gives phi_1 = 0 (breakdown)
    D = synth.from_dense(np.array([[1.0, 0.0], [0.0, 0.0]]))
    with plss.Context(D) as ctx:
        x, r = ctx.solve(np.array([0.0, 1.0]), tol=1e-12)
        assert r["status"] == "breakdown"
    # a 1 x 1 system and an empty-row / empty-column system
    with plss.Context(synth.from_dense(np.array([[4.0]]))) as ctx:
        x, r = ctx.solve(np.array([2.0]), tol=1e-14)
        assert r["status"] == "converged" and abs(x[0] - 0.5) < 1e-15
    Dz = np.zeros((5, 6))
    Dz[0, 1] = 2.0
    Dz[3, 4] = -1.0
    Dz[3, 1] = 0.5
    bz = Dz @ np.arange(1.0, 7.0)
    ref = oracle.residual(synth.from_dense(Dz), bz, tol=1e-13)
    with plss.Context(synth.from_dense(Dz)) as ctx:
        x, r = ctx.solve(bz, tol=1e-13)
    assert r["status"] == "converged" and r["iters"] == ref["iters"]
    assert rel(x, ref["x"]) < RTOL


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("schedule", ["grid", "small"])
def test_nonfinite_right_hand_side_ends_in_breakdown(plss, precision, schedule):
    """A NaN or an infinity in b (the library does not scan b) makes the
    first scalar step non-finite: the solve ends with PLSS_ERR_BREAKDOWN
    within a few bodies instead of running to the cap, in either storage
    and on either schedule, and the context solves the next system."""
    A, b, xs = synth.square_diag_dominant(n=300, per_row=4, seed=2)
    Ap = A.astype(np.float32) if precision == "fp32" else A
    with plss.Context(Ap, precision=precision) as ctx:
        for bad in (np.nan, np.inf):
            bb = b.copy()
            bb[17] = bad
            x, r = ctx.solve(bb, tol=1e-10, maxit=5000, schedule=schedule)
            assert r["status"] == "breakdown", r
            assert r["iters"] <= 1, r
        x, r = ctx.solve(b, tol=1e-8, maxit=5000, schedule=schedule)
        assert r["status"] == "converged" and r["relres_true"] <= 1e-8, r


@pytest.mark.parametrize("layout,schedule", SCHEDULES)
def test_ragged_tails(plss, layout, schedule):
    """Row counts just off the tile, slice and group boundaries."""
    for m in (1, 31, 33, 255, 257, 2049):
        A, b, xs = synth.powerlaw_underdetermined(m=m, n=3 * m + 7, mean_len=6, max_len=50, seed=m)
        A = A.astype(np.float64)
        K = 12
        ref = _parity.reference(A, b, K)
        with plss.Context(A, layout=layout) as ctx:
            x, res, hist = ctx.solve(b, tol=0.0, maxit=K, hist=K, schedule=schedule)
        assert res["iters"] == ref["iters"], m
        _parity.check_scalars(hist, ref, min_strict=1)
        if res["iters"]:
            _parity.check_x(x, ref, res["iters"])


@pytest.mark.parametrize("schedule", ["small", "grid"])
def test_batched_matches_single(plss, schedule):
    """Independent systems packed into one context: each system's trajectory
    equals the oracle's solve of that system alone, and each stops on its own."""
    systems = synth.batched_systems(nsys=6, m_lo=200, m_hi=4000, len_lo=5, len_hi=20, seed0=50)
    As = [A.astype(np.float64) for A, _, _ in systems]
    bs = [b for _, b, _ in systems]
    K = 40
    with plss.Context(As) as ctx:
        xs, rs = ctx.solve_batched(bs, tol=0.0, maxit=K, schedule=schedule)
        for A, b, x, r in zip(As, bs, xs, rs):
            ref = _parity.reference(A, b, K)
            assert r["iters"] == K and r["status"] == "not_converged"
            _parity.check_x(x, ref, K)
        xs, rs = ctx.solve_batched(bs, tol=1e-6, maxit=20000, stop_on_true=1, schedule=schedule)
    iters = set()
    for A, b, x, r in zip(As, bs, xs, rs):
        assert r["status"] == "converged" and r["relres_true"] <= 1e-6
        iters.add(r["iters"])
    assert len(iters) > 1     # systems stopped independently


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_symmetric_reuses_the_csr(plss, precision):
    """A symmetric matrix declared symmetric (A^T r reads the CSR and its
    sliced copy; no transpose stored) gives bit for bit the iterates of the
    same matrix with its transpose stored (the transpose is the same array),
    and those follow the oracle."""
    A = synth.laplacian7(N=18, dtype=np.float64)
    xs = synth.rng_for(31).standard_normal(A.n)
    b = synth.rhs(A, xs)
    K = 30
    Ap = A if precision == "fp64" else A.astype(np.float32)
    with plss.Context(Ap, precision=precision, symmetric=True) as cs, \
            plss.Context(Ap, precision=precision) as cg:
        assert cs.layout()["row_sliced"] > 0
        xa, ra = cs.solve(b, tol=0.0, maxit=K)
        xb, rb = cg.solve(b, tol=0.0, maxit=K)
        np.testing.assert_array_equal(xa, xb)
        if precision == "fp64":
            ref = _parity.reference(A, b, K)
            _parity.check_x(xa, ref, K)
        xa, ra = cs.solve(b, tol=1e-8, maxit=20000, stop_on_true=1)
    assert ra["status"] == "converged" and ra["relres_true"] <= 1e-8
    assert rel(xa, xs) < 1e-5      # nonsingular: the solution is x*


@pytest.mark.parametrize("w_mode", [0, 2])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_coop_schedule_parity(plss, w_mode, precision):
    """Schedule COOP (whole updates in one cooperative launch, grid barriers
    between the phases, scalar steps taken by every CTA): per-update scalars
    and x against the oracle (FP64), or against the oracle's FP32 emulation
    on the first updates and the FP64 answer (FP32 storage), and the same
    answer as the GRID schedule."""
    A, b, xs = synth.overdetermined_scaled(m=40000, n=8000, per_row=8, seed=14, scale_decades=1.0)
    w = oracle.colweights(A.astype(np.float64), w_mode) if w_mode else None
    with plss.Context(A if precision == "fp32" else A.astype(np.float64), precision=precision) as ctx:
        lay = ctx.layout()
        assert lay["row_sliced"] == lay["row_tiles"] and lay["col_sliced"] == lay["col_tiles"]
        if precision == "fp64":
            K = 60
            ref = _parity.reference(A.astype(np.float64), b, K, w=w)
            x, res, hist = ctx.solve(b, tol=0.0, maxit=K, hist=K, w_mode=w_mode, schedule="coop")
            assert res["iters"] == K
            _parity.check_scalars(hist, ref, min_strict=10)
            _parity.check_x(x, ref, K)
        else:
            K = 8
            ref = oracle.residual(A.astype(np.float64), b, w=w, tol=0.0, maxit=K, prec=1, hist=K)
            x, res, hist = ctx.solve(b, tol=0.0, maxit=K, hist=K, w_mode=w_mode, schedule="coop")
            assert scal_rel(hist, ref["hist_s"]) < 1e-4
        xc, rc = ctx.solve(b, tol=1e-8, maxit=20000, w_mode=w_mode, stop_on_true=1, schedule="coop")
        xg, rg = ctx.solve(b, tol=1e-8, maxit=20000, w_mode=w_mode, stop_on_true=1, schedule="grid")
    fin = oracle.residual(A.astype(np.float64), b, w=w, tol=1e-8, maxit=20000, stop_on_true=True)
    assert rc["status"] == rg["status"] == fin["status"] == "converged"
    assert rc["relres_true"] <= 1e-8
    assert rel(xc, fin["x"]) < 1e-5 and rel(xc, xg) < 1e-5


def test_gather_bound_diagnostic(plss):
    """plss_gather_bound times the gather-only walk of a sweep's own index
    stream on both sides (positive times, min <= median), and refuses an
    unknown side and a context whose sweeps run over plain CSR tiles (no
    warp ranges)."""
    A, b, _ = synth.overdetermined_scaled(m=200_000, n=40_000, per_row=8, seed=15)
    A = A.astype(np.float64)
    with plss.Context(A) as ctx:
        lay = ctx.layout()
        assert lay["row_sliced"] == lay["row_tiles"] and lay["col_sliced"] == lay["col_tiles"]
        for side in (0, 1):
            med, mn = ctx.gather_bound(side, reps=3)
            assert 0.0 < mn <= med
        with pytest.raises(plss.PlssError):
            ctx.gather_bound(2)
    with plss.Context(A, layout="csr") as ctx:
        with pytest.raises(plss.PlssError):
            ctx.gather_bound(0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_residual_replacement_parity(plss, precision):
    """Refinement by residual replacement (refine_mode REPLACE): the fresh
    b - A x replaces the recursive residual every 3 updates and the
    recursion goes on (no update after the first has beta = 0). FP64: every
    update's scalars and x against the oracle with the same schedule (the
    parity bar); FP32 storage: the first updates against the oracle's FP32
    emulation, and the solve to 1e-8 against the FP64 answer."""
    A, b, xs = synth.overdetermined_scaled(m=30000, n=6000, per_row=8, seed=16, scale_decades=1.0)
    A64 = A.astype(np.float64)
    K = 30
    kw = dict(refine_period=3, refine_mode="replace", inner_tol=0.0)
    with plss.Context(A64 if precision == "fp64" else A, precision=precision) as ctx:
        x, res, hist = ctx.solve(b, tol=0.0, maxit=K, hist=K, **kw)
        assert res["iters"] == K
        assert np.all(hist[1:K, 2] != 0.0)
        if precision == "fp64":
            r1 = oracle.residual(A64, b, tol=0.0, maxit=K, refine=3, replace=True, hist=K)
            r2 = oracle.residual(A64, b * _parity.F, tol=0.0, maxit=K, refine=3, replace=True, hist=K)
            ref = dict(r1)
            h2 = r2["hist_s"].copy()
            h2[:, [0, 1, 4]] /= _parity.F * _parity.F
            ss = np.maximum.accumulate(_parity.rel_rows(h2, r1["hist_s"]))
            sx = np.maximum.accumulate(_parity.rel_vec_rows(r2["hist_x"] / _parity.F, r1["hist_x"]))
            ref.update(tol_s=np.maximum(_parity.FLOOR, _parity.MARGIN * ss), spread_s=ss,
                       tol_x=np.maximum(_parity.FLOOR, _parity.MARGIN * sx), spread_x=sx)
            _parity.check_scalars(hist, ref, min_strict=8)
            _parity.check_x(x, ref, K)
        else:
            emu = oracle.residual(A64, b, tol=0.0, maxit=8, prec=1, refine=3, replace=True, hist=8)
            assert scal_rel(hist[:8], emu["hist_s"]) < 1e-4
        xf, rf = ctx.solve(b, tol=1e-8, maxit=40000, stop_on_true=1, **kw)
    fin = oracle.residual(A64, b, tol=1e-8, maxit=40000, stop_on_true=True)
    assert rf["status"] == "converged" and rf["relres_true"] <= 1e-8
    assert rel(xf, fin["x"]) < 1e-5


def test_replacement_converges_where_restarts_stall(plss):
    """The column-scaled system at 1/10 of the headline size, FP32 storage,
    W = I: refinement by restarts (inner tolerance 1e-4) stalls near 1e-6
    (the oracle's FP32 emulation stalls the same way: 7e-6 after 400,000
    updates), while residual replacement every 100 updates reaches 1e-8 in
    a number of updates close to FP64's (the emulation: 142,000 against
    135,000)."""
    A, b, _ = synth.overdetermined_scaled(m=100_000, n=20_000, per_row=8, seed=1)
    with plss.Context(A.astype(np.float64)) as c64:
        _, r64 = c64.solve(b, tol=1e-8, maxit=400_000, stop_on_true=1)
    with plss.Context(A, precision="fp32") as c32:
        _, rr = c32.solve(b, tol=1e-8, maxit=400_000, stop_on_true=1, refine_period=100,
                          refine_mode="replace", inner_tol=0.0)
        _, rs = c32.solve(b, tol=1e-8, maxit=200_000, stop_on_true=1)
    print(f"FP64 {r64['iters']} updates; FP32 replacement {rr['iters']} ({rr['relres_true']:.2e}); "
          f"FP32 restarts {rs['iters']} ({rs['relres_true']:.2e})")
    assert r64["status"] == "converged"
    assert rr["status"] == "converged" and rr["relres_true"] <= 1e-8
    assert rr["iters"] <= 1.3 * r64["iters"]
    assert rs["status"] == "not_converged" and rs["relres_true"] > 1e-7
