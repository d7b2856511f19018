"""Continuous-batching server (plss_submit / plss_poll) on the GPU.

Two properties: every served request follows the CPU oracle (Algorithm 1
with the same options: the iteration count within the oracle's own rounding
spread, and x equal to the oracle's to that spread, or at least within the
solve's tolerance of it on the residual), and a request's result in the mix
equals the same request solved alone (plss_solve with the same options):
each system's tiles, partial sums and reduction order do not depend on its
neighbours, so the two agree bit for bit.
"""
import time

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


def requests(count, seed=500, m_lo=300, m_hi=6000):
    """Serving-shaped requests: m log-uniform, n/m in {0.5, 1, 2}, 8-32
    nonzeros per row, N(0,1) values, b = A x*."""
    out = []
    for i in range(count):
        rng = synth.rng_for(seed + i)
        m = int(round(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi)))))
        n = max(1, int(round(m * (0.5, 1.0, 2.0)[int(rng.integers(0, 3))])))
        lengths = np.minimum(rng.integers(8, 33, size=m), n).astype(np.int64)
        cols = synth.distinct_columns(rng, lengths, n)
        rp = np.zeros(m + 1, dtype=np.int64)
        np.cumsum(lengths, out=rp[1:])
        A = synth.CSR(m, n, rp, cols, rng.standard_normal(int(lengths.sum())))
        out.append((A, synth.rhs(A, rng.standard_normal(n))))
    return out


def drain(srv, tickets, timeout=300.0):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        for t in tickets:
            if t in res:
                continue
            r = srv.poll(t)
            if r is not None:
                res[t] = r
        assert time.time() - t0 < timeout, "server did not finish in time"
        time.sleep(0.001)
    return res


@pytest.mark.parametrize("layout", ["auto", "csr"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mix_equals_alone(plss, precision, layout):
    """Each request in the mix gets bit for bit what it gets alone: with the
    CSR layout, what a context created with it computes; with sliced tiles,
    what the same request served alone computes."""
    reqs = requests(14)
    kw = dict(tol=1e-6, maxit=3000, w_mode=1)
    srv = plss.Server(max_slots=4, precision=precision, hbm_budget_bytes=256 << 20, layout=layout)
    try:
        tickets = [srv.submit(A, b, **kw) for A, b in reqs]
        assert all(t is not None for t in tickets)
        got = drain(srv, tickets)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["queued"] == 0 and st["running"] == 0
    finally:
        srv.close()
    for (A, b), t in zip(reqs, tickets):
        _check_oracle(A, b, *got[t], precision=precision, **kw)
    alone = None
    if layout == "auto":
        alone = plss.Server(max_slots=1, precision=precision, hbm_budget_bytes=256 << 20, layout=layout)
    try:
        for (A, b), t in zip(reqs, tickets):
            x_mix, r_mix = got[t]
            if alone is not None:
                t1 = alone.submit(A, b, **kw)
                x_one, r_one = drain(alone, [t1])[t1]
            else:
                with plss.Context(A, precision=precision, layout="csr") as ctx:
                    x_one, r_one = ctx.solve(b, stop_on_true=1, schedule="grid", **kw)
            _check_same(r_mix, r_one, x_mix, x_one)
    finally:
        if alone is not None:
            alone.close()


_ORACLE = {}


def _oracle_runs(A, b, precision, tol, maxit, w_mode):
    """The oracle with the server's options (stop on the true residual; FP32
    storage refines once rho has fallen by 1e-4^2 since the last start), on b
    and on b scaled by 1 + j eps, j = -2, -1, 1, 2 -- rounding-level changes
    of the input (eps = 2^-50 in FP64; 2^-24, the float unit roundoff, for
    FP32 storage, whose GPU form sums products in double-float where the
    oracle's emulation sums them in float). Cached per request."""
    key = (A.m, A.n, A.nnz, float(A.val[:4].sum()), float(b[:4].sum()), precision, tol, maxit, w_mode)
    if key not in _ORACLE:
        w = oracle.colweights(A, w_mode) if w_mode else None
        kw = dict(w=w, tol=tol, maxit=maxit, stop_on_true=True)
        eps = 2.0 ** -50
        if precision == "fp32":
            kw.update(prec=1, inner_tol=1e-4)
            eps = 2.0 ** -24
        runs = [oracle.residual(A, b * (1.0 + j * eps), **kw) for j in (0, -2, -1, 1, 2)]
        _ORACLE[key] = (runs, eps)
    return _ORACLE[key]


def _check_oracle(A, b, x, res, precision, tol, maxit, w_mode):
    """A served request against the oracle run with the same options. The
    oracle's own iteration counts over rounding-level changes of b (see
    _oracle_runs) give the spread that rounding alone causes in this
    Lanczos-type recursion. A one-time change of b under-represents a
    different summation order in every sweep, which perturbs every update
    (over 1,500 updates the GPU's count moved by up to 0.6 % from the
    oracle's while the oracle's own spread was 0.3 %), so the served count
    must lie within max(2, 2 x that spread, 1 % of the oracle's count) of
    the oracle's. When the counts agree in FP64, x must equal the
    oracle's to within the parity margin times the oracle's own x spread.
    Every converged request has both b - A x_served and b - A x_oracle within
    tol ||b||, so ||A (x_served - x_oracle)|| <= 2 tol ||b|| (checked with
    25 % slack for the final rounding)."""
    runs, eps = _oracle_runs(A, b, precision, tol, maxit, w_mode)
    o1 = runs[0]
    its = [o["iters"] for o in runs]
    spread_it = max(its) - min(its)
    assert res["status"] == o1["status"]
    bound = max(2, 2 * spread_it, int(np.ceil(0.01 * o1["iters"])))
    assert abs(res["iters"] - o1["iters"]) <= bound, (res["iters"], its)
    nx = max(np.linalg.norm(o1["x"]), 1e-300)
    if res["iters"] == o1["iters"] and precision == "fp64":
        spread_x = max(np.linalg.norm(o["x"] / (1.0 + j * eps) - o1["x"]) / nx
                       for o, j in zip(runs[1:], (-2, -1, 1, 2)))
        dx = np.linalg.norm(x - o1["x"]) / nx
        assert dx <= max(_parity.FLOOR, _parity.MARGIN * spread_x), (dx, spread_x)
    if o1["status"] == "converged":
        d = oracle.spmv(A, x - o1["x"])
        assert np.linalg.norm(d) <= 2.5 * tol * np.linalg.norm(b)


def _check_same(r_mix, r_one, x_mix, x_one):
    assert r_mix["status"] == r_one["status"]
    assert r_mix["iters"] == r_one["iters"]
    np.testing.assert_array_equal(x_mix, x_one)
    if r_mix["status"] == "converged":
        assert r_mix["relres_true"] <= 1e-6
    assert r_mix["seconds"] > 0


def test_admission_by_memory(plss):
    """A small arena: requests queue until earlier ones free room."""
    reqs = requests(10, seed=900, m_lo=2000, m_hi=6000)
    srv = plss.Server(max_slots=16, hbm_budget_bytes=6 << 20, layout="csr")
    try:
        tickets = [srv.submit(A, b, tol=1e-6, maxit=2000, w_mode=1) for A, b in reqs]
        peak_running, peak_bytes = 0, 0
        res = {}
        t0 = time.time()
        while len(res) < len(tickets):
            s = srv.stats()
            peak_running = max(peak_running, s["running"])
            peak_bytes = max(peak_bytes, s["bytes_in_use"])
            for t in tickets:
                if t not in res:
                    r = srv.poll(t)
                    if r is not None:
                        res[t] = r
            assert time.time() - t0 < 300
        assert peak_bytes <= 6 << 20
        assert 1 <= peak_running < len(reqs)
    finally:
        srv.close()


def test_busy_and_unknown_ticket(plss):
    srv = plss.Server(max_slots=2, hbm_budget_bytes=16 << 20)
    try:
        big, bb = synth.overdetermined_scaled(m=400000, n=100000, per_row=8, seed=3)[:2]
        assert srv.submit(big, bb) is None                   # can never fit: BUSY
        with pytest.raises(plss.PlssError):
            srv.poll(123456)                                 # unknown ticket
        A, b = requests(1)[0]
        t = srv.submit(A, b, tol=1e-6, maxit=3000)
        drain(srv, [t])
        with pytest.raises(plss.PlssError):
            srv.poll(t)                                      # already collected
    finally:
        srv.close()
