"""plss_residual_noalloc: the residual entry point for callers that cannot
allocate device memory (their GPU memory belongs to their own pool, or is
fixed at start-up). It keeps its scratch in a static device array instead of
taking it from a context, so calls in a row must each give the same answer
as the context-based entry point (plss_spmv: r = b - A x from its A x) and
as the CPU oracle's product; calls of different sizes in a row show that
the shared scratch starts clean every time.

This file sorts last so that a failure here never hides another test's.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2207_07615_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-10   # the FP64 parity bar of the other GPU tests
MAX_ROWS = 4_194_304


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2207_07615_gb300 import plss
    return torch, plss


def _dev(torch, A):
    return (torch.from_numpy(np.ascontiguousarray(A.row_ptr, dtype=np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(A.col_idx, dtype=np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(A.val, dtype=np.float64)).cuda())


def _call(torch, plss, A_dev, m, n, nnz, x, b):
    rp, ci, val = A_dev
    r = torch.empty(max(m, 1), dtype=torch.float64, device="cuda")
    norm2 = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    xd = x if x.numel() else torch.zeros(1, dtype=torch.float64, device="cuda")
    bd = b if b.numel() else torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = plss.lib().plss_residual_noalloc(m, n, nnz, rp.data_ptr(), ci.data_ptr(), val.data_ptr(),
                                            xd.data_ptr(), bd.data_ptr(), r.data_ptr(),
                                            norm2.data_ptr(), stream)
    assert code == 0, plss.lib().plss_last_error().decode()
    torch.cuda.synchronize()
    return r.cpu().numpy()[:m], float(norm2.item())


def _check(r, n2, r_ref, b, ax):
    scale = np.abs(b) + np.abs(ax) + 1e-300
    assert np.max(np.abs(r - r_ref) / scale, initial=0.0) < RTOL
    np.testing.assert_allclose(n2, r_ref @ r_ref, rtol=RTOL)


def test_noalloc_matches_context_entry_point_and_oracle(env):
    """Two calls in a row on the same matrix: against plss_spmv (the
    context-based entry point) and against the oracle's product."""
    torch, plss = env
    A, _, _ = synth.powerlaw_underdetermined(m=30000, n=50000, mean_len=20, max_len=3000, seed=77)
    A = A.astype(np.float64)
    A_dev = _dev(torch, A)
    with plss.Context(A) as ctx:
        for seed in (1, 2):                      # two calls in a row
            rng = synth.rng_for(seed)
            x = rng.standard_normal(A.n)
            b = rng.standard_normal(A.m) * (10.0 ** seed)
            r, n2 = _call(torch, plss, A_dev, A.m, A.n, A.nnz,
                          torch.from_numpy(x).cuda(), torch.from_numpy(b).cuda())
            ax = ctx.spmv(x)                     # the existing entry point
            _check(r, n2, b - ax, b, ax)
            axo = oracle.spmv(A, x)              # the CPU oracle
            _check(r, n2, b - axo, b, axo)


def test_noalloc_calls_of_different_sizes(env):
    """A call over 30 blocks then one over 5 blocks (neither m a multiple of
    the 1,024-row block) and the first again: each matches the oracle, so
    no partial sum or arrival count of an earlier call leaks into a later
    one."""
    torch, plss = env
    mats = []
    for m, n, seed in ((30000 + 517, 4000, 5), (4099, 900, 6)):
        A, _, _ = synth.overdetermined_scaled(m=m, n=n, per_row=7, seed=seed, scale_decades=1.0)
        mats.append(A.astype(np.float64))
    for A in (mats[0], mats[1], mats[0]):
        rng = synth.rng_for(A.m)
        x = rng.standard_normal(A.n)
        b = rng.standard_normal(A.m)
        r, n2 = _call(torch, plss, _dev(torch, A), A.m, A.n, A.nnz,
                      torch.from_numpy(x).cuda(), torch.from_numpy(b).cuda())
        ax = oracle.spmv(A, x)
        _check(r, n2, b - ax, b, ax)


def test_noalloc_empty_inputs(env):
    """m = 0 gives ||r||^2 = 0; nnz = 0 gives r = b."""
    torch, plss = env
    A0 = synth.from_dense(np.zeros((0, 3)))
    r, n2 = _call(torch, plss, _dev(torch, A0), 0, 3, 0,
                  torch.zeros(3, dtype=torch.float64, device="cuda"),
                  torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert n2 == 0.0 and r.size == 0
    Ae = synth.from_dense(np.zeros((2500, 7)))
    assert Ae.nnz == 0
    b = synth.rng_for(3).standard_normal(2500)
    r, n2 = _call(torch, plss, _dev(torch, Ae), 2500, 7, 0,
                  torch.zeros(7, dtype=torch.float64, device="cuda"), torch.from_numpy(b).cuda())
    np.testing.assert_array_equal(r, b)
    np.testing.assert_allclose(n2, b @ b, rtol=RTOL)


def test_noalloc_at_its_row_limit(env):
    """m = 4,194,304, the most rows the static scratch covers (4,096 blocks),
    against the oracle."""
    torch, plss = env
    m, n, per = MAX_ROWS, 5000, 2
    rng = synth.rng_for(11)
    row_ptr = np.arange(m + 1, dtype=np.int64) * per
    col = np.sort(rng.integers(0, n, size=(m, per)), axis=1)
    col[:, 1] = np.where(col[:, 1] == col[:, 0], (col[:, 0] + 1) % n, col[:, 1])
    col = np.sort(col, axis=1).astype(np.int32).ravel()
    val = rng.standard_normal(m * per)
    A = synth.CSR(m, n, row_ptr, col, val)
    x = rng.standard_normal(n)
    b = rng.standard_normal(m)
    r, n2 = _call(torch, plss, _dev(torch, A), m, n, A.nnz,
                  torch.from_numpy(x).cuda(), torch.from_numpy(b).cuda())
    ax = oracle.spmv(A, x)
    _check(r, n2, b - ax, b, ax)


def test_noalloc_flags_a_broken_csr_and_recovers(env):
    """A column index outside [0, n) and a row range beyond nnz are skipped by
    the kernel's own guards (nothing is read out of bounds) and reported as
    ||r||^2 = NaN; the next valid call is unaffected."""
    torch, plss = env
    A, _, _ = synth.overdetermined_scaled(m=3000, n=500, per_row=5, seed=9, scale_decades=0.5)
    A = A.astype(np.float64)
    x = synth.rng_for(1).standard_normal(A.n)
    b = synth.rng_for(2).standard_normal(A.m)
    xd, bd = torch.from_numpy(x).cuda(), torch.from_numpy(b).cuda()
    rp, ci, val = _dev(torch, A)
    bad_ci = ci.clone()
    bad_ci[17] = A.n + 5                            # column beyond n
    _, n2 = _call(torch, plss, (rp, bad_ci, val), A.m, A.n, A.nnz, xd, bd)
    assert np.isnan(n2)
    bad_rp = rp.clone()
    bad_rp[A.m] = A.nnz + 40                        # last row runs past nnz
    _, n2 = _call(torch, plss, (bad_rp, ci, val), A.m, A.n, A.nnz, xd, bd)
    assert np.isnan(n2)
    r, n2 = _call(torch, plss, (rp, ci, val), A.m, A.n, A.nnz, xd, bd)
    ax = oracle.spmv(A, x)
    _check(r, n2, b - ax, b, ax)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, plss = env
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    code = plss.lib().plss_residual_noalloc(MAX_ROWS + 1, 1, 0, p, p, p, p, p, p, p, None)
    assert code == -1
    assert "4194304" in plss.lib().plss_last_error().decode()
