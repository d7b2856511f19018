"""plss_residual_noalloc: the residual entry point for callers that cannot
allocate device memory (their GPU memory belongs to their own pool, or is
fixed at start-up). It keeps its scratch in a static device array instead of
taking it from a context, so two calls in a row must each give the same
answer as the context-based entry point (plss_spmv: r = b - A x from its A x)
-- the second call shows the shared scratch starts clean.

This file sorts last so that a failure here never hides another test's.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2207_07615_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-10   # the FP64 parity bar of the other GPU tests


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2207_07615_gb300 import plss
    return torch, plss


def _call(torch, plss, A_dev, m, n, nnz, x, b):
    rp, ci, val = A_dev
    r = torch.empty(m, dtype=torch.float64, device="cuda")
    norm2 = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = plss.lib().plss_residual_noalloc(m, n, nnz, rp.data_ptr(), ci.data_ptr(), val.data_ptr(),
                                            x.data_ptr(), b.data_ptr(), r.data_ptr(),
                                            norm2.data_ptr(), stream)
    assert code == 0, plss.lib().plss_last_error().decode()
    torch.cuda.synchronize()
    return r.cpu().numpy(), float(norm2.item())


def test_noalloc_matches_context_entry_point_twice(env):
    torch, plss = env
    A, _, _ = synth.powerlaw_underdetermined(m=30000, n=50000, mean_len=20, max_len=3000, seed=77)
    A = A.astype(np.float64)
    A_dev = (torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col_idx).cuda(),
             torch.from_numpy(A.val).cuda())
    with plss.Context(A) as ctx:
        for seed in (1, 2):                      # two calls in a row
            rng = synth.rng_for(seed)
            x = rng.standard_normal(A.n)
            b = rng.standard_normal(A.m) * (10.0 ** seed)
            ax = ctx.spmv(x)                     # the existing entry point
            r_ref = b - ax
            r, n2 = _call(torch, plss, A_dev, A.m, A.n, A.nnz,
                          torch.from_numpy(x).cuda(), torch.from_numpy(b).cuda())
            scale = np.abs(b) + np.abs(ax) + 1e-300
            assert np.max(np.abs(r - r_ref) / scale) < RTOL
            np.testing.assert_allclose(n2, r_ref @ r_ref, rtol=RTOL)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, plss = env
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    code = plss.lib().plss_residual_noalloc(4_194_305, 1, 0, p, p, p, p, p, p, p, None)
    assert code == -1
    assert "4194304" in plss.lib().plss_last_error().decode()
