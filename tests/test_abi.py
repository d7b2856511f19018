"""C ABI checks that need no GPU: the library builds, loads, exports every
symbol include/plss.h declares, and rejects malformed input on the host."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2207_07615_gb300 import build as pbuild
from paper_2207_07615_gb300 import plss, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    pbuild.build()
    return plss.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "plss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(plss_[a-z_]+)\s*\(", src)))


def test_exports_match_header(L):
    names = header_functions()
    assert set(names) == set(plss.EXPORTS), (names, plss.EXPORTS)
    for name in names:
        assert hasattr(L, name), name


def test_struct_layouts(L):
    assert C.sizeof(plss.Opts) == 120
    assert C.sizeof(plss.Csr) == 56
    assert C.sizeof(plss.Result) == 40
    assert C.sizeof(plss.ServerOpts) == 32
    assert C.sizeof(plss.TuneEntry) == 24
    o = plss.Opts()
    L.plss_opts_default(C.byref(o))
    assert o.tol == 1e-8 and o.maxit == -1 and o.sketch == 0 and o.precision == 0
    assert o.inner_tol == 1e-4 and o.tile_shift == 0 and o.refine_mode == 0


def _create(L, csr):
    h = C.c_void_p()
    o = plss.Opts()
    L.plss_opts_default(C.byref(o))
    code = L.plss_create(C.byref(csr), C.byref(o), C.byref(h))
    return code, L.plss_last_error().decode(), h


def _csr(rp, ci, val, m, n):
    rp = np.asarray(rp, dtype=np.int64)
    ci = np.asarray(ci, dtype=np.int32)
    val = np.asarray(val, dtype=np.float64)
    keep = (rp, ci, val)
    c = plss.Csr(m, n, int(rp[-1]), rp.ctypes.data, ci.ctypes.data, val.ctypes.data, 0, 0)
    return c, keep


@pytest.mark.parametrize("case,msg", [
    (([1, 2], [0, 1], [1.0, 1.0], 1, 2), "row_ptr[0]"),
    (([0, 2, 1], [0], [1.0], 2, 2), "decreases"),
    (([0, 2], [1, 0], [1.0, 1.0], 1, 2), "strictly increasing"),
    (([0, 2], [0, 0], [1.0, 1.0], 1, 2), "strictly increasing"),
    (([0, 1], [5], [1.0], 1, 2), "outside"),
    (([0, 1], [-1], [1.0], 1, 2), "outside"),
    (([0, 1], [0], [np.nan], 1, 2), "non-finite"),
])
def test_malformed_csr_rejected(L, case, msg):
    rp, ci, val, m, n = case
    if rp[-1] != len(ci):
        pytest.skip("inconsistent fixture")
    c, keep = _csr(rp, ci, val, m, n)
    code, err, h = _create(L, c)
    assert code == plss.ERR_INVALID
    assert msg in err
    assert not h.value


def test_rowptr_end_mismatch(L):
    rp = np.array([0, 1], dtype=np.int64)
    ci = np.array([0], dtype=np.int32)
    val = np.array([1.0])
    c = plss.Csr(1, 2, 2, rp.ctypes.data, ci.ctypes.data, val.ctypes.data, 0, 0)
    code, err, h = _create(L, c)
    assert code == plss.ERR_INVALID and "row_ptr[m]" in err


def test_null_and_negative(L):
    h = C.c_void_p()
    assert L.plss_create(None, None, C.byref(h)) == plss.ERR_INVALID
    c = plss.Csr(-1, 2, 0, None, None, None, 0, 0)
    code, err, _ = _create(L, c)
    assert code == plss.ERR_INVALID and "negative" in err
    assert L.plss_solve(None, None, None, None, None, None) == plss.ERR_INVALID
    assert L.plss_create_batched(None, 0, None, C.byref(h)) == plss.ERR_INVALID


def test_last_error_is_per_thread(L):
    import threading
    c = plss.Csr(-1, 2, 0, None, None, None, 0, 0)
    _create(L, c)
    seen = {}

    def other():
        seen["err"] = L.plss_last_error().decode()
    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["err"] == ""
    assert "negative" in L.plss_last_error().decode()


def test_sizes_beyond_int32_rejected(L):
    """Indices are int32 on the device: larger sizes are refused before any
    array is read (the pointers here are NULL)."""
    for m, n, nnz in ((2**31, 2, 0), (2, 2**31, 0), (2, 2, 2**31)):
        c = plss.Csr(m, n, nnz, None, None, None, 0, 0)
        code, err, h = _create(L, c)
        assert code == plss.ERR_INVALID and "2^31" in err and not h.value


def test_unknown_options_rejected(L):
    """Option values outside their enums are refused at create."""
    rp = np.array([0, 1], dtype=np.int64)
    ci = np.array([0], dtype=np.int32)
    val = np.array([1.0])
    c = plss.Csr(1, 1, 1, rp.ctypes.data, ci.ctypes.data, val.ctypes.data, 0, 0)
    for field, bad in (("precision", 7), ("layout", 5), ("tile_shift", 3), ("tile_shift", -3)):
        o = plss.Opts()
        L.plss_opts_default(C.byref(o))
        setattr(o, field, bad)
        h = C.c_void_p()
        assert L.plss_create(C.byref(c), C.byref(o), C.byref(h)) == plss.ERR_INVALID
        assert not h.value


def test_tune_rejects_bad_arguments(L):
    """plss_tune validates its arguments before it builds anything."""
    rp = np.array([0, 1], dtype=np.int64)
    ci = np.array([0], dtype=np.int32)
    val = np.array([1.0])
    c = plss.Csr(1, 1, 1, rp.ctypes.data, ci.ctypes.data, val.ctypes.data, 0, 0)
    best = plss.Opts()
    cnt = C.c_int32()
    ent = (plss.TuneEntry * 4)()
    cases = [(None, 1, 5, C.byref(best), ent, 4, C.byref(cnt)),
             (C.byref(c), 0, 5, C.byref(best), ent, 4, C.byref(cnt)),
             (C.byref(c), 1, 0, C.byref(best), ent, 4, C.byref(cnt)),
             (C.byref(c), 1, 100001, C.byref(best), ent, 4, C.byref(cnt)),
             (C.byref(c), 1, 5, None, ent, 4, C.byref(cnt)),
             (C.byref(c), 1, 5, C.byref(best), None, 4, C.byref(cnt)),
             (C.byref(c), 1, 5, C.byref(best), ent, -1, C.byref(cnt)),
             (C.byref(c), 1, 5, C.byref(best), ent, 4, None)]
    for As, nsys, upd, b, e, cap, n in cases:
        assert L.plss_tune(As, nsys, None, upd, b, e, cap, n) == plss.ERR_INVALID


def test_binding_marshals_names_and_vectors(L):
    """The binding only translates: enum names to the header's values, host
    vectors to contiguous float64 of the stated length (else ValueError)."""
    o = plss.make_opts(sketch="identity", precision="fp32", layout="csr", schedule="small", tile_shift=-1,
                       tol=1e-6)
    assert (o.sketch, o.precision, o.layout, o.schedule, o.tile_shift, o.tol) == (1, 1, 1, 2, -1, 1e-6)
    assert o.inner_tol == 1e-4 and o.maxit == -1                 # untouched fields keep their defaults
    v = plss._vec_in([1, 2, 3], 3, "b", False)
    assert v.dtype == np.float64 and v.flags.c_contiguous and list(v) == [1.0, 2.0, 3.0]
    with pytest.raises(ValueError):
        plss._vec_in(np.zeros(4), 3, "b", False)
    r = plss.Result(status=-4, iters=7, relres_rec=0.5, relres_true=0.25, seconds=1.0).as_dict()
    assert r["status"] == "breakdown" and r["code"] == -4 and r["iters"] == 7


def test_server_rejects_bad_arguments(L):
    """Server entry points refuse bad arguments before touching a device."""
    so = plss.ServerOpts()
    L.plss_server_opts_default(C.byref(so))
    assert (so.max_slots, so.max_queue, so.bodies_per_poll, so.layout) == (64, 4096, 8, plss.LAYOUT["csr"])
    h = C.c_void_p()
    assert L.plss_server_create(C.byref(so), None) == plss.ERR_INVALID
    for field, bad in (("max_slots", 0), ("max_queue", 0), ("bodies_per_poll", 0), ("precision", 9),
                       ("layout", 4)):
        o = plss.ServerOpts()
        L.plss_server_opts_default(C.byref(o))
        setattr(o, field, bad)
        assert L.plss_server_create(C.byref(o), C.byref(h)) == plss.ERR_INVALID, field
        assert not h.value
    t = C.c_uint64()
    res = plss.Result()
    assert L.plss_submit(None, None, None, None, None, C.byref(t)) == plss.ERR_INVALID
    assert L.plss_poll(None, 1, None, C.byref(res)) == plss.ERR_INVALID
    assert L.plss_server_stats(None, None, None, None, None) == plss.ERR_INVALID
    L.plss_server_destroy(None)                                   # a no-op


def test_context_calls_refuse_a_null_context(L):
    assert L.plss_solve_rhs(None, 1, None, None, None, None, None) == plss.ERR_INVALID
    assert L.plss_solve_batched(None, None, None, None, None, None) == plss.ERR_INVALID
    assert L.plss_spmv(None, 0, None, None, None) == plss.ERR_INVALID
    assert L.plss_kernel_times(None, None, None, 0) == plss.ERR_INVALID
    assert L.plss_ctx_info(None, None, None, None, None) == plss.ERR_INVALID
    assert L.plss_ctx_layout(None, None) == plss.ERR_INVALID
    assert L.plss_gather_bound(None, 0, 1, None, None) == plss.ERR_INVALID
    assert L.plss_resume(None, None, None, None) == plss.ERR_INVALID
    assert L.plss_state_bytes(None) == -1
    assert "NULL" in L.plss_last_error().decode()
    buf = (C.c_ubyte * 64)()
    assert L.plss_state_save(None, buf, 64) == plss.ERR_INVALID
    assert L.plss_state_load(None, buf, 64) == plss.ERR_INVALID
    L.plss_destroy(None)                                          # a no-op


def test_noalloc_residual_checks_sizes_first(L):
    """plss_residual_noalloc refuses negative sizes, more rows than its static
    scratch covers, and NULL arrays, with nothing launched."""
    n2 = (C.c_double * 1)()
    rp = np.zeros(2, dtype=np.int64)
    f = L.plss_residual_noalloc
    assert f(-1, 1, 0, rp.ctypes.data, None, None, None, None, None, n2, None) == plss.ERR_INVALID
    assert f(4_194_305, 1, 0, rp.ctypes.data, None, None, None, None, None, n2, None) == plss.ERR_INVALID
    assert "4194304" in L.plss_last_error().decode()
    assert f(1, 1, 0, None, None, None, None, None, None, n2, None) == plss.ERR_INVALID
    assert f(1, 1, 0, rp.ctypes.data, None, None, None, None, None, None, None) == plss.ERR_INVALID
    assert f(1, 1, 1, rp.ctypes.data, None, None, None, None, None, n2, None) == plss.ERR_INVALID


def test_trace_ranges_are_compiled_in(L):
    """The host phases carry NVTX range names for timeline profilers."""
    so = open(pbuild.build(), "rb").read()
    for name in (b"plss: create context", b"plss: solve (residual sketch)", b"plss: resume (residual sketch)",
                 b"plss: solve (identity sketch)", b"plss: solve (general sketch)",
                 b"plss: solve (many right-hand sides)", b"plss server: scheduling round", b"plss: tune"):
        assert name in so, name
