"""Python binding of libplss (C ABI in include/plss.h): argument marshalling only.

Every step of a solve runs in the CUDA library. Vectors may be numpy arrays
(host memory) or torch CUDA tensors (device memory, run on torch's current
stream). There is no CPU fallback: if libplss.so cannot be loaded, lib()
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libplss.so")

OK, NOT_CONVERGED, PENDING = 0, 1, 2
ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_BUSY, ERR_NOT_FOUND = \
    -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "converged", 1: "not_converged", 2: "pending", -1: "invalid", -2: "nomem",
                -3: "cuda", -4: "breakdown", -5: "timeout", -6: "busy", -7: "not_found"}
SKETCH = {"residual": 0, "identity": 1, "general": 2}
PRECISION = {"fp64": 0, "fp32": 1}
LAYOUT = {"auto": 0, "csr": 1}
SCHEDULE = {"auto": 0, "grid": 1, "small": 2, "coop": 3}
REFINE = {"restart": 0, "replace": 1}

#: every symbol declared in include/plss.h
EXPORTS = ["plss_opts_default", "plss_create", "plss_create_batched", "plss_destroy",
           "plss_ctx_info", "plss_ctx_layout", "plss_solve", "plss_solve_batched", "plss_solve_rhs", "plss_spmv",
           "plss_kernel_times", "plss_residual_noalloc", "plss_last_error", "plss_server_opts_default",
           "plss_server_create", "plss_submit", "plss_poll", "plss_server_stats", "plss_server_destroy",
           "plss_tune", "plss_gather_bound", "plss_resume", "plss_state_bytes", "plss_state_save",
           "plss_state_load"]


class Csr(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p),
                ("val_f32", C.c_int32), ("on_device", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("sketch", C.c_int32), ("precision", C.c_int32), ("w_mode", C.c_int32),
                ("stop_on_true", C.c_int32), ("tol", C.c_double), ("maxit", C.c_int64),
                ("refine_period", C.c_int64), ("kacz_hist", C.c_int64), ("seed", C.c_uint64),
                ("io_device", C.c_int32), ("symmetric", C.c_int32), ("stream", C.c_void_p),
                ("hist", C.c_void_p), ("hist_cap", C.c_int64), ("profile", C.c_int32),
                ("layout", C.c_int32), ("inner_tol", C.c_double), ("schedule", C.c_int32),
                ("tile_shift", C.c_int32), ("refine_mode", C.c_int32)]


class TuneEntry(C.Structure):
    _fields_ = [("layout", C.c_int32), ("tile_shift", C.c_int32), ("schedule", C.c_int32),
                ("status", C.c_int32), ("us_per_update", C.c_double)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("reserved", C.c_int32), ("iters", C.c_int64),
                ("relres_rec", C.c_double), ("relres_true", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return dict(status=STATUS_NAMES.get(self.status, self.status), code=int(self.status),
                    iters=int(self.iters), relres_rec=float(self.relres_rec),
                    relres_true=float(self.relres_true), seconds=float(self.seconds))


class ServerOpts(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("max_queue", C.c_int32),
                ("hbm_budget_bytes", C.c_int64), ("precision", C.c_int32),
                ("bodies_per_poll", C.c_int32), ("layout", C.c_int32), ("reserved", C.c_int32)]


_lib = None
_lock = threading.Lock()


def lib() -> C.CDLL:
    """Loads libplss.so (built by paper_2207_07615_gb300.build). Raises when
    the library is missing: there is no fallback path."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libplss.so not found at {LIB_PATH}; run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'` first")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
            L.plss_opts_default.argtypes = [vp]
            L.plss_opts_default.restype = None
            L.plss_create.argtypes = [vp, vp, vp]
            L.plss_create_batched.argtypes = [vp, i32, vp, vp]
            L.plss_destroy.argtypes = [vp]
            L.plss_destroy.restype = None
            L.plss_ctx_info.argtypes = [vp, vp, vp, vp, vp]
            L.plss_ctx_layout.argtypes = [vp, vp]
            L.plss_solve.argtypes = [vp, vp, vp, vp, vp, vp]
            L.plss_solve_batched.argtypes = [vp, vp, vp, vp, vp, vp]
            L.plss_solve_rhs.argtypes = [vp, i32, vp, vp, vp, vp, vp]
            L.plss_spmv.argtypes = [vp, i32, vp, vp, vp]
            L.plss_kernel_times.argtypes = [vp, vp, vp, i32]
            L.plss_residual_noalloc.argtypes = [i64, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp]
            L.plss_residual_noalloc.restype = C.c_int32
            L.plss_last_error.argtypes = []
            L.plss_last_error.restype = C.c_char_p
            L.plss_server_opts_default.argtypes = [vp]
            L.plss_server_opts_default.restype = None
            L.plss_server_create.argtypes = [vp, vp]
            L.plss_submit.argtypes = [vp, vp, vp, vp, vp, vp]
            L.plss_poll.argtypes = [vp, C.c_uint64, vp, vp]
            L.plss_server_stats.argtypes = [vp, vp, vp, vp, vp]
            L.plss_server_destroy.argtypes = [vp]
            L.plss_server_destroy.restype = None
            L.plss_tune.argtypes = [vp, i32, vp, i32, vp, vp, i32, vp]
            L.plss_gather_bound.argtypes = [vp, i32, i32, vp, vp]
            L.plss_resume.argtypes = [vp, vp, vp, vp]
            L.plss_state_bytes.argtypes = [vp]
            L.plss_state_bytes.restype = i64
            L.plss_state_save.argtypes = [vp, vp, i64]
            L.plss_state_load.argtypes = [vp, vp, i64]
            for name in ("plss_create", "plss_create_batched", "plss_ctx_info", "plss_ctx_layout",
                         "plss_solve",
                         "plss_kernel_times",
                         "plss_solve_batched", "plss_solve_rhs", "plss_spmv",
                         "plss_server_create", "plss_submit", "plss_poll", "plss_server_stats", "plss_tune",
                         "plss_gather_bound", "plss_resume", "plss_state_save", "plss_state_load"):
                getattr(L, name).restype = C.c_int32
            _lib = L
    return _lib


class PlssError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(code, allowed=(OK, NOT_CONVERGED, ERR_BREAKDOWN)):
    if code not in allowed:
        raise PlssError(code, lib().plss_last_error().decode(errors="replace"))
    return code


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _stream_of(a):
    if a is not None and _is_torch(a) and a.is_cuda:
        import torch
        return C.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return None


def _vec_in(a, length, name, dev):
    if a is None:
        return None
    if _is_torch(a):
        import torch
        if not dev:
            raise ValueError(f"{name}: mix of torch and numpy inputs")
        if not a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != length:
            raise ValueError(f"{name}: need a contiguous CUDA float64 tensor of {length} entries")
        return a
    if dev:
        raise ValueError(f"{name}: mix of torch and numpy inputs")
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != length:
        raise ValueError(f"{name}: need {length} entries, got {a.size}")
    return a


def _new_like(ref, length):
    if _is_torch(ref):
        import torch
        return torch.empty(length, dtype=torch.float64, device=ref.device)
    return np.empty(length, dtype=np.float64)


def make_opts(**kw) -> Opts:
    o = Opts()
    lib().plss_opts_default(C.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "sketch" and isinstance(v, str):
            v = SKETCH[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k == "layout" and isinstance(v, str):
            v = LAYOUT[v]
        if k == "schedule" and isinstance(v, str):
            v = SCHEDULE[v]
        if k == "refine_mode" and isinstance(v, str):
            v = REFINE[v]
        setattr(o, k, v)
    return o


class _CsrHold:
    """Keeps the arrays of one CSR alive while the C structure is in use."""

    def __init__(self, A):
        if _is_torch(A.row_ptr):
            import torch
            self.keep = (A.row_ptr.to(torch.int64).contiguous(), A.col_idx.to(torch.int32).contiguous(),
                         A.val.contiguous())
            f32 = A.val.dtype == torch.float32
            dev = int(A.row_ptr.is_cuda)
        else:
            f32 = A.val.dtype == np.float32
            self.keep = (np.ascontiguousarray(A.row_ptr, dtype=np.int64),
                         np.ascontiguousarray(A.col_idx, dtype=np.int32),
                         np.ascontiguousarray(A.val, dtype=np.float32 if f32 else np.float64))
            dev = 0
        rp, ci, v = self.keep
        self.c = Csr(int(A.m), int(A.n), int(A.nnz), _ptr(rp), _ptr(ci), _ptr(v), int(f32), dev)


_LAYOUT_NAMES = {v: k for k, v in LAYOUT.items()}
_SCHEDULE_NAMES = {v: k for k, v in SCHEDULE.items()}


def tune(A, updates=20, precision="fp64", symmetric=False, w_mode=0, stream=None):
    """plss_tune: measures the candidate sweep plans of A (a CSR, or a list of
    them for a batched context) and returns (best, table). `best` holds the
    Context and solve keywords of the fastest plan ({"layout", "tile_shift"}
    for Context, {"schedule"} for solve); `table` lists every candidate with
    its wall time per update in microseconds."""
    L = lib()
    As = list(A) if isinstance(A, (list, tuple)) else [A]
    holds = [_CsrHold(a) for a in As]
    arr = (Csr * len(holds))(*[h.c for h in holds])
    o = make_opts(precision=precision, symmetric=int(bool(symmetric)), w_mode=w_mode, stream=stream)
    best = Opts()
    cap = 32
    ent = (TuneEntry * cap)()
    cnt = C.c_int32()
    _check(L.plss_tune(arr, len(holds), C.byref(o), int(updates), C.byref(best), ent, cap, C.byref(cnt)), (OK,))
    table = [dict(layout=_LAYOUT_NAMES[e.layout], tile_shift=int(e.tile_shift),
                  schedule=_SCHEDULE_NAMES[e.schedule],
                  status="ok" if e.status == OK else STATUS_NAMES.get(e.status, e.status),
                  us_per_update=float(e.us_per_update)) for e in ent[:min(cap, cnt.value)]]
    return (dict(layout=_LAYOUT_NAMES[best.layout], tile_shift=int(best.tile_shift),
                 schedule=_SCHEDULE_NAMES[best.schedule]), table)


class Context:
    """A matrix (or a batch of independent matrices) resident on the GPU."""

    def __init__(self, A, precision="fp64", symmetric=False, layout="auto", tile_shift=0):
        L = lib()
        self._h = C.c_void_p()
        o = make_opts(precision=precision, symmetric=int(bool(symmetric)), layout=layout, tile_shift=tile_shift)
        if isinstance(A, (list, tuple)):
            holds = [_CsrHold(a) for a in A]
            arr = (Csr * len(holds))(*[h.c for h in holds])
            _check(L.plss_create_batched(arr, len(holds), C.byref(o), C.byref(self._h)), (OK,))
            self.shapes = [(int(a.m), int(a.n)) for a in A]
        else:
            h = _CsrHold(A)
            _check(L.plss_create(C.byref(h.c), C.byref(o), C.byref(self._h)), (OK,))
            self.shapes = [(int(A.m), int(A.n))]
        self.nsys = len(self.shapes)
        self.m = sum(s[0] for s in self.shapes)
        self.n = sum(s[1] for s in self.shapes)

    def layout(self):
        """Tile schedule: row/column tiles, how many are sliced, and the
        elements (nonzeros plus padding) of the sliced copies."""
        out = (C.c_int64 * 6)()
        _check(lib().plss_ctx_layout(self._h, out), (OK,))
        keys = ("row_tiles", "row_sliced", "col_tiles", "col_sliced", "row_sliced_elems",
                "col_sliced_elems")
        return dict(zip(keys, [int(v) for v in out]))

    def close(self):
        if self._h:
            lib().plss_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, b, x0=None, *, hist=0, **kw):
        """Solves A x = b. Returns (x, result) or (x, result, hist[k, 5])."""
        m, n = self.shapes[0]
        dev = _is_torch(b)
        b = _vec_in(b, m, "b", dev)
        x0 = _vec_in(x0, n, "x0", dev)
        x = _new_like(b, n)
        H = np.zeros((int(hist), 5)) if hist else None
        o = make_opts(io_device=int(dev), stream=_stream_of(b), **kw)
        if H is not None:
            o.hist = H.ctypes.data_as(C.c_void_p).value
            o.hist_cap = int(hist)
        res = Result()
        _check(lib().plss_solve(self._h, _ptr(b), _ptr(x0), _ptr(x), C.byref(o), C.byref(res)))
        r = res.as_dict()
        if H is not None:
            return x, r, H[:min(int(hist), r["iters"])]
        return x, r

    def solve_batched(self, bs, x0s=None, **kw):
        """Solves every system of a batched context; returns (xs, results)."""
        dev = _is_torch(bs[0])
        bl = [_vec_in(b, s[0], f"b[{i}]", dev) for i, (b, s) in enumerate(zip(bs, self.shapes))]
        xl = [None] * self.nsys if x0s is None else \
            [_vec_in(x, s[1], f"x0[{i}]", dev) for i, (x, s) in enumerate(zip(x0s, self.shapes))]
        outs = [_new_like(bl[0], s[1]) for s in self.shapes]
        P = C.c_void_p * self.nsys
        bp = P(*[_ptr(b) for b in bl])
        xp = P(*[_ptr(x) for x in xl])
        op = P(*[_ptr(x) for x in outs])
        res = (Result * self.nsys)()
        o = make_opts(io_device=int(dev), stream=_stream_of(bl[0]), **kw)
        _check(lib().plss_solve_batched(self._h, bp, xp, op, C.byref(o), res))
        return outs, [r.as_dict() for r in res]

    def resume(self, *, hist=0, device=False, **kw):
        """Goes on with the residual-sketch solve the update cap stopped (or a
        loaded state) up to maxit updates in total; returns (xs, results),
        one entry per system, or (xs, results, hist) with hist=k (system 0's
        rows from the update count it resumed at)."""
        outs = []
        for (m, n) in self.shapes:
            if device:
                import torch
                outs.append(torch.empty(n, dtype=torch.float64, device="cuda"))
            else:
                outs.append(np.empty(n))
        P = C.c_void_p * self.nsys
        op = P(*[_ptr(x) for x in outs])
        H = np.zeros((int(hist), 5)) if hist else None
        o = make_opts(io_device=int(device), stream=_stream_of(outs[0]) if device else None, **kw)
        if H is not None:
            o.hist = H.ctypes.data_as(C.c_void_p).value
            o.hist_cap = int(hist)
        res = (Result * self.nsys)()
        _check(lib().plss_resume(self._h, op, C.byref(o), res))
        rs = [r.as_dict() for r in res]
        if H is not None:
            return outs, rs, H
        return outs, rs

    def state_save(self):
        """The context's residual-sketch state as bytes (plss_state_save)."""
        nb = int(lib().plss_state_bytes(self._h))
        if nb < 0:
            raise PlssError(ERR_INVALID, lib().plss_last_error().decode())
        buf = (C.c_ubyte * nb)()
        _check(lib().plss_state_save(self._h, buf, nb), (OK,))
        return bytes(buf)

    def state_load(self, data):
        """Loads a state saved from a context of the same shape (plss_state_load)."""
        buf = (C.c_ubyte * len(data)).from_buffer_copy(data)
        _check(lib().plss_state_load(self._h, buf, len(data)), (OK,))

    def solve_rhs(self, B, X0=None, **kw):
        """Many right-hand sides: B (m x k), X0 (n x k) row-major; returns (X, results)."""
        m, n = self.shapes[0]
        dev = _is_torch(B)
        k = int(B.shape[1])
        Bf = _vec_in(B.reshape(-1), m * k, "B", dev)
        X0f = None if X0 is None else _vec_in(X0.reshape(-1), n * k, "X0", dev)
        X = _new_like(Bf, n * k)
        res = (Result * k)()
        o = make_opts(io_device=int(dev), stream=_stream_of(Bf), **kw)
        _check(lib().plss_solve_rhs(self._h, k, _ptr(Bf), _ptr(X0f), _ptr(X), C.byref(o), res))
        return X.reshape(n, k), [r.as_dict() for r in res]

    def kernel_times(self, reset=True):
        """(ms[3], launches[3]) of row sweep, column sweep, update over the
        profiled solves since the last reset."""
        ms = (C.c_double * 3)()
        n = (C.c_int64 * 4)()
        _check(lib().plss_kernel_times(self._h, ms, n, int(bool(reset))), (OK,))
        names = ("row_sweep", "col_sweep", "update")
        out = {k: (float(ms[i]), int(n[i])) for i, k in enumerate(names)}
        out["all_launches"] = int(n[3])
        return out

    def gather_bound(self, side, reps=5):
        """Device time (us: median, min) of gathering the sweep's vector along
        the sweep's own index stream and nothing else (side 0 = rows, A p;
        1 = columns, A^T r): the floor set by the sweep's random gathers."""
        med, mn = C.c_double(), C.c_double()
        _check(lib().plss_gather_bound(self._h, int(side), int(reps), C.byref(med), C.byref(mn)), (OK,))
        return med.value, mn.value

    def spmv(self, v, transpose=False, stream=None):
        m, n = self.shapes[0]
        lin, lout = (m, n) if transpose else (n, m)
        dev = _is_torch(v)
        v = _vec_in(v, lin, "v", dev)
        out = _new_like(v, lout)
        o = make_opts(io_device=int(dev), stream=_stream_of(v))
        _check(lib().plss_spmv(self._h, int(bool(transpose)), _ptr(v), _ptr(out), C.byref(o)), (OK,))
        return out


class Server:
    """Continuous-batching solve server (plss_server_*)."""

    def __init__(self, max_slots=64, max_queue=4096, hbm_budget_bytes=0, precision="fp64",
                 bodies_per_poll=8, layout="csr"):
        L = lib()
        so = ServerOpts()
        L.plss_server_opts_default(C.byref(so))
        so.max_slots, so.max_queue = int(max_slots), int(max_queue)
        so.bodies_per_poll = int(bodies_per_poll)
        so.hbm_budget_bytes = int(hbm_budget_bytes)
        so.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        so.layout = LAYOUT[layout] if isinstance(layout, str) else int(layout)
        self._h = C.c_void_p()
        _check(L.plss_server_create(C.byref(so), C.byref(self._h)), (OK,))
        self._n = {}

    def submit(self, A, b, x0=None, **kw):
        h = _CsrHold(A)
        b = np.ascontiguousarray(b, dtype=np.float64)
        x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        o = make_opts(**kw)
        t = C.c_uint64()
        code = lib().plss_submit(self._h, C.byref(h.c), _ptr(b), _ptr(x0), C.byref(o), C.byref(t))
        _check(code, (OK, ERR_BUSY))
        if code == ERR_BUSY:
            return None
        self._n[t.value] = int(A.n)
        return t.value

    def poll(self, ticket):
        """Returns None while pending, else (x, result)."""
        n = self._n.get(ticket)
        x = np.empty(n if n is not None else 0)
        res = Result()
        code = lib().plss_poll(self._h, C.c_uint64(ticket), _ptr(x) if n else None, C.byref(res))
        if code == PENDING:
            return None
        _check(code, (OK, NOT_CONVERGED, ERR_BREAKDOWN))
        self._n.pop(ticket, None)
        return x, res.as_dict()

    def stats(self):
        v = [C.c_int64() for _ in range(4)]
        _check(lib().plss_server_stats(self._h, *[C.byref(a) for a in v]), (OK,))
        return dict(completed=v[0].value, queued=v[1].value, running=v[2].value,
                    bytes_in_use=v[3].value)

    def close(self):
        if self._h:
            lib().plss_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
