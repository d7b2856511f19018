"""CPU oracle for PLSS (arXiv 2207.07615): plain FP64 C, called through ctypes.

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU baseline are the only callers. The CUDA library never loads
or calls anything here, and this package never imports the CUDA library.

Functions follow the paper step by step (see plss_oracle.c):
  residual()    Algorithm 1 / Theorem 4.1, optional diagonal W (Sec. 4.1)
  kaczmarz()    identity sketch, eq:pkKacz (Sec. 7)
  general()     general sketch of random sign columns, Theorem 2.1 and
                Corollary 2.2 (Sec. 2.4); sketch_entry() gives its columns
  spmv(), spmvt(), colweights(), permutation()  plain building blocks
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "plss_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libplss_oracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "libplss_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

STATUS = {0: "converged", 1: "not_converged", -4: "breakdown", -1: "invalid", -2: "nomem"}


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (plain -O2, no FMA contraction), and the
    same source with -fopenmp as a second library used only to time it on
    all host cores."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    for lib, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", *extra, "-fPIC",
                   "-shared", _SRC, "-o", tmp, "-lm"]
            if lib == _LIB:
                subprocess.check_call(cmd)
            elif subprocess.call(cmd, stderr=subprocess.DEVNULL) != 0:
                continue        # no OpenMP here: only the timing variant is missing
            os.replace(tmp, lib)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            i64, i32, d, vp, u64 = C.c_int64, C.c_int, C.c_double, C.c_void_p, C.c_uint64
            lib.plss_oracle_residual.restype = i32
            lib.plss_oracle_residual.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp, d, i64, i32, i64,
                                                 d, i32, i32, i32, vp, vp, vp, vp, i64, vp, vp, vp, vp,
                                                 vp]
            lib.plss_oracle_kaczmarz.restype = i32
            lib.plss_oracle_kaczmarz.argtypes = [i64, i64, vp, vp, vp, vp, vp, d, i64, i64, u64,
                                                 i32, vp, vp, vp, vp]
            lib.plss_oracle_spmv.restype = None
            lib.plss_oracle_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
            lib.plss_oracle_spmvt.restype = i32
            lib.plss_oracle_spmvt.argtypes = [i64, i64, vp, vp, vp, vp, vp]
            lib.plss_oracle_colweights.restype = None
            lib.plss_oracle_colweights.argtypes = [i64, i64, vp, vp, vp, i32, vp]
            lib.plss_oracle_general.restype = i32
            lib.plss_oracle_general.argtypes = [i64, i64, vp, vp, vp, vp, vp, d, i64, i64, u64, i32,
                                                vp, vp, vp, vp, i64, vp]
            lib.plss_oracle_sketch_entry.restype = d
            lib.plss_oracle_sketch_entry.argtypes = [u64, i64, i64, i64]
            lib.plss_oracle_permutation.restype = None
            lib.plss_oracle_permutation.argtypes = [vp, i64, vp]
            _lib = lib
    return _lib


def _load_omp():
    """The OpenMP build (timing only); RuntimeError when it could not be built."""
    global _lib_omp
    _load()
    if not os.path.exists(_LIB_OMP):
        raise RuntimeError("the OpenMP build of the oracle is not available (gcc -fopenmp failed)")
    with _lock:
        if _lib_omp is None:
            lib = C.CDLL(_LIB_OMP)
            lib.plss_oracle_residual.restype = _lib.plss_oracle_residual.restype
            lib.plss_oracle_residual.argtypes = _lib.plss_oracle_residual.argtypes
            _lib_omp = lib
    return _lib_omp


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _csr(A):
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(A.val, dtype=np.float64)
    return rp, ci, v


def _vec(a, length, name):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (length,):
        raise ValueError(f"{name} must have shape ({length},), got {a.shape}")
    return a


def spmv(A, v):
    lib = _load()
    rp, ci, val = _csr(A)
    v = _vec(v, A.n, "v")
    out = np.empty(A.m)
    lib.plss_oracle_spmv(A.m, _p(rp), _p(ci), _p(val), _p(v), _p(out))
    return out


def spmvt(A, r):
    lib = _load()
    rp, ci, val = _csr(A)
    r = _vec(r, A.m, "r")
    out = np.empty(A.n)
    if lib.plss_oracle_spmvt(A.m, A.n, _p(rp), _p(ci), _p(val), _p(r), _p(out)) != 0:
        raise MemoryError("oracle spmvt")
    return out


def colweights(A, mode: int = 1):
    lib = _load()
    rp, ci, val = _csr(A)
    w = np.empty(A.n)
    lib.plss_oracle_colweights(A.m, A.n, _p(rp), _p(ci), _p(val), int(mode), _p(w))
    return w


def permutation(state: int, m: int):
    """One Fisher-Yates permutation of 0..m-1 from a SplitMix64 stream.
    Returns (perm, new_state)."""
    lib = _load()
    st = np.array([state], dtype=np.uint64)
    perm = np.empty(m, dtype=np.int32)
    lib.plss_oracle_permutation(_p(st), m, _p(perm))
    return perm, int(st[0])


def residual(A, b, x0=None, w=None, tol=1e-10, maxit=None, prec=0, refine=0, inner_tol=0.0,
             stop_on_true=False, gamma_form=0, hist=0, plant=0, threads=False, replace=False):
    """PLSS residual sketch (Algorithm 1). Returns a dict with x, iters,
    status, relres_rec, relres_true and, when hist > 0, the per-update
    history: s[k] = (rho_k, phi_{k+1}, beta_k, gamma_k, theta_{k+1}),
    x[k] = x_{k+1}, p[k] = p_{k+1}, y[k] = A^T r_k, r[k] = r_k.
    gamma_form=1 (same as plant=1) and plant=2/3 plant a defect for the
    tests that show the pins reject it (see plss_oracle.c). threads=True
    runs the OpenMP build on all host cores (for timing). replace=True:
    refinement refreshes replace the residual instead of restarting."""
    lib = _load_omp() if threads else _load()
    rp, ci, val = _csr(A)
    b = _vec(b, A.m, "b")
    x0 = _vec(x0, A.n, "x0")
    w = _vec(w, A.n, "w")
    if maxit is None:
        maxit = A.n
    x = np.empty(A.n)
    it = np.zeros(1, dtype=np.int64)
    rr = np.zeros(1)
    rt = np.zeros(1)
    H = int(hist)
    hs = np.zeros((H, 5)) if H else None
    hx = np.zeros((H, A.n)) if H else None
    hp = np.zeros((H, A.n)) if H else None
    hy = np.zeros((H, A.n)) if H else None
    hr = np.zeros((H + 1, A.m)) if H else None
    st = lib.plss_oracle_residual(A.m, A.n, _p(rp), _p(ci), _p(val), _p(b), _p(x0), _p(w),
                                  float(tol), int(maxit), int(prec), int(refine), float(inner_tol),
                                  int(bool(stop_on_true)), 1 if gamma_form == 1 else int(plant),
                                  int(bool(replace)), _p(x), _p(it),
                                  _p(rr), _p(rt), H, _p(hs), _p(hx), _p(hp), _p(hy), _p(hr))
    if st == -2:
        raise MemoryError("oracle residual")
    out = dict(x=x, iters=int(it[0]), status=STATUS.get(st, st), relres_rec=float(rr[0]),
               relres_true=float(rt[0]))
    if H:
        k = min(H, out["iters"])
        out.update(hist_s=hs[:k], hist_x=hx[:k], hist_p=hp[:k], hist_y=hy[:k],
                   hist_r=hr[:k + 1])
    return out


def kaczmarz(A, b, x0=None, tol=1e-8, maxit=None, K=0, seed=0, plant=0):
    """PLSS Kaczmarz (identity sketch, eq:pkKacz) with history cap K.
    plant=1/2/3 plants a wrong window reset (late, early, never) for the
    tests that show the pins reject it (see plss_oracle.c)."""
    lib = _load()
    rp, ci, val = _csr(A)
    b = _vec(b, A.m, "b")
    x0 = _vec(x0, A.n, "x0")
    if maxit is None:
        maxit = 100 * A.m
    x = np.empty(A.n)
    it = np.zeros(1, dtype=np.int64)
    sk = np.zeros(1, dtype=np.int64)
    rt = np.zeros(1)
    st = lib.plss_oracle_kaczmarz(A.m, A.n, _p(rp), _p(ci), _p(val), _p(b), _p(x0), float(tol),
                                  int(maxit), int(K), int(seed) & (2**64 - 1), int(plant),
                                  _p(x), _p(it),
                                  _p(sk), _p(rt))
    if st == -2:
        raise MemoryError("oracle kaczmarz")
    return dict(x=x, iters=int(it[0]), skipped=int(sk[0]), status=STATUS.get(st, st),
                relres_true=float(rt[0]))


def sketch_entry(seed: int, m: int, k: int, i: int) -> float:
    """Entry i of general-sketch column k (0-based): +1 or -1."""
    return float(_load().plss_oracle_sketch_entry(int(seed) & (2**64 - 1), int(m), int(k), int(i)))


def general(A, b, x0=None, tol=1e-8, maxit=None, K=0, seed=0, hist=0, plant=0):
    """PLSS with a general sketch of random sign columns (Theorem 2.1,
    Corollary 2.2), history of at most K columns. hist > 0 returns the
    iterate after each of the first `hist` columns as hist_x."""
    lib = _load()
    rp, ci, val = _csr(A)
    b = _vec(b, A.m, "b")
    x0 = _vec(x0, A.n, "x0")
    if maxit is None:
        maxit = A.n
    x = np.empty(A.n)
    it = np.zeros(1, dtype=np.int64)
    sk = np.zeros(1, dtype=np.int64)
    rt = np.zeros(1)
    H = int(hist)
    hx = np.zeros((H, A.n)) if H else None
    st = lib.plss_oracle_general(A.m, A.n, _p(rp), _p(ci), _p(val), _p(b), _p(x0), float(tol),
                                 int(maxit), int(K), int(seed) & (2**64 - 1), int(plant),
                                 _p(x), _p(it), _p(sk), _p(rt), H, _p(hx))
    if st == -2:
        raise MemoryError("oracle general")
    out = dict(x=x, iters=int(it[0]), skipped=int(sk[0]), status=STATUS.get(st, st),
               relres_true=float(rt[0]))
    if H:
        out["hist_x"] = hx[:min(H, out["iters"])]
    return out
