"""Parity helpers: iterate-by-iterate comparison of a GPU trajectory with the
oracle's, with a tolerance calibrated by the recursion's own rounding
sensitivity.

The PLSS recursion (Theorem 4.1) is, like every Lanczos-type recursion,
sensitive to rounding once the residuals lose orthogonality: two correct
FP64 implementations that differ only in summation order follow the same
trajectory to ~1e-15 at first and drift apart later. That drift is measured
on the oracle alone, by running it again on b scaled by (1 + 2^-50) (and
x0 alike), which changes nothing but the rounding. An update k of the GPU
path passes when its difference from the oracle is below
max(1e-10, MARGIN * s_k), where s_k is the running maximum of that
oracle-only spread. While s_k stays at rounding level the bar is the plain
1e-10.

Every check also records the ratio of the GPU's deviation to that spread
(`RECORD`); the test session prints the largest ratio per test, which is
what MARGIN must cover.
"""
import numpy as np

import oracle

F = 1.0 + 2.0 ** -50
FLOOR = 1e-10
MARGIN = 400.0   # 11x the largest measured need (36.5, power-law rows, cluster schedule)

# (test id, what, max d/s over the updates whose bar the spread sets,
#  max d/FLOOR over the updates held to the plain 1e-10) -- filled by the
# checks, printed by conftest
RECORD = []
CURRENT = {"test": "?"}


def _ratio(d, s, tol):
    d = np.asarray(d, dtype=np.float64)
    s = np.maximum(np.asarray(s, dtype=np.float64), 1e-300)
    gov = tol > FLOOR
    g = float((d[gov] / s[gov]).max()) if np.any(gov) else 0.0
    f = float((d[~gov] / FLOOR).max()) if np.any(~gov) else 0.0
    return g, f


def rel_rows(g, r):
    g = np.asarray(g, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    den = np.abs(r)
    d = np.abs(g - r) / np.where(den > 0, den, 1.0)
    return d.max(axis=1) if d.ndim == 2 else d


def rel_vec_rows(G, R):
    G = np.asarray(G, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    return np.linalg.norm(G - R, axis=1) / np.maximum(np.linalg.norm(R, axis=1), 1e-300)


def reference(A, b, K, x0=None, w=None, prec=0, stop_on_true=False):
    """Oracle trajectory of K updates plus the per-update tolerances
    (scalars, x_k) from its own rounding sensitivity."""
    r1 = oracle.residual(A, b, x0=x0, w=w, tol=0.0, maxit=K, prec=prec,
                         stop_on_true=stop_on_true, hist=K)
    r2 = oracle.residual(A, b * F, x0=None if x0 is None else x0 * F, w=w, tol=0.0, maxit=K,
                         prec=prec, stop_on_true=stop_on_true, hist=K)
    h1 = r1["hist_s"]
    h2 = r2["hist_s"].copy()
    h2[:, [0, 1, 4]] /= F * F
    k = min(len(h1), len(h2))
    ss = np.maximum.accumulate(rel_rows(h2[:k], h1[:k]))
    sx = np.maximum.accumulate(rel_vec_rows(r2["hist_x"][:k] / F, r1["hist_x"][:k]))
    r1["tol_s"] = np.maximum(FLOOR, MARGIN * ss)
    r1["tol_x"] = np.maximum(FLOOR, MARGIN * sx)
    r1["spread_s"] = ss
    r1["spread_x"] = sx
    return r1


def check_scalars(hist_gpu, ref, min_strict=5):
    """Every update's scalars within the calibrated tolerance; returns the
    number of leading updates held to the plain 1e-10."""
    k = min(len(hist_gpu), len(ref["hist_s"]))
    d = rel_rows(hist_gpu[:k], ref["hist_s"][:k])
    tol = ref["tol_s"][:k]
    if k:
        RECORD.append((CURRENT["test"], "scalars", *_ratio(d, ref["spread_s"][:k], tol)))
    bad = np.nonzero(d > tol)[0]
    assert bad.size == 0, (f"update {bad[0] + 1}: scalar difference {d[bad[0]]:.3e} above "
                           f"tolerance {tol[bad[0]]:.3e}")
    strict = int(np.argmax(tol > FLOOR)) if np.any(tol > FLOOR) else k
    assert strict >= min(min_strict, k), f"only {strict} updates at the 1e-10 bar"
    return strict


def check_x(x_gpu, ref, k):
    """x_k (after k updates) against the oracle's within the calibrated tolerance."""
    d = float(np.linalg.norm(np.asarray(x_gpu) - ref["hist_x"][k - 1]) /
              np.linalg.norm(ref["hist_x"][k - 1]))
    RECORD.append((CURRENT["test"], f"x_{k}", *_ratio([d], [ref["spread_x"][k - 1]],
                                                     np.array([ref["tol_x"][k - 1]]))))
    assert d <= ref["tol_x"][k - 1], f"x_{k}: difference {d:.3e} above {ref['tol_x'][k - 1]:.3e}"
    return d
