"""Independent reference mathematics used to pin the oracle.

Nothing here shares code with the oracle or the CUDA library:
  pk_long()          eq:pkLong evaluated densely (pseudo-inverse), Sec. 1.3
  projection_run()   the generic iteration x_k = x_{k-1} + p_k, eq:xko, with
                     a residual sketch (eq:S) or an identity sketch (Sec. 7)
  craig()            Craig's method from Golub-Kahan bidiagonalization
                     (Paige & Saunders 1982, Sec. 7.2), as used by Thm 6.1
  limit_solution()   x0 + W A^T (A W A^T)^+ (b - A x0) (Thm 3.1, Cor. 3.3)
  kaczmarz_classic() x += (r_i/||a_i||^2) a_i
  window_projection_exact()
                     the identity sketch with a window of K rows, in exact
                     rational arithmetic: each step projects x onto the
                     intersection of the hyperplanes of the window's rows
                     (eq:pkLong with S = the window's identity columns)
  projection_run_restarted()
                     projection_run whose residual sketch starts afresh
                     (S = [b - A x]) whenever a given restart rule fires
"""
from __future__ import annotations

from fractions import Fraction
import os

import numpy as np


def pk_long(A, Wd, S, r):
    """p = W A^T S (S^T A W A^T S)^+ S^T r with W = diag(Wd)."""
    WAt = Wd[:, None] * A.T
    Y = WAt @ S
    M = S.T @ A @ Y
    return Y @ (np.linalg.pinv(M) @ (S.T @ r))


def projection_run(A, b, x0, Wd, K, sketch="residual", order=None):
    """Runs K steps of x_k = x_{k-1} + p_k with p_k from pk_long and the
    sketch S_k = [r_0 ... r_{k-1}] (residual) or [e_{i_1} ... e_{i_k}]
    (identity, rows taken from `order`). Returns (xs, ps, rs)."""
    m, n = A.shape
    x = np.array(x0, dtype=np.float64)
    cols = []
    xs, ps, rs = [], [], []
    for k in range(K):
        r = b - A @ x
        rs.append(r)
        if sketch == "residual":
            cols.append(r)
        else:
            e = np.zeros(m)
            e[order[k]] = 1.0
            cols.append(e)
        S = np.stack(cols, axis=1)
        p = pk_long(A, Wd, S, r)
        x = x + p
        xs.append(x.copy())
        ps.append(p)
    return xs, ps, rs


def craig(A, b, K, reorth=True):
    """Craig's method with x0 = 0: beta1 u1 = b, alpha1 v1 = A^T u1,
    beta_{k+1} u_{k+1} = A v_k - alpha_k u_k,
    alpha_{k+1} v_{k+1} = A^T u_{k+1} - beta_{k+1} v_k;
    zeta_1 = beta1/alpha1, zeta_k = -(beta_k/alpha_k) zeta_{k-1},
    x_k = x_{k-1} + zeta_k v_k. Full reorthogonalization keeps U, V
    orthonormal as in exact arithmetic. Returns the list of updates."""
    m, n = A.shape
    beta = np.linalg.norm(b)
    u = b / beta
    v = A.T @ u
    alpha = np.linalg.norm(v)
    v = v / alpha
    U, V = [u], [v]
    zeta = beta / alpha
    updates = [zeta * v]
    for _ in range(1, K):
        w = A @ v - alpha * u
        if reorth:
            for q in U:
                w -= (q @ w) * q
        beta = np.linalg.norm(w)
        u = w / beta
        z = A.T @ u - beta * v
        if reorth:
            for q in V:
                z -= (q @ z) * q
        alpha = np.linalg.norm(z)
        v = z / alpha
        U.append(u)
        V.append(v)
        zeta = -(beta / alpha) * zeta
        updates.append(zeta * v)
    return updates


def limit_solution(A, b, x0, Wd=None):
    """x0 + W A^T (A W A^T)^+ (b - A x0): the limit of updates in range(W A^T)."""
    if Wd is None:
        Wd = np.ones(A.shape[1])
    WAt = Wd[:, None] * A.T
    return x0 + WAt @ (np.linalg.pinv(A @ WAt) @ (b - A @ x0))


def kaczmarz_classic(A, b, x0, order):
    x = np.array(x0, dtype=np.float64)
    for i in order:
        a = A[i]
        x = x + ((b[i] - a @ x) / (a @ a)) * a
    return x


def _solve_exact(G, rhs):
    """Gauss-Jordan elimination over the rationals (G square, nonsingular)."""
    k = len(G)
    M = [list(G[i]) + [rhs[i]] for i in range(k)]
    for c in range(k):
        piv = next(i for i in range(c, k) if M[i][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for i in range(k):
            if i != c and M[i][c] != 0:
                f = M[i][c] / M[c][c]
                M[i] = [a - f * b for a, b in zip(M[i], M[c])]
    return [M[i][k] / M[i][i] for i in range(k)]


def window_projection_exact(D, b, order, K):
    """Identity sketch with a window of at most K rows, exactly: before a
    row is taken, a full window (K rows) is emptied; the row is added to the
    window and x is projected onto {x : a_j^T x = b_j for every row j of the
    window}, x <- x + A_S^T (A_S A_S^T)^{-1} (b_S - A_S x). K = 0 keeps no
    window (classical Kaczmarz). D, b hold integers or Fractions; the rows of
    each window must be linearly independent. Returns the list of iterates."""
    D = [[Fraction(v) for v in row] for row in np.asarray(D).tolist()]
    b = [Fraction(v) for v in np.asarray(b).tolist()]
    n = len(D[0])
    x = [Fraction(0)] * n
    win, out = [], []
    for i in order:
        if K > 0 and len(win) == K:
            win = []
        rows = win + [int(i)]
        AS = [D[j] for j in rows]
        G = [[sum(a * c for a, c in zip(ra, rc)) for rc in AS] for ra in AS]
        res = [b[j] - sum(a * c for a, c in zip(D[j], x)) for j in rows]
        z = _solve_exact(G, res)
        x = [x[t] + sum(z[q] * AS[q][t] for q in range(len(rows))) for t in range(n)]
        if K > 0:
            win = rows
        out.append(list(x))
    return out


def projection_run_restarted(A, b, x0, Wd, K, restart):
    """K steps of x_k = x_{k-1} + p_k, p_k from pk_long with the residual
    sketch S = [r_s, r_{s+1}, ..., r_{k-1}] that starts afresh at the last
    restart s. After update k the rule restart(rho_k, rho_s, k - s) (rho_k =
    ||b - A x_k||^2, exact to double rounding; rho_s at the last restart)
    says whether the sketch restarts from r_k. Returns (xs, rhos, restarts)
    with restarts = the update indices k after which the sketch restarted."""
    x = np.array(x0, dtype=np.float64)
    r = b - A @ x
    rho_s = float(r @ r)
    s = 0
    cols, xs, rhos, restarts = [], [], [], []
    for k in range(1, K + 1):
        cols.append(r)
        S = np.stack(cols, axis=1)
        x = x + pk_long(A, Wd, S, r)
        xs.append(x.copy())
        r = b - A @ x
        rho = float(r @ r)
        rhos.append(rho)
        if restart(rho, rho_s, k - s):
            restarts.append(k)
            cols, rho_s, s = [], rho, k
    return xs, rhos, restarts


def load_golden(name):
    """Reads `key = v1 v2 ...` lines (fractions allowed; `;` separates rows)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    out = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            rows = [[float(Fraction(t)) for t in row.split()] for row in v.split(";")]
            arr = np.array(rows)
            out[k] = arr[0] if arr.shape[0] == 1 else arr
            if out[k].shape == (1,):
                out[k] = float(out[k][0])
    return out
