"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks. None of them compares the oracle
with itself: the references are exact fractions worked by hand, eq:pkLong
evaluated densely, Craig's method from Golub-Kahan bidiagonalization,
LAPACK pseudo-inverses, scipy sparse products and classical Kaczmarz.
"""
import numpy as np
import pytest

import oracle
from paper_2207_07615_gb300 import synth
from tests import _pins


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


# ---------------------------------------------------------------- golden

def test_golden_2x2_residual_sketch():
    """Algorithm 1 on a 2x2 system, every scalar and iterate worked by hand."""
    g = _pins.load_golden("plss_2x2_hand.txt")
    A = synth.from_dense(g["A"])
    out = oracle.residual(A, g["b"], tol=0.0, maxit=2, hist=2)
    s = out["hist_s"]
    assert out["iters"] == 2
    np.testing.assert_allclose(s[0, 0], g["rho0"], rtol=1e-15)
    np.testing.assert_allclose(s[0, 1], g["phi1"], rtol=1e-15)
    np.testing.assert_allclose(s[0, 3], g["gamma0"], rtol=1e-15)
    np.testing.assert_allclose(s[0, 4], g["theta1"], rtol=1e-14)
    np.testing.assert_allclose(out["hist_x"][0], g["x1"], rtol=1e-15)
    np.testing.assert_allclose(out["hist_r"][1], g["r1"], rtol=1e-13)
    np.testing.assert_allclose(s[1, 0], g["rho1"], rtol=1e-13)
    np.testing.assert_allclose(s[1, 1], g["phi2"], rtol=1e-13)
    np.testing.assert_allclose(s[1, 2], g["beta1"], rtol=1e-11)
    np.testing.assert_allclose(s[1, 3], g["gamma1"], rtol=1e-11)
    np.testing.assert_allclose(out["hist_p"][1], g["p2"], rtol=1e-11)
    np.testing.assert_allclose(s[1, 4], g["theta2"], rtol=1e-11)
    np.testing.assert_allclose(out["hist_x"][1], g["x2"], rtol=1e-13)
    # r_1 orthogonal to r_0 (eq:orthSr)
    assert abs(out["hist_r"][1] @ out["hist_r"][0]) < 1e-14


def _seed_for_order(order, m=2):
    for seed in range(1000):
        perm, _ = oracle.permutation(seed, m)
        if tuple(perm) == tuple(order):
            return seed
    raise AssertionError("no seed")


@pytest.mark.parametrize("order", [(0, 1), (1, 0)])
def test_golden_2x2_kaczmarz(order):
    """eq:pkKacz on the 2x2 system worked by hand for both row orders; with
    no history (K=0) the second step is the classical Kaczmarz step."""
    g = _pins.load_golden("plss_2x2_hand.txt")
    A = synth.from_dense(g["A"])
    seed = _seed_for_order(order)
    tag = "kz%d%d" % order
    x1 = oracle.kaczmarz(A, g["b"], tol=0.0, maxit=1, K=4, seed=seed)["x"]
    x2 = oracle.kaczmarz(A, g["b"], tol=0.0, maxit=2, K=4, seed=seed)["x"]
    np.testing.assert_allclose(x1, g[tag + "_x1"], rtol=1e-15)
    np.testing.assert_allclose(x2, g[tag + "_x2"], rtol=1e-14)
    if order == (0, 1):
        x2k0 = oracle.kaczmarz(A, g["b"], tol=0.0, maxit=2, K=0, seed=seed)["x"]
        np.testing.assert_allclose(x2k0, g["kz01_k0_x2"], rtol=1e-14)


# ------------------------------------------------- tiny dense systems

def _cases():
    rng = synth.rng_for(7)
    out = []
    for (m, n, rank) in [(6, 6, 6), (8, 5, 5), (5, 8, 5), (8, 8, 5), (9, 7, 4)]:
        D = synth.dense_rank_deficient(rng, m, n, rank)
        xs = rng.standard_normal(n)
        out.append((D, D @ xs, rank))
    return out


CASES = _cases()


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("weighted", [False, True])
def test_recursion_equals_pklong(ci, weighted):
    """Theorem 4.1: the 1-step recursion reproduces eq:pkLong with the
    residual sketch S_k = [r_0 ... r_{k-1}] (eq:S) for every k <= rank."""
    D, b, rank = CASES[ci]
    A = synth.from_dense(D)
    rng = synth.rng_for(11 + ci)
    Wd = rng.uniform(0.5, 2.0, size=D.shape[1]) if weighted else np.ones(D.shape[1])
    x0 = rng.standard_normal(D.shape[1])
    out = oracle.residual(A, b, x0=x0, w=Wd if weighted else None, tol=0.0, maxit=rank, hist=rank)
    xs, ps, rs = _pins.projection_run(D, b, x0, Wd, rank, "residual")
    for k in range(rank):
        assert rel(out["hist_p"][k], ps[k]) < 1e-8, k
        assert rel(out["hist_x"][k], xs[k]) < 1e-10, k


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_orthogonality_identities(ci):
    """Residuals mutually orthogonal (Sec. 4), updates orthogonal
    (eq:orthogonal-updates), y_k^T p_{k-1} = -rho_{k-1} and y_k^T p_k = rho_{k-1}
    (proof of Theorem 4.1)."""
    D, b, rank = CASES[ci]
    A = synth.from_dense(D)
    out = oracle.residual(A, b, tol=0.0, maxit=rank, hist=rank)
    R = out["hist_r"][:-1]      # r_0 .. r_{k-1}; r_k is at rounding level
    P = out["hist_p"]
    Y = out["hist_y"]
    rho = out["hist_s"][:, 0]
    k = P.shape[0]
    Gr = R @ R.T
    Gp = P @ P.T
    sc_r = np.sqrt(np.outer(np.diag(Gr), np.diag(Gr)))
    sc_p = np.sqrt(np.outer(np.diag(Gp), np.diag(Gp)))
    off = ~np.eye(Gr.shape[0], dtype=bool)
    assert np.max(np.abs(Gr[off]) / sc_r[off]) < 1e-9
    off = ~np.eye(k, dtype=bool)
    if k > 1:
        assert np.max(np.abs(Gp[off]) / sc_p[off]) < 1e-9
    for j in range(k):
        np.testing.assert_allclose(Y[j] @ P[j], rho[j], rtol=1e-9)
        if j > 0:
            np.testing.assert_allclose(Y[j] @ P[j - 1], -rho[j], rtol=1e-9)


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_finite_termination_and_limit(ci):
    """Theorem 3.1 / Corollary 3.3: at most rank(A) updates reach the
    solution; the limit is x0 + A^T (A A^T)^+ (b - A x0) (updates lie in
    range(A^T)), checked against LAPACK's pseudo-inverse."""
    D, b, rank = CASES[ci]
    A = synth.from_dense(D)
    x0 = synth.rng_for(99).standard_normal(D.shape[1])
    out = oracle.residual(A, b, x0=x0, tol=1e-12, maxit=rank + 2)
    assert out["status"] == "converged"
    assert out["iters"] <= rank + 1
    assert out["relres_true"] < 1e-11
    assert rel(out["x"], _pins.limit_solution(D, b, x0)) < 1e-10


def test_weighted_limit():
    """Sec. 4.1: with W = diag(w) the updates lie in range(W A^T); the limit
    is x0 + W A^T (A W A^T)^+ (b - A x0)."""
    D, b, rank = CASES[3]
    A = synth.from_dense(D)
    rng = synth.rng_for(5)
    Wd = rng.uniform(0.3, 3.0, size=D.shape[1])
    x0 = rng.standard_normal(D.shape[1])
    out = oracle.residual(A, b, x0=x0, w=Wd, tol=1e-12, maxit=rank + 2)
    assert out["status"] == "converged"
    assert rel(out["x"], _pins.limit_solution(D, b, x0, Wd)) < 1e-10
    # and it differs from the unweighted limit (the pin would see a dropped W)
    assert rel(out["x"], _pins.limit_solution(D, b, x0)) > 1e-3


@pytest.mark.parametrize("ci", [0, 1, 2])
def test_craig_equivalence(ci):
    """Theorem 6.1: with W = I and x0 = 0 the PLSS updates equal Craig's."""
    D, b, rank = CASES[ci]
    A = synth.from_dense(D)
    out = oracle.residual(A, b, tol=0.0, maxit=rank, hist=rank)
    cu = _pins.craig(D, b, rank)
    for k in range(rank):
        assert rel(out["hist_p"][k], cu[k]) < 1e-9, k


def test_weighted_equals_transformed():
    """Sec. 4.1: PLSS with W = diag(w) on A equals PLSS with W = I on
    A_W = A diag(sqrt(w)), mapped back by x = diag(sqrt(w)) x^W."""
    rng = synth.rng_for(21)
    A = synth.overdetermined_scaled(m=300, n=60, per_row=6, seed=21,
                                   scale_decades=0.5)[0].astype(np.float64)
    xs = rng.standard_normal(A.n)
    b = synth.rhs(A, xs)
    w = oracle.colweights(A, 1)
    D = A.to_dense()
    Aw = synth.from_dense(D * np.sqrt(w)[None, :])
    a = oracle.residual(A, b, w=w, tol=0.0, maxit=25, hist=25)
    t = oracle.residual(Aw, b, tol=0.0, maxit=25, hist=25)
    for k in range(25):
        assert rel(a["hist_x"][k], np.sqrt(w) * t["hist_x"][k]) < 1e-8, k
        np.testing.assert_allclose(a["hist_s"][k, 0], t["hist_s"][k, 0], rtol=1e-8)


def test_planted_gamma_defect_is_caught():
    """The gamma printed in the statement of Theorem 4.1 differs from
    Algorithm 1's by a factor rho; planting it in the oracle must break the
    identity y_k^T p_k = rho_{k-1} and the agreement with eq:pkLong."""
    D, b, rank = CASES[0]
    A = synth.from_dense(D)
    bad = oracle.residual(A, b * 10.0, tol=0.0, maxit=rank, hist=rank, gamma_form=1)
    xs, ps, rs = _pins.projection_run(D, b * 10.0, np.zeros(D.shape[1]), np.ones(D.shape[1]),
                                      rank, "residual")
    assert rel(bad["hist_p"][1], ps[1]) > 1e-3
    Y, P, rho = bad["hist_y"], bad["hist_p"], bad["hist_s"][:, 0]
    assert abs(Y[1] @ P[1] - rho[1]) / rho[1] > 1e-3


# ------------------------------------------------------ edge cases

def test_zero_rhs_returns_x0():
    A, b, _ = synth.square_diag_dominant(n=50, per_row=3, seed=3)
    x0 = np.arange(50.0)
    out = oracle.residual(A, np.zeros(50), x0=x0, tol=1e-10)
    assert out["status"] == "converged" and out["iters"] == 0
    np.testing.assert_array_equal(out["x"], x0)


def test_exact_start_needs_no_update():
    A, b, xs = synth.square_diag_dominant(n=50, per_row=3, seed=3)
    out = oracle.residual(A, b, x0=xs, tol=1e-10)
    assert out["iters"] == 0 and out["status"] == "converged"


def test_maxit_zero_and_not_converged():
    A, b, xs = synth.square_diag_dominant(n=200, per_row=5, seed=4)
    out = oracle.residual(A, b, tol=1e-14, maxit=0)
    assert out["iters"] == 0 and out["status"] == "not_converged"
    out = oracle.residual(A, b, tol=1e-14, maxit=3)
    assert out["iters"] == 3 and out["status"] == "not_converged"
    assert out["relres_true"] < 1.0


def test_breakdown_on_zero_ATr():
    """A^T r_0 = 0 with r_0 != 0 (b outside range(A)) gives phi_1 = 0."""
    D = np.array([[1.0, 0.0], [0.0, 0.0]])
    A = synth.from_dense(D)
    out = oracle.residual(A, np.array([0.0, 1.0]), tol=1e-12)
    assert out["status"] == "breakdown"


# --------------------------------------------------- building blocks

def test_spmv_spmvt_against_scipy():
    A, b, xs = synth.powerlaw_underdetermined(m=500, n=3000, mean_len=20, max_len=400, seed=9)
    A = A.astype(np.float64)
    S = A.scipy()
    v = synth.rng_for(1).standard_normal(A.n)
    r = synth.rng_for(2).standard_normal(A.m)
    np.testing.assert_allclose(oracle.spmv(A, v), S @ v, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.spmvt(A, r), S.T @ r, rtol=1e-12, atol=1e-12)


def test_colweights():
    A, _, _ = synth.overdetermined_scaled(m=400, n=50, per_row=4, seed=8)
    D = A.astype(np.float64).to_dense()
    nrm = np.linalg.norm(D, axis=0)
    np.testing.assert_allclose(oracle.colweights(A, 1), np.where(nrm > 0, 1 / nrm, 1.0), rtol=1e-13)
    np.testing.assert_allclose(oracle.colweights(A, 2), np.where(nrm > 0, 1 / nrm**2, 1.0), rtol=1e-13)


def test_permutation_is_uniform_permutation():
    st = 12345
    counts = np.zeros((4, 4))
    for _ in range(4000):
        perm, st = oracle.permutation(st, 4)
        assert sorted(perm) == [0, 1, 2, 3]
        counts[np.arange(4), perm] += 1
    assert np.all(np.abs(counts / 1000.0 - 1.0) < 0.15)


# ------------------------------------------------------- Kaczmarz

def test_kaczmarz_no_history_is_classical():
    """Sec. 7: with P = 0 the update is the Kaczmarz step."""
    A, b, xs = synth.powerlaw_underdetermined(m=40, n=120, mean_len=6, max_len=30, seed=4)
    A = A.astype(np.float64)
    D = A.to_dense()
    seed = 77
    perm, _ = oracle.permutation(seed, A.m)
    out = oracle.kaczmarz(A, b, tol=0.0, maxit=A.m, K=0, seed=seed)
    ref = _pins.kaczmarz_classic(D, b, np.zeros(A.n), perm)
    assert rel(out["x"], ref) < 1e-12


def test_kaczmarz_history_matches_pklong_and_terminates():
    """eq:pkKacz equals eq:pkLong with S_k = [e_{i_1} ... e_{i_k}]; with the
    whole history on a full-row-rank wide A, x_m = A^+ b (Corollary 3.3)."""
    rng = synth.rng_for(31)
    m, n = 12, 30
    D = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.4)
    D[np.arange(m), np.arange(m)] += 3.0
    A = synth.from_dense(D)
    b = D @ rng.standard_normal(n)
    seed = 5
    perm, _ = oracle.permutation(seed, m)
    xs, ps, _ = _pins.projection_run(D, b, np.zeros(n), np.ones(n), m, "identity", order=perm)
    prev = np.zeros(n)
    P = []
    for k in range(1, m + 1):
        x = oracle.kaczmarz(A, b, tol=0.0, maxit=k, K=m, seed=seed)["x"]
        assert rel(x, xs[k - 1]) < 1e-9, k
        P.append(x - prev)
        prev = x
    P = np.stack(P)
    G = P @ P.T
    sc = np.sqrt(np.outer(np.diag(G), np.diag(G)))
    off = ~np.eye(m, dtype=bool)
    assert np.max(np.abs(G[off]) / sc[off]) < 1e-8
    assert rel(prev, np.linalg.pinv(D) @ b) < 1e-9


def test_kaczmarz_converges_with_restarts():
    A, b, xs = synth.powerlaw_underdetermined(m=200, n=800, mean_len=10, max_len=100, seed=6)
    A = A.astype(np.float64)
    out = oracle.kaczmarz(A, b, tol=1e-8, maxit=200 * 400, K=8, seed=1)
    assert out["status"] == "converged" and out["relres_true"] <= 1e-8


# -------------------------------------------------- configurations

def test_square_2000_converges():
    """The 2,000 x 2,000 diagonally dominant system reaches 1e-10 and, being
    nonsingular, its solution x*."""
    A, b, xs = synth.square_diag_dominant()
    out = oracle.residual(A, b, tol=1e-10, maxit=2000)
    assert out["status"] == "converged"
    assert out["relres_true"] < 2e-10
    assert rel(out["x"], xs) < 1e-8


def test_fp32_storage_with_refinement_reaches_1e8():
    """FP32 storage + FP64 refinement (an extension, not in the paper)
    reaches the FP64 tolerance on the true residual and the FP64 answer."""
    A, b, xs = synth.overdetermined_scaled(m=6000, n=1200, per_row=8, seed=12, scale_decades=1.0)
    ref = oracle.residual(A, b, tol=1e-10, maxit=20000)
    out = oracle.residual(A, b, tol=1e-8, maxit=20000, prec=1, refine=50, stop_on_true=True)
    assert out["status"] == "converged"
    assert out["relres_true"] <= 1e-8
    assert rel(out["x"], ref["x"]) < 1e-5


def test_fp32_first_update_within_float_error_bounds():
    """The FP32-storage mode (an extension, not in the paper) against the
    FP64 mode on the first update, with the textbook error bounds of float
    arithmetic (unit roundoff u = 2^-24; a float sum of k products of floats
    is within gamma_k = k u / (1 - k u) times the sum of their magnitudes):
    r_0 = fl(b) changes rho_0 by at most 2u(1+u) rho_0; each y_j = (A^T r_0)_j
    summed in float is within (gamma_{n_j} (1 + u) + u) sum_i |a_ij b_i| of
    the exact value; phi_1 = y^T y, gamma_1 = rho_0 / phi_1 and
    theta_1 = ||fl(gamma_1 y)||^2 follow with their first-order bounds. The
    differences must also be well above double rounding, so that a mode
    that kept everything in double fails."""
    A, b, xs = synth.overdetermined_scaled(m=3000, n=600, per_row=8, seed=21, scale_decades=1.0)
    A = A.astype(np.float64)                        # values already float-exact
    assert np.array_equal(A.val, A.val.astype(np.float32).astype(np.float64))
    r64 = oracle.residual(A, b, tol=0.0, maxit=1, hist=1)
    r32 = oracle.residual(A, b, tol=0.0, maxit=1, prec=1, hist=1)
    rho64, phi64, _, gam64, th64 = r64["hist_s"][0]
    rho32, phi32, _, gam32, th32 = r32["hist_s"][0]
    u = 2.0 ** -24
    S = A.scipy()
    nj = np.diff(S.tocsc().indptr)                  # products summed per column
    g = nj * u / (1 - nj * u)
    absAb = abs(S).T @ np.abs(b)                    # sum_i |a_ij| |b_i|
    y = S.T @ b                                     # exact to double rounding
    E = (g * (1 + u) + u) * absAb + 1e-12 * absAb   # |y32_j - y_j|, plus double slack
    # rho_0
    assert abs(rho32 - rho64) <= (2 * u * (1 + u) + 1e-12) * rho64
    # phi_1 = sum y_j^2 (u = W y = y)
    dphi = float(np.sum(E * (2 * np.abs(y) + E)))
    assert abs(phi32 - phi64) <= dphi * (1 + 1e-6) + 1e-12 * phi64
    # gamma_1 = rho_0 / phi_1
    rel_rho = 2 * u * (1 + u) + 1e-12
    rel_phi = dphi / (phi64 - dphi)
    rel_gam = rel_rho + rel_phi + rel_rho * rel_phi + 1e-12
    assert abs(gam32 - gam64) <= rel_gam * abs(gam64)
    # theta_1 = sum fl(gamma_1 y_j)^2 against sum (gamma_1 y_j)^2
    dp = abs(gam32 - gam64) * (np.abs(y) + E) + abs(gam64) * E
    p64 = gam64 * y
    dp = dp + u * (np.abs(p64) + dp)                # the float rounding of p
    dth = float(np.sum(dp * (2 * np.abs(p64) + dp)))
    assert abs(th32 - th64) <= dth * (1 + 1e-6) + 1e-12 * th64
    # float arithmetic, not double, was used
    for a32, a64 in ((rho32, rho64), (phi32, phi64), (gam32, gam64), (th32, th64)):
        assert abs(a32 - a64) > 1e-4 * u * abs(a64)
