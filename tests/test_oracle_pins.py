"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage it follows.  None of them re-types the oracle's own
formula: they check closed forms, invariants, an independent solver (HiGHS), brute
force on micro LPs, alternative forms of the same update printed in the paper, the
complexity bounds of Proposition 2.9 / Theorem 3.7 and Pock-Chambolle's norm bound.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog, minimize_scalar

from paper_2408_12179_b300 import lpgen
from oracle import kkt as K

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lp_from_dense(A, m1, b, c, l, u):
    A = np.asarray(A, float)
    return lpgen.LP(lpgen._canonical(A[:m1]), lpgen._canonical(A[m1:]), np.asarray(b[:m1], float),
                    np.asarray(b[m1:], float), np.asarray(c, float), np.asarray(l, float),
                    np.asarray(u, float))


def _f(v):
    return np.array([float(t) for t in v])


# ------------------------------------------------------------------ preprocessing (Section 4.1)

def test_scaling_closed_form_diag(orc):
    g = json.load(open(os.path.join(GOLDEN, "scaling_diag.json")))
    lp = _lp_from_dense(g["A"], g["m1"], g["b"], g["c"], _f(g["l"]), _f(g["u"]))
    s = orc.scale(lp)
    assert np.allclose(s["Dr"], g["Dr"], rtol=1e-15, atol=0)
    assert np.allclose(s["Dc"], g["Dc"], rtol=1e-15, atol=0)
    assert np.allclose(s["As"], [1.0, 1.0], rtol=1e-15)
    assert s["beta_b"] == pytest.approx(g["beta_b"], rel=1e-15)
    assert s["beta_c"] == pytest.approx(g["beta_c"], rel=1e-15)
    assert np.array_equal(s["ls"], _f(g["ls"]))
    assert np.allclose(s["us"], g["us"], rtol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_scaling_is_diagonal_congruence(orc, seed):
    """A_s = D_r A D_c entrywise (the scaling only multiplies rows and columns)."""
    lp = lpgen.planted_tiny(seed)
    s = orc.scale(lp)
    A = lp.A
    rows = np.repeat(np.arange(lp.m), np.diff(A.indptr))
    rebuilt = s["Dr"][rows] * A.data * s["Dc"][A.indices]
    assert np.allclose(s["As"], rebuilt, rtol=1e-14, atol=0)


@pytest.mark.parametrize("seed", range(4))
def test_ruiz_equilibrates(orc, seed):
    """Ruiz's infinity-norm iteration (Ruiz 2001): after one step every |a_ij| <= 1, and
    from then on each row max r'_i >= sqrt(r_i) (the entry that made the old row max is
    divided by sqrt(r_i * kappa_j) with kappa_j <= 1), likewise for columns; so the
    largest |log r| over rows and columns at least halves per step."""
    lp = lpgen.planted_medium(seed, 0.002)
    A = lp.A

    def dev(iters):
        s = orc.scale(lp, ruiz_iters=iters, pc_alpha=-1.0)  # Ruiz only
        As = sp.csr_matrix((s["As"], A.indices, A.indptr), shape=A.shape)
        r = abs(As).max(axis=1).toarray().ravel()
        c = abs(As).max(axis=0).toarray().ravel()
        assert np.abs(s["As"]).max() <= 1.0 + 4e-16 or iters == 0
        return max(np.abs(np.log2(r[r > 0])).max(), np.abs(np.log2(c[c > 0])).max())

    d1 = dev(1)
    prev = d1
    for it in (2, 5, 10):
        d = dev(it)
        assert d <= d1 * 2.0 ** -(it - 1) * (1 + 1e-9) + 1e-14
        assert d <= prev
        prev = d


@pytest.mark.parametrize("ruiz", [0, 10])
def test_pock_chambolle_norm_bound(orc, ruiz):
    """Pock & Chambolle (2011), Lemma 2: with alpha = 1 the preconditioned operator has
    spectral norm at most 1, so lambda_1(A_s A_s^T) <= 1."""
    lp = lpgen.planted_tiny(7)
    s = orc.scale(lp, ruiz_iters=ruiz, pc_alpha=1.0)
    A = lp.A
    As = sp.csr_matrix((s["As"], A.indices, A.indptr), shape=A.shape).toarray()
    assert np.linalg.norm(As, 2) <= 1.0 + 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_scaled_problem_keeps_planted_optimum(orc, seed):
    """The planted KKT point maps to a KKT point of the scaled LP:
    x_s = x / (beta_b D_c), y_s = y / (beta_c D_r), z_s = z D_c / beta_c."""
    lp = lpgen.planted_tiny(seed)
    s = orc.scale(lp)
    A = lp.A
    As = sp.csr_matrix((s["As"], A.indices, A.indptr), shape=A.shape)
    xs = lp.x_star / (s["beta_b"] * s["Dc"])
    ys = lp.y_star / (s["beta_c"] * s["Dr"])
    zs = lp.z_star * s["Dc"] / s["beta_c"]
    r = As @ xs - s["bs"]
    assert np.abs(r[:lp.m1]).max() < 1e-12
    assert r[lp.m1:].min() > -1e-12
    assert np.abs(s["cs"] - As.T @ ys - zs).max() < 1e-12
    assert np.all(xs >= s["ls"] - 1e-15) and np.all(xs <= s["us"] + 1e-15)
    at_l = zs > 0
    at_u = zs < 0
    assert np.allclose(xs[at_l], s["ls"][at_l], rtol=1e-14, atol=1e-15)
    assert np.allclose(xs[at_u], s["us"][at_u], rtol=1e-14, atol=1e-15)
    assert np.linalg.norm(s["bs"]) < 1.0 and np.linalg.norm(s["cs"]) < 1.0


# ------------------------------------------------------------------ power method (Section 4.1)

@pytest.mark.parametrize("seed", range(4))
def test_power_method_matches_dense_eigensolver(orc, seed):
    lp = lpgen.planted_tiny(seed)
    s = orc.scale(lp)
    A = lp.A
    As = sp.csr_matrix((s["As"], A.indices, A.indptr), shape=A.shape)
    lam, it = orc.power(As, tol=1e-14, max_iter=20000)
    ev = np.linalg.eigvalsh((As @ As.T).toarray())
    assert lam == pytest.approx(ev[-1], rel=1e-9)


def test_power_start_vector_is_splitmix64(orc):
    """On a diagonal A the first Rayleigh quotient is sum(a_i^2 u_i^2)/sum(u_i^2) with u
    the SplitMix64 start vector; one iteration with max_iter=1 returns it."""
    d = np.array([1.0, 2.0, 3.0, 0.5])
    A = sp.diags(d).tocsr()
    u = 2.0 * lpgen.splitmix64_uniform(99, 4) - 1.0
    lam, _ = orc.power(A, seed=99, max_iter=1)
    assert lam == pytest.approx(np.sum(d ** 2 * u ** 2) / np.sum(u ** 2), rel=1e-14)


# ------------------------------------------------------------------ final results vs planted / HiGHS / brute force

@pytest.mark.parametrize("seed", range(6))
def test_planted_tiny_solved(orc, seed):
    lp = lpgen.planted_tiny(seed)
    r = orc.solve(lp, tol=1e-8, max_iter=100_000)
    assert r["info"]["status"] == 0
    ind = K.kkt(lp, r["x"], r["y"], r["z"])
    assert ind["kkt"] <= 1e-8
    assert ind["kkt"] == pytest.approx(r["info"]["kkt"], rel=1e-6, abs=1e-15)
    assert abs(ind["pobj"] - lp.planted_objective) <= 1e-7 * abs(lp.planted_objective)
    assert K.in_C(r["x"], lp.l, lp.u)
    assert K.in_D(r["y"], lp.m1)


def _highs(lp):
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b)
              for a, b in zip(lp.l, lp.u)]
    kw = {}
    if lp.m1:
        kw.update(A_eq=lp.A1.toarray(), b_eq=lp.b1)
    if lp.m2:
        kw.update(A_ub=-lp.A2.toarray(), b_ub=-lp.b2)
    res = linprog(lp.c, bounds=bounds, method="highs", **kw)
    assert res.status == 0
    return res.fun


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_tiny_vs_highs(orc, seed):
    lp = lpgen.planted_tiny(seed, m1=30, m2=50, n=150, density=0.07)
    ref = _highs(lp)
    r = orc.solve(lp, tol=1e-8, max_iter=200_000)
    assert r["info"]["status"] == 0
    assert abs(r["info"]["pobj"] - ref) <= 1e-7 * max(1.0, abs(ref))


def _vertex_enumeration(lp):
    """Brute force: the optimum of a bounded feasible LP is attained at a vertex; a
    vertex makes n linearly independent constraints active (all equalities plus n - m1
    of the inequality rows and bounds)."""
    A1 = lp.A1.toarray()
    A2 = lp.A2.toarray()
    n = lp.n
    cand = [("row", i) for i in range(lp.m2)] + [("l", j) for j in range(n)] + [("u", j) for j in range(n)]
    best = math.inf
    for S in itertools.combinations(cand, n - lp.m1):
        M = [A1[i] for i in range(lp.m1)]
        rhs = list(lp.b1)
        for kind, i in S:
            if kind == "row":
                M.append(A2[i]); rhs.append(lp.b2[i])
            else:
                e = np.zeros(n); e[i] = 1.0
                M.append(e); rhs.append(lp.l[i] if kind == "l" else lp.u[i])
        M = np.array(M)
        if abs(np.linalg.det(M)) < 1e-10:
            continue
        x = np.linalg.solve(M, np.array(rhs))
        if np.all(x >= lp.l - 1e-9) and np.all(x <= lp.u + 1e-9) and \
                np.all(np.abs(A1 @ x - lp.b1) <= 1e-9) and np.all(A2 @ x >= lp.b2 - 1e-9):
            best = min(best, float(lp.c @ x))
    return best


@pytest.mark.parametrize("seed", range(8))
def test_micro_vs_vertex_enumeration(orc, seed):
    lp = lpgen.micro_lp(seed, n=4 + seed % 2, m1=1, m2=2 + seed % 2)
    ref = _vertex_enumeration(lp)
    r = orc.solve(lp, tol=1e-10, max_iter=400_000)
    assert r["info"]["status"] == 0
    assert abs(r["info"]["pobj"] - ref) <= 1e-8 * max(1.0, abs(ref))


def test_simplex_closed_form(orc):
    c = np.array([3.0, -1.5, 2.0, -1.25, 0.5])
    r = orc.solve(lpgen.simplex_lp(c), tol=1e-10, max_iter=200_000)
    assert r["info"]["status"] == 0
    assert r["info"]["pobj"] == pytest.approx(c.min(), abs=1e-8)


def test_knapsack_closed_form(orc):
    a = [2.0, 1.0, 4.0, 3.0]
    cost = [3.0, 2.5, 5.0, 6.0]
    ub = [1.0, 2.0, 0.5, 4.0]
    beta = 5.0
    r = orc.solve(lpgen.knapsack_lp(a, cost, beta, ub), tol=1e-10, max_iter=200_000)
    assert r["info"]["status"] == 0
    assert r["info"]["pobj"] == pytest.approx(lpgen.knapsack_optimum(a, cost, beta, ub), rel=1e-8)


# ------------------------------------------------------------------ the iteration (Section 3.3, Algorithm 2)

def _scaled(orc, lp):
    s = orc.scale(lp)
    A = lp.A
    s["A"] = sp.csr_matrix((s["As"], A.indices, A.indptr), shape=A.shape)
    return s


def _prev(tr, key, k, size):
    return tr[key][k - 1] if k > 0 else np.zeros(size)


def test_feasibility_invariants(orc):
    """x_bar in C and y_bar in D for every iteration (Section 4.1, termination)."""
    lp = lpgen.planted_tiny(3)
    s = _scaled(orc, lp)
    r = orc.solve(lp, max_iter=400, trace_iters=400)
    tr = r["trace"]
    assert np.all(tr["xbar"] >= s["ls"]) and np.all(tr["xbar"] <= s["us"])
    assert np.all(tr["ybar"][:, lp.m1:] >= 0.0)


def test_y_update_alternative_form(orc):
    """eq. (update-y) with R_y = x_bar/sigma + (A^* y + z_bar - c) gives the same y_bar as
    the form eq. (update-y-2) that the oracle implements; z_bar from eq. (update-z)."""
    lp = lpgen.planted_tiny(4)
    s = _scaled(orc, lp)
    lam = 0.75
    r = orc.solve(lp, max_iter=60, trace_iters=60, lambda_fixed=lam)
    tr = r["trace"]
    A, m1, sigma = s["A"], lp.m1, 1.0
    for k in range(0, 60, 7):
        x = _prev(tr, "x", k, lp.n)
        y = _prev(tr, "y", k, lp.m)
        v = x + sigma * (A.T @ y - s["cs"])
        zbar = (np.clip(v, s["ls"], s["us"]) - v) / sigma
        Ry = tr["xbar"][k] / sigma + (A.T @ y + zbar - s["cs"])
        yb = y + (s["bs"] / sigma - A @ Ry) / lam
        yb[m1:] = np.maximum(yb[m1:], 0.0)
        assert np.allclose(yb, tr["ybar"][k], rtol=1e-12, atol=1e-13)


def test_x_and_z_steps_are_argmins(orc):
    """Steps 1-2 of Algorithm 2 from the definition of L_sigma (Section 2): z_bar
    minimises delta_C^*(-z) + <x, z> + sigma/2 ||A^* y + z - c||^2 coordinate-wise, and
    x_bar = x + sigma (A^* y + z_bar - c)."""
    lp = lpgen.planted_tiny(5)
    s = _scaled(orc, lp)
    r = orc.solve(lp, max_iter=30, trace_iters=30, lambda_fixed=0.8)
    tr = r["trace"]
    k = 20
    x = tr["x"][k - 1]
    y = tr["y"][k - 1]
    g = s["A"].T @ y - s["cs"]
    sigma = 1.0
    for j in range(0, lp.n, 9):
        lo, hi = s["ls"][j], s["us"][j]

        def f(z):  # delta_C^*(-z) = max over [lo, hi] of -z x
            sup = max(-z * lo if np.isfinite(lo) or z < 0 else np.inf,
                      -z * hi if np.isfinite(hi) or z > 0 else np.inf)
            if z == 0:
                sup = 0.0
            return sup + x[j] * z + 0.5 * sigma * (g[j] + z) ** 2

        if not np.isfinite(hi):
            res = minimize_scalar(f, bounds=(0.0, 1e3), method="bounded", options={"xatol": 1e-13})
        else:
            res = minimize_scalar(f, bounds=(-1e3, 1e3), method="bounded", options={"xatol": 1e-13})
        xb = x[j] + sigma * (g[j] + res.x)
        assert xb == pytest.approx(tr["xbar"][k][j], abs=1e-6)


def test_y_step_is_argmin(orc):
    """Step 3 of Algorithm 2 from its definition: y_bar minimises
    L_sigma(y, z_bar; x_bar) + sigma/2 ||y - y^k||^2_{T1} over y with y2 >= 0,
    T1 = lambda I - A A^*; solved here as a bound-constrained QP (L-BFGS-B)."""
    from scipy.optimize import minimize

    lp = lpgen.planted_tiny(6, m1=8, m2=12, n=30, density=0.2)
    s = _scaled(orc, lp)
    lam = float(np.linalg.eigvalsh((s["A"] @ s["A"].T).toarray())[-1]) * 1.5
    r = orc.solve(lp, max_iter=12, trace_iters=12, lambda_fixed=lam)
    tr = r["trace"]
    A = s["A"].toarray()
    k, sigma = 10, 1.0
    x, y = tr["x"][k - 1], tr["y"][k - 1]
    v = x + sigma * (A.T @ y - s["cs"])
    xb = np.clip(v, s["ls"], s["us"])
    zb = (xb - v) / sigma
    T1 = lam * np.eye(lp.m) - A @ A.T

    def obj(yy):
        rr = A.T @ yy + zb - s["cs"]
        d = yy - y
        val = -s["bs"] @ yy + xb @ rr + 0.5 * sigma * rr @ rr + 0.5 * sigma * d @ T1 @ d
        grad = -s["bs"] + A @ xb + sigma * A @ rr + sigma * T1 @ d
        return val, grad

    bnds = [(None, None)] * lp.m1 + [(0.0, None)] * lp.m2
    res = minimize(obj, y.copy(), jac=True, method="L-BFGS-B", bounds=bnds,
                   options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 10000})
    assert np.allclose(res.x, tr["ybar"][k], atol=1e-6)


def _M_norm(A, sigma, lam, dy, dx):
    q = sigma * lam * dy @ dy + 2.0 * dy @ (A @ dx) + dx @ dx / sigma
    return math.sqrt(max(q, 0.0))


def test_merit_is_the_M_norm_of_its_definition(orc):
    """The merit that drives the restart criteria (Section 3.1), R~ = ||w - w_hat||_M =
    2 ||w - w_bar||_M, with M built as a dense matrix from its block definition (eq. def:M,
    unsimplified: sigma A A^* + sigma T1 with T1 = lambda I - A A^*, a zero z block, A and
    A^* off the diagonal, I / sigma), equals the oracle's recorded value at every check of
    the traced iterations: the R~_{r,0} evaluations and the periodic checks, across restarts
    and sigma changes.  The z part of w - w_bar is random: the zero block must ignore it."""
    lp = lpgen.planted_tiny(0)
    s = _scaled(orc, lp)
    A = s["A"].toarray()
    m, n = lp.m, lp.n
    N = 1200
    r = orc.solve(lp, max_iter=N, trace_iters=N)
    lam = r["info"]["lambda"]
    tr = r["trace"]
    rng = np.random.default_rng(5)
    seen_kinds, sigmas = set(), set()
    for c in r["checks"]:
        k = int(c["k"])
        if k >= min(N, int(r["info"]["iters"]) - 1):    # (the terminating iteration is not traced)
            continue
        sigma = c["sigma"]
        T1 = lam * np.eye(m) - A @ A.T
        M = np.zeros((m + 2 * n, m + 2 * n))
        M[:m, :m] = sigma * (A @ A.T) + sigma * T1
        M[:m, m + n:] = A
        M[m + n:, :m] = A.T
        M[m + n:, m + n:] = np.eye(n) / sigma
        d = np.concatenate([_prev(tr, "y", k, m) - tr["ybar"][k], rng.standard_normal(n),
                            _prev(tr, "x", k, n) - tr["xbar"][k]])
        q = d @ M @ d
        assert q >= -1e-12 * (d @ d)
        assert c["Rt"] == pytest.approx(2.0 * math.sqrt(max(q, 0.0)), rel=1e-8, abs=1e-14), (k, c["kind"])
        seen_kinds.add(int(c["kind"]))
        sigmas.add(sigma)
    assert {1, 2} <= seen_kinds and len(sigmas) >= 2     # periodic checks, R~_{r,0}, several sigmas


@pytest.mark.parametrize("seed", range(3))
def test_prop_2_9_and_theorem_3_7_bounds(orc, seed):
    """Proposition 2.9: ||w^k - w_hat^{k+1}||_M <= 2 ||w^0 - w*||_M / (k+1) and Theorem 3.7:
    ||R(w_bar^{k+1})|| <= (sigma (||A|| + ||sqrt(T1)||) + 1)/sqrt(sigma) R_0/(k+1), for the
    plain HPR (fixed sigma, no restart), lambda >= lambda_1(A A^*), w* the planted KKT
    point mapped to the scaled LP, R_0 = ||w^0 - w*||_M."""
    lp = lpgen.planted_tiny(seed)
    s = _scaled(orc, lp)
    A = s["A"]
    lam = float(np.linalg.eigvalsh((A @ A.T).toarray())[-1]) * (1 + 1e-12)
    sigma = 1.0
    N = 600
    r = orc.solve(lp, max_iter=N, trace_iters=N, lambda_fixed=lam, restart=0, sigma_update=0,
                  check_every=10 ** 9)
    tr = r["trace"]
    xs = lp.x_star / (s["beta_b"] * s["Dc"])
    ys = lp.y_star / (s["beta_c"] * s["Dr"])
    R0 = _M_norm(A, sigma, lam, -ys, -xs)
    normA = math.sqrt(lam)
    for k in range(N):
        x = _prev(tr, "x", k, lp.n)
        y = _prev(tr, "y", k, lp.m)
        xh = tr["xhat"][k]
        yh = 2.0 * tr["ybar"][k] - y
        assert _M_norm(A, sigma, lam, y - yh, x - xh) <= 2.0 * R0 / (k + 1) * (1 + 1e-9)
        # KKT residual map of Section 2 on the scaled LP at w_bar^{k+1}
        xb, yb = tr["xbar"][k], tr["ybar"][k]
        v = x + sigma * (A.T @ y - s["cs"])
        zb = (xb - v) / sigma
        t = yb - A @ xb + s["bs"]
        t[lp.m1:] = np.maximum(t[lp.m1:], 0.0)
        R = np.concatenate([yb - t, xb - np.clip(xb - zb, s["ls"], s["us"]), s["cs"] - A.T @ yb - zb])
        bound = (sigma * (normA + math.sqrt(lam)) + 1.0) / math.sqrt(sigma) * R0 / (k + 1)
        assert np.linalg.norm(R) <= bound * (1 + 1e-9)


def test_sigma_update_matches_general_formula(orc):
    """eq. (sigma_T1!=0) is eq. (sigma_approx) with Delta_y of eq. (Dx&Dy) for
    T1 = lambda I - A A^*: Delta_y^2 = ||dy||^2_{T1} + ||A^* dy||^2."""
    lp = lpgen.planted_tiny(1)
    s = _scaled(orc, lp)
    r = orc.solve(lp, max_iter=400, trace_iters=400)
    first = [c for c in r["checks"] if c["cause"] > 0][0]
    k = int(first["k"])
    assert first["r"] == 0          # anchors are the origin
    A = s["A"]
    lam = r["info"]["lambda"]
    dx = r["trace"]["xbar"][k]
    dy = r["trace"]["ybar"][k]
    dyT1 = lam * dy @ dy - np.linalg.norm(A.T @ dy) ** 2
    Dx = np.linalg.norm(dx)
    Dy = math.sqrt(dyT1 + np.linalg.norm(A.T @ dy) ** 2)
    assert 1e-16 < Dx < 1e12 and 1e-16 < Dy < 1e12
    ratio = first["err_d"] / first["err_p"]
    assert 1e-8 < ratio < 1e8
    assert first["sigma_next"] == pytest.approx(Dx / Dy, rel=1e-12)


def test_termination_quantities_match_independent_evaluator(orc):
    lp = lpgen.planted_tiny(2)
    r = orc.solve(lp, tol=1e-6, max_iter=100_000)
    ind = K.kkt(lp, r["x"], r["y"], r["z"])
    for key in ("err_p", "err_d", "err_gap", "pobj", "dobj"):
        assert ind[key] == pytest.approx(r["info"][key], rel=1e-9, abs=1e-14)


def test_thread_count_does_not_change_results(tmp_path):
    """Rows are summed in index order whatever the OpenMP thread count."""
    import subprocess
    import sys

    code = ("import sys, numpy as np; sys.path.insert(0, %r); import oracle; "
            "from paper_2408_12179_b300 import lpgen; lp = lpgen.planted_medium(1, 0.03); "
            "r = oracle.solve(lp, max_iter=300); np.save(sys.argv[1], np.concatenate([r['x'], r['y']]))"
            % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    outs = []
    for th in ("1", "4"):
        p = tmp_path / f"o{th}.npy"
        env = dict(os.environ, OMP_NUM_THREADS=th)
        subprocess.run([sys.executable, "-c", code, str(p)], check=True, env=env)
        outs.append(np.load(p))
    assert np.array_equal(outs[0], outs[1])


# ------------------------------------------------------------------ ablation variants (Section 4.2)

VARIANTS = {  # Section 4.2, Figure 1: DR -> + restart & Halpern -> + sigma update -> + relaxation
    "DR": dict(halpern=0, reflect=0, restart=0, sigma_update=0),
    "HDR_fixed_sigma": dict(halpern=1, reflect=0, restart=1, sigma_update=0),
    "HDR": dict(halpern=1, reflect=0, restart=1, sigma_update=1),
    "HPR": dict(halpern=1, reflect=1, restart=1, sigma_update=1),
}


@pytest.mark.parametrize("reflect", [0, 1])
def test_dr_and_pr_fixed_point_residual_is_monotone(orc, reflect):
    """Without the Halpern step the iteration is w^{k+1} = G(w^k) with G: w -> w_bar =
    (M + T)^{-1} M w, the preconditioned proximal point map of the dPPM form of
    Algorithm 1 (Proposition prop:equ-acc-PADMM-acc-dPPM), firmly nonexpansive in the
    M-seminorm (DR, reflect 0), or its reflection 2G - I, nonexpansive (PR, reflect 1).
    Either way ||w^{k+1} - w^k||_M cannot increase.  Checked on the trace with an M-norm
    written here from eq. (def:M) with T1 = lambda I - A A^*, lambda >= lambda_1(A A^*)
    from a dense eigensolver."""
    lp = lpgen.planted_tiny(4)
    s = _scaled(orc, lp)
    A = s["A"]
    lam = float(np.linalg.eigvalsh((A @ A.T).toarray())[-1]) * (1 + 1e-12)
    N = 300
    r = orc.solve(lp, max_iter=N, trace_iters=N, lambda_fixed=lam, restart=0, sigma_update=0,
                  halpern=0, reflect=reflect, check_every=10 ** 9)
    tr = r["trace"]
    steps = []
    for k in range(N):
        dx = tr["x"][k] - _prev(tr, "x", k, lp.n)
        dy = tr["y"][k] - _prev(tr, "y", k, lp.m)
        steps.append(_M_norm(A, 1.0, lam, dy, dx))
    assert steps[0] > 0.0
    for k in range(1, N):
        assert steps[k] <= steps[k - 1] * (1 + 1e-9) + 1e-15, (k, steps[k], steps[k - 1])
    # the DR step is w_bar itself, the PR step its reflection
    k = 57
    target = tr["xbar"][k] if reflect == 0 else 2.0 * tr["xbar"][k] - _prev(tr, "x", k, lp.n)
    assert np.array_equal(tr["x"][k], target)


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_ablation_variants_reach_planted_optimum(orc, variant):
    """Each variant of the Section 4.2 ablation converges on a planted LP (the DR method,
    Steps 1-3 of Algorithm 1 iterated, at a looser tolerance: it is the slow baseline)."""
    lp = lpgen.planted_tiny(2)
    tol = 1e-6 if variant == "DR" else 1e-8
    r = orc.solve(lp, tol=tol, max_iter=400_000, **VARIANTS[variant])
    assert r["info"]["status"] == 0, variant
    ind = K.kkt(lp, r["x"], r["y"], r["z"])
    assert ind["kkt"] <= tol * (1 + 1e-6)
    assert abs(ind["pobj"] - lp.planted_objective) <= 10 * tol * (1 + abs(lp.planted_objective))


# ------------------------------------------------------------------ min-cost multicommodity flow

def test_mcf_small_vs_highs(orc):
    """The min-cost multicommodity-flow family (random geometric k-NN digraph, shared
    capacities): no planted optimum, so the oracle's objective is pinned to HiGHS and its
    returned point to the independent KKT evaluator."""
    lp = lpgen.mcf_lp(0, nodes=300)
    r = orc.solve(lp, tol=1e-8, max_iter=200_000)
    assert r["info"]["status"] == 0
    ind = K.kkt(lp, r["x"], r["y"], r["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    def csr32(M, sign=1.0):   # HiGHS' sparse input wants 32-bit row pointers
        return sp.csr_matrix((sign * M.data, M.indices.astype(np.int32), M.indptr.astype(np.int32)),
                             shape=M.shape)

    res = linprog(lp.c, A_eq=csr32(lp.A1), b_eq=lp.b1, A_ub=csr32(lp.A2, -1.0), b_ub=-lp.b2,
                  bounds=[(0, None)] * lp.n, method="highs")
    assert res.status == 0
    assert abs(ind["pobj"] - res.fun) <= 1e-7 * abs(res.fun)


# ------------------------------------------------------------------ sigma policy network oracle

def _mlp_data(seed, n=40):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 64)), rng.integers(0, 5, n), rng.standard_normal(n)


def test_mlp_gradient_matches_finite_differences():
    """The chain-rule gradient equals central differences of the loss (FP64 weights, no
    BF16 rounding) on 200 random coordinates, every layer included."""
    from oracle import mlp
    X, a, y = _mlp_data(1)
    w = mlp.init(3).astype(np.float64)
    L, g = mlp.loss_grad(w, X, a, y, bf16=False)
    rng = np.random.default_rng(5)
    coords = np.concatenate([rng.choice(mlp.P, 192, replace=False),
                             [0, 4096, 4160, 8256, 8320, 12416, 12480, 12800]])
    h = 1e-6
    for c in coords:
        wp, wm = w.copy(), w.copy()
        wp[c] += h
        wm[c] -= h
        fd = (mlp.loss_grad(wp, X, a, y, bf16=False)[0] - mlp.loss_grad(wm, X, a, y, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[c]) <= 1e-6 * (1 + abs(fd)), (c, fd, g[c])


def test_mlp_closed_form_with_only_output_bias():
    """All weights 0 but b4: q = b4 for every input, L = mean 1/2 (b4[a] - y)^2, dL/db4[o]
    = mean over samples of [a = o] (b4[o] - y), every other gradient 0."""
    from oracle import mlp
    X, a, y = _mlp_data(2)
    w = np.zeros(mlp.P)
    b4 = np.array([0.5, -1.0, 2.0, 0.25, -0.75])
    w[-5:] = b4
    L, g = mlp.loss_grad(w, X, a, y, bf16=False)
    assert L == pytest.approx(0.5 * np.mean((b4[a] - y) ** 2), rel=1e-15)
    want = np.array([np.sum((b4[o] - y)[a == o]) for o in range(5)]) / len(y)
    assert np.allclose(g[-5:], want, rtol=1e-14, atol=1e-16)
    assert not np.any(g[:-5])


def test_bf16_rounding_is_nearest_even():
    """BF16 keeps the top 16 bits of the FP32 pattern, rounding to nearest, ties to even."""
    from oracle import mlp
    one = np.float32(1.0)
    ulp = 2.0 ** -7                                    # BF16 spacing at 1
    cases = {1.0: 1.0, 1.0 + ulp / 2: 1.0, 1.0 + 3 * ulp / 2: 1.0 + 2 * ulp,
             1.0 + ulp / 2 + 2.0 ** -20: 1.0 + ulp, -(1.0 + 3 * ulp / 2): -(1.0 + 2 * ulp),
             3.0e38: 226 * 2.0 ** 120}                 # 3e38 / 2^120 = 225.7: the upper neighbour
    for x, want in cases.items():
        got = mlp.bf16_round(np.array([x], np.float32))[0]
        assert got == pytest.approx(want, rel=1e-7), (x, got, want)
    assert mlp.bf16_round(np.array([one], np.float32))[0] == 1.0


# ------------------------------------------------------------------ QAP (Adams-Johnson) workload

def _perm_point(N, perm):
    """The LP point of an assignment: x_ij = [perm(i) = j], s_ijkl = x_ij x_kl."""
    X = np.zeros((N, N))
    X[np.arange(N), perm] = 1.0
    S = np.einsum("ij,kl->ijkl", X, X)
    return np.concatenate([X.ravel(), S.ravel()])


@pytest.mark.parametrize("N", [4, 5])
def test_qap_lp_relaxes_the_qap(orc, N):
    """Every assignment, lifted by s_ijkl = x_ij x_kl, satisfies the linearisation's rows
    and costs sum a_ik b_perm(i)perm(k); the LP optimum found by the oracle matches HiGHS
    and lies below the best assignment (brute force over all N! of them)."""
    lp = lpgen.qap_lp(3, N)
    a, b = lpgen.qap_matrices(3, N)
    best = np.inf
    for perm in itertools.permutations(range(N)):
        perm = np.array(perm)
        v = _perm_point(N, perm)
        assert np.allclose(lp.A1 @ v, lp.b1, atol=1e-12)
        cost = float(lp.c @ v)
        assert cost == pytest.approx(float(np.sum(a * b[np.ix_(perm, perm)])), abs=1e-9)
        best = min(best, cost)
    r = orc.solve(lp, tol=1e-8, max_iter=400_000)
    assert r["info"]["status"] == 0
    ind = K.kkt(lp, r["x"], r["y"], r["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    A1 = sp.csr_matrix((lp.A1.data, lp.A1.indices.astype(np.int32), lp.A1.indptr.astype(np.int32)), shape=lp.A1.shape)
    res = linprog(lp.c, A_eq=A1, b_eq=lp.b1, bounds=list(zip(lp.l, [None if not np.isfinite(u) else u for u in lp.u])),
                  method="highs")
    assert res.status == 0
    assert abs(ind["pobj"] - res.fun) <= 1e-7 * max(1.0, abs(res.fun))
    assert res.fun <= best + 1e-9


# ------------------------------------------------------------------ degenerate LPs

def test_fixed_variables_keep_the_planted_optimum(orc):
    """Fixing columns at their planted values (l = u = x*_j) keeps x* optimal (both bounds
    active, z*_j of either sign is allowed): the oracle reaches the planted objective."""
    lp = lpgen.planted_tiny(3)
    fix = np.arange(0, lp.n, 7)
    lp.l = lp.l.copy(); lp.u = lp.u.copy()
    lp.l[fix] = lp.x_star[fix]
    lp.u[fix] = lp.x_star[fix]
    r = orc.solve(lp, tol=1e-8, max_iter=400_000)
    assert r["info"]["status"] == 0
    assert np.array_equal(r["x"][fix], lp.x_star[fix])
    ind = K.kkt(lp, r["x"], r["y"], r["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    assert abs(ind["pobj"] - lp.planted_objective) <= 1e-7 * abs(lp.planted_objective)


def test_infeasible_lp_runs_to_the_cap(orc):
    """An infeasible LP (x1 + x2 = 1 and x1 + x2 >= 3): the iteration stays finite, stops at
    max_iter, and its primal residual does not vanish."""
    A1 = lpgen._canonical(sp.csr_matrix(np.array([[1.0, 1.0]])))
    A2 = lpgen._canonical(sp.csr_matrix(np.array([[1.0, 1.0]])))
    lp = lpgen.LP(A1, A2, np.array([1.0]), np.array([3.0]), np.array([1.0, 2.0]), np.zeros(2), np.full(2, 10.0))
    r = orc.solve(lp, tol=1e-8, max_iter=3000)
    assert r["info"]["status"] == 1
    assert np.all(np.isfinite(r["x"])) and np.all(np.isfinite(r["y"]))
    assert r["info"]["err_p"] > 1e-3
    assert K.kkt(lp, r["x"], r["y"], r["z"])["err_p"] > 1e-3
