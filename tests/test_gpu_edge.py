"""Degenerate LPs on the CUDA paths (multi-CTA, persistent single-CTA and persistent cluster) against the
oracle: fixed variables (l = u), a pure feasibility problem (c = 0), all-free columns, and
an infeasible LP (the solve must stop at the iteration cap with finite output, not fail)."""
import numpy as np
import pytest

from paper_2408_12179_b300 import hpr, lpgen

pytestmark = pytest.mark.gpu

import oracle
from oracle import kkt as K


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hpr.load()


def _fixed(seed):
    lp = lpgen.planted_tiny(seed)
    fix = np.arange(0, lp.n, 7)                      # every 7th column fixed at its planted value
    lp.l = lp.l.copy(); lp.u = lp.u.copy()
    lp.l[fix] = lp.x_star[fix]
    lp.u[fix] = lp.x_star[fix]
    return lp


def _feasibility(seed):
    lp = lpgen.planted_tiny(seed)
    lp.c = np.zeros(lp.n)
    return lp


def _all_free(seed):
    rng = np.random.default_rng(seed)
    lp = lpgen.planted_tiny(seed, m1=60, m2=0, n=80, density=0.2)
    lp.l = np.full(lp.n, -np.inf)
    lp.u = np.full(lp.n, np.inf)
    y = rng.standard_normal(lp.m1)
    lp.c = lp.A1.T @ y                               # z* = 0: any feasible x with this y is optimal
    return lp


CASES = {"fixed": _fixed, "feasibility": _feasibility, "all_free": _all_free}


@pytest.mark.parametrize("persistent", [0, 2, 4])
@pytest.mark.parametrize("name", list(CASES))
def test_degenerate_lps(name, persistent):
    lp = CASES[name](3)
    ref = oracle.solve(lp, tol=1e-8, max_iter=400_000)
    assert ref["info"]["status"] == 0
    with hpr.Solver(lp, persistent=persistent, max_iter=400_000) as s:
        res = s.solve(1e-8)
    assert res["status"] == hpr.HPR_OK
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    assert abs(res["info"]["primal_obj"] - ref["info"]["pobj"]) <= 1e-7 * max(1.0, abs(ref["info"]["pobj"]))
    assert K.in_C(res["x"], lp.l, lp.u) and K.in_D(res["y"], lp.m1)


@pytest.mark.parametrize("persistent", [0, 2, 4])
def test_infeasible_lp_stops_at_the_cap(persistent):
    """x1 + x2 = 1 and x1 + x2 >= 3 with 0 <= x <= 10: no feasible point.  The solve runs to
    max_iter and returns HPR_MAX_ITER with finite iterates and a primal residual that stays
    away from zero."""
    import scipy.sparse as sp
    A1 = lpgen._canonical(sp.csr_matrix(np.array([[1.0, 1.0]])))
    A2 = lpgen._canonical(sp.csr_matrix(np.array([[1.0, 1.0]])))
    lp = lpgen.LP(A1, A2, np.array([1.0]), np.array([3.0]), np.array([1.0, 2.0]), np.zeros(2), np.full(2, 10.0))
    with hpr.Solver(lp, persistent=persistent, max_iter=3000) as s:
        res = s.solve(1e-8)
    assert res["status"] == hpr.HPR_MAX_ITER
    for key in ("x", "y", "z"):
        assert np.all(np.isfinite(res[key]))
    assert res["info"]["err_p"] > 1e-3
