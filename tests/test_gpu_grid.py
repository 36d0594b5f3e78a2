"""The persistent grid path (one cooperative launch runs the whole solve; software grid
barriers between the two phases of Algorithm 2) against the oracle, and its bounded
barrier waits.

* full solves at tol 1e-8: lambda to 1e-10, objective within 1e-7 of the oracle's, an
  independently evaluated KKT residual <= tol, and the decision sequence (Section 3.1,
  Algorithm 3) rebuilt from the path's own values and compared with the oracle's;
* 100 iterations with lambda fixed (no restart decision is taken before the cap): the
  returned w_bar against the oracle's, normwise 1e-11 and entry by entry, and bitwise the
  same whatever the number of CTAs and on the single-CTA path (the row sums and updates do
  not depend on how rows are spread over CTAs);
* a CTA that skips one barrier arrival (HPR_FAULT_BARRIER, host-injected) makes every wait
  run out of its budget: the solve returns HPR_ERR_DEVICE_TIMEOUT within milliseconds and
  the context and the GPU stay usable.
"""
import os

import numpy as np
import pytest

from paper_2408_12179_b300 import hpr, lpgen

pytestmark = pytest.mark.gpu

import oracle
from oracle import kkt as K
from decisions import compare_decisions


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def elem(a, b, floor=1e-6):
    scale = np.maximum(np.abs(b), floor * np.max(np.abs(b), initial=0.0))
    d = np.abs(a - b)
    return float(np.max(np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), np.where(d > 0, np.inf, 0.0)),
                        initial=0.0))


CASES = {
    "tiny0": lambda: lpgen.planted_tiny(0),
    "medium/500": lambda: lpgen.planted_medium(1, 0.002),
    "medium/200": lambda: lpgen.planted_medium(0, 0.005),
    "qap6": lambda: lpgen.qap_lp(2, 6),
}


@pytest.fixture(autouse=True)
def _clean_env():
    for key in ("HPR_FAULT_BARRIER", "HPR_GRID_CTAS"):
        os.environ.pop(key, None)
    yield
    for key in ("HPR_FAULT_BARRIER", "HPR_GRID_CTAS"):
        os.environ.pop(key, None)


@pytest.mark.parametrize("name", list(CASES))
def test_grid_full_solve_matches_oracle(name):
    lp = CASES[name]()
    ref = oracle.solve(lp, tol=1e-8, max_iter=2_000_000)
    assert ref["info"]["status"] == 0
    with hpr.Solver(lp, persistent=3, max_iter=2_000_000) as s:
        res = s.solve(1e-8)
        checks = s.checks()
    I = res["info"]
    assert res["status"] == hpr.HPR_OK and I["launches"] <= 3
    assert I["lambda"] == pytest.approx(ref["info"]["lambda"], rel=1e-10)
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    assert abs(I["primal_obj"] - ref["info"]["pobj"]) <= 1e-7 * max(1.0, abs(ref["info"]["pobj"]))
    assert K.in_C(res["x"], lp.l, lp.u) and K.in_D(res["y"], lp.m1)
    where = compare_decisions(checks, ref["checks"], 1e-8)
    print(f"{name}: {I['iters']} iterations, decisions equal over {where} of {len(ref['checks'])} records")


@pytest.mark.parametrize("name", ["tiny0", "medium/200"])
def test_grid_first_100_iterations(name):
    lp = CASES[name]()
    N = 100
    ref = oracle.solve(lp, max_iter=N)
    lam = ref["info"]["lambda"]
    outs = []
    for ctas in ("", "2", "7", "148"):
        os.environ["HPR_GRID_CTAS"] = ctas
        res = hpr.solve(lp, tol=1e-12, max_iter=N, lambda_fixed=lam, persistent=3)
        assert res["status"] == hpr.HPR_MAX_ITER
        for key in ("x", "y", "z"):
            assert rel(res[key], ref[key]) <= 1e-11, (ctas, key)
            assert elem(res[key], ref[key]) <= 1e-8, (ctas, key)
        outs.append(np.concatenate([res["x"], res["y"], res["z"]]))
    os.environ.pop("HPR_GRID_CTAS")
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    if name == "tiny0":                              # the single-CTA path does the same row arithmetic
        res = hpr.solve(lp, tol=1e-12, max_iter=N, lambda_fixed=lam, persistent=2)
        assert np.array_equal(np.concatenate([res["x"], res["y"], res["z"]]), outs[0])


def test_grid_barrier_timeout_is_reported():
    lp = lpgen.planted_medium(0, 0.005)
    os.environ["HPR_FAULT_BARRIER"] = "5"
    with hpr.Solver(lp, persistent=3) as s:
        os.environ.pop("HPR_FAULT_BARRIER")
        with pytest.raises(hpr.HprError) as e:
            s.solve(1e-8)
        assert e.value.code == hpr.HPR_ERR_DEVICE_TIMEOUT
        assert "barrier 4" in str(e.value)
    # the GPU and a new context are fine afterwards
    ref = oracle.solve(lp, tol=1e-8, max_iter=2_000_000)
    res = hpr.solve(lp, tol=1e-8, persistent=3)
    assert res["status"] == hpr.HPR_OK
    assert abs(res["info"]["primal_obj"] - ref["info"]["pobj"]) <= 1e-7 * max(1.0, abs(ref["info"]["pobj"]))


def test_grid_refused_when_it_cannot_run():
    with hpr.Solver(lpgen.planted_tiny(0), persistent=3, precision=1) as s:
        with pytest.raises(hpr.HprError) as e:
            s.solve(1e-8)
        assert e.value.code == hpr.HPR_ERR_ARG
