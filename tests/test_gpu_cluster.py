"""The persistent cluster path (one launch of one thread-block cluster of up to 16 CTAs runs
the whole solve; y and x_hat gathered from replicas in every CTA's shared memory, filled by
st.async stores counted on a transaction barrier per replica; each CTA's slices of A and
A^T and its rows' state in its own shared memory) against the oracle.

* full solves at tol 1e-8: lambda to 1e-10, objective within 1e-7 of the oracle's, an
  independently evaluated KKT residual <= tol, and the decision sequence (Section 3.1,
  Algorithm 3) rebuilt from the path's own values and compared with the oracle's;
* the same solve on the persistent grid path with the same number of CTAs gives bitwise
  the same result (the replicas change where a gather reads, not what it reads);
* 100 iterations with lambda fixed: the returned w_bar against the oracle's, normwise 1e-11
  and entry by entry, bitwise the same for every cluster size, on the grid path and on the
  single-CTA path;
* LPs whose data do not fit in the cluster's shared memory, and the FP32 form, are refused;
* a lost fill of a replica (host-injected) ends in HPR_ERR_DEVICE_TIMEOUT, not a hang.
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
    os.environ.pop("HPR_GRID_CTAS", None)
    yield
    os.environ.pop("HPR_GRID_CTAS", None)


def _wbar(res):
    return np.concatenate([res["x"], res["y"], res["z"]])


@pytest.mark.parametrize("name", list(CASES))
def test_cluster_full_solve_matches_oracle(name):
    lp = CASES[name]()
    ref = oracle.solve(lp, tol=1e-8, max_iter=2_000_000)
    assert ref["info"]["status"] == 0
    with hpr.Solver(lp, persistent=4, max_iter=2_000_000) as s:
        res = s.solve(1e-8)
        checks = s.checks()
    I = res["info"]
    assert res["status"] == hpr.HPR_OK and I["launches"] <= 3 and I["path"] == 4 and 2 <= I["path_ctas"] <= 16
    assert I["lambda"] == pytest.approx(ref["info"]["lambda"], rel=1e-10)
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    assert abs(I["primal_obj"] - ref["info"]["pobj"]) <= 1e-7 * max(1.0, abs(ref["info"]["pobj"]))
    assert K.in_C(res["x"], lp.l, lp.u) and K.in_D(res["y"], lp.m1)
    where = compare_decisions(checks, ref["checks"], 1e-8)
    print(f"{name}: {I['iters']} iterations, decisions equal over {where} of {len(ref['checks'])} records")


@pytest.mark.parametrize("ctas", ["7", "16"])
def test_cluster_equals_grid_path_bitwise(ctas):
    lp = CASES["medium/200"]()
    os.environ["HPR_GRID_CTAS"] = ctas
    a = hpr.solve(lp, tol=1e-8, persistent=4)
    b = hpr.solve(lp, tol=1e-8, persistent=3)
    assert a["status"] == b["status"] == hpr.HPR_OK
    assert (a["info"]["path"], b["info"]["path"]) == (4, 3)
    assert a["info"]["path_ctas"] == b["info"]["path_ctas"] == int(ctas)
    for key in ("iters", "restarts", "power_iters", "lambda", "primal_obj", "dual_obj", "kkt", "sigma"):
        assert a["info"][key] == b["info"][key], key
    assert np.array_equal(_wbar(a), _wbar(b))


@pytest.mark.parametrize("name,sizes", [("tiny0", ("", "2", "7", "16")), ("medium/200", ("", "7", "16"))])
def test_cluster_first_100_iterations(name, sizes):
    lp = CASES[name]()
    N = 100
    ref = oracle.solve(lp, max_iter=N)
    lam = ref["info"]["lambda"]
    outs = []
    for ctas in sizes:
        os.environ["HPR_GRID_CTAS"] = ctas
        res = hpr.solve(lp, tol=1e-12, max_iter=N, lambda_fixed=lam, persistent=4)
        assert res["status"] == hpr.HPR_MAX_ITER
        for key in ("x", "y", "z"):
            assert rel(res[key], ref[key]) <= 1e-11, (ctas, key)
            assert elem(res[key], ref[key]) <= 1e-8, (ctas, key)
        outs.append(_wbar(res))
    os.environ.pop("HPR_GRID_CTAS")
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    res = hpr.solve(lp, tol=1e-12, max_iter=N, lambda_fixed=lam, persistent=3)
    assert np.array_equal(_wbar(res), outs[0])
    if name == "tiny0":                              # the single-CTA path does the same row arithmetic
        res = hpr.solve(lp, tol=1e-12, max_iter=N, lambda_fixed=lam, persistent=2)
        assert np.array_equal(_wbar(res), outs[0])


def test_cluster_fill_timeout_is_reported():
    """A CTA that does not send its rows of x_hat in one iteration (HPR_FAULT_BARRIER,
    host-injected) leaves every CTA's wait for that fill to run out of its budget (200 us
    under injection): the solve returns HPR_ERR_DEVICE_TIMEOUT naming the iteration, and the
    context and the GPU stay usable."""
    lp = lpgen.planted_medium(0, 0.005)
    os.environ["HPR_FAULT_BARRIER"] = "5"
    try:
        s = hpr.Solver(lp, persistent=4)
    finally:
        os.environ.pop("HPR_FAULT_BARRIER", None)
    with s:
        with pytest.raises(hpr.HprError) as e:
            s.solve(1e-8)
        assert e.value.code == hpr.HPR_ERR_DEVICE_TIMEOUT
        assert "iteration 4" in str(e.value)
    ref = oracle.solve(lp, tol=1e-8, max_iter=2_000_000)
    res = hpr.solve(lp, tol=1e-8, persistent=4)
    assert res["status"] == hpr.HPR_OK and res["info"]["iters"] == ref["info"]["iters"]


def test_cluster_refused_when_it_cannot_run():
    with hpr.Solver(lpgen.planted_tiny(0), persistent=4, precision=1) as s:
        with pytest.raises(hpr.HprError) as e:
            s.solve(1e-8)
        assert e.value.code == hpr.HPR_ERR_ARG
    lp = lpgen.planted_medium(0, 0.05)               # the replicas alone, (m + n) 8 bytes, are 280 KB
    with hpr.Solver(lp, persistent=4) as s:
        with pytest.raises(hpr.HprError) as e:
            s.solve(1e-8)
        assert e.value.code == hpr.HPR_ERR_ARG and "shared memory" in str(e.value)
