"""Error paths of the C ABI, driven by host-side faults only (no GPU is faulted).

* allocation failure: HPR_FAULT_ALLOC=n makes the n-th allocation of a context report
  out-of-memory; every n up to the number of allocations a create + solve makes must give
  HPR_ERR_NOMEM from hpr_create or hpr_solve, leave nothing behind (the context, if one
  exists, destroys cleanly), and a normal solve afterwards must still be right;
* non-finite residual: HPR_FAULT_NAN_CHECK=n poisons the n-th check period's read-back
  scalars: HPR_ERR_NUMERIC, and the same context solves normally afterwards;
* time limit (Section 4.1 runs have time limits): HPR_TIME_LIMIT with the last w_bar
  retrievable, x in C and y in D.
"""
import os

import numpy as np
import pytest

from paper_2408_12179_b300 import hpr, lpgen

pytestmark = pytest.mark.gpu

import oracle
from oracle import kkt as K


@pytest.fixture(autouse=True)
def _clean_env():
    for key in ("HPR_FAULT_ALLOC", "HPR_FAULT_NAN_CHECK"):
        os.environ.pop(key, None)
    yield
    for key in ("HPR_FAULT_ALLOC", "HPR_FAULT_NAN_CHECK"):
        os.environ.pop(key, None)


@pytest.mark.parametrize("persistent", [0, 2])
def test_every_allocation_failure_is_reported(persistent):
    lp = lpgen.planted_tiny(1)
    opts = dict(persistent=persistent, trace_iters=0 if persistent else 5)
    failures = 0
    for n in range(1, 400):
        os.environ["HPR_FAULT_ALLOC"] = str(n)
        s = None
        try:
            s = hpr.Solver(lp, **opts)
            s.solve(1e-8)
        except hpr.HprError as e:
            assert e.code == hpr.HPR_ERR_NOMEM, (n, e)
            assert "HPR_FAULT_ALLOC" in str(e), (n, e)
            failures += 1
            continue
        finally:
            if s is not None:
                s.close()
        break                                        # n beyond the last allocation
    else:
        pytest.fail("the allocation count never ran out")
    assert failures >= 10
    os.environ.pop("HPR_FAULT_ALLOC")
    ref = oracle.solve(lp, tol=1e-8)
    res = hpr.solve(lp, tol=1e-8, **opts)
    assert res["status"] == hpr.HPR_OK
    assert abs(res["info"]["primal_obj"] - ref["info"]["pobj"]) <= 1e-7 * abs(ref["info"]["pobj"])


def test_non_finite_residual_is_reported():
    lp = lpgen.planted_medium(0, 0.005)
    os.environ["HPR_FAULT_NAN_CHECK"] = "3"
    with hpr.Solver(lp, persistent=0) as s:
        os.environ.pop("HPR_FAULT_NAN_CHECK")
        with pytest.raises(hpr.HprError) as e:
            s.solve(1e-8)
        assert e.value.code == hpr.HPR_ERR_NUMERIC
        assert "non-finite" in str(e.value)
        res = s.solve(1e-8)                          # the context is still usable
        assert res["status"] == hpr.HPR_OK
        ind = K.kkt(lp, res["x"], res["y"], res["z"])
        assert ind["kkt"] <= 1e-8 * (1 + 1e-6)


def test_time_limit_returns_the_last_iterate():
    lp = lpgen.planted_medium(1, 0.01)
    with hpr.Solver(lp, persistent=0, time_limit_s=1e-6) as s:
        res = s.solve(1e-8)
        checks = s.checks()
    assert res["status"] == hpr.HPR_TIME_LIMIT
    info = res["info"]
    assert info["status"] == hpr.HPR_TIME_LIMIT and 0 < info["iters"] <= 150
    assert K.in_C(res["x"], lp.l, lp.u) and K.in_D(res["y"], lp.m1)
    last = [c for c in checks if int(c["kind"]) & 1][-1]
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] == pytest.approx(last["kkt"], rel=1e-6)   # the returned point is the checked w_bar
    assert np.all(np.isfinite(res["z"]))
