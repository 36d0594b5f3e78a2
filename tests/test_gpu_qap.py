"""The QAP workload (Adams-Johnson linearisation with random flow / distance matrices) on
the CUDA path against the oracle: the first 100 iterates and full solves."""
import numpy as np
import pytest

from paper_2408_12179_b300 import hpr, lpgen

pytestmark = pytest.mark.gpu

import oracle
from oracle import kkt as K


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hpr.load()


def test_qap_first_100_iterates():
    lp = lpgen.qap_lp(1, 7)
    N = 100
    ref = oracle.solve(lp, max_iter=N, trace_iters=N)
    with hpr.Solver(lp, max_iter=N, trace_iters=N, lambda_fixed=ref["info"]["lambda"]) as s:
        s.solve(1e-8)
        for k in range(N):
            g = s.trace(k)
            for key in ("x", "xhat", "xbar", "y", "ybar"):
                assert rel(g[key], ref["trace"][key][k]) <= 1e-11, (k, key)


@pytest.mark.parametrize("N,precision", [(5, 0), (6, 0), (6, 1)])
def test_qap_full_solve(N, precision):
    lp = lpgen.qap_lp(2, N)
    ref = oracle.solve(lp, tol=1e-8, max_iter=400_000)
    assert ref["info"]["status"] == 0
    with hpr.Solver(lp, lambda_fixed=ref["info"]["lambda"], precision=precision) as s:
        res = s.solve(1e-8)
    assert res["status"] == hpr.HPR_OK
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    assert abs(res["info"]["primal_obj"] - ref["info"]["pobj"]) <= 1e-7 * max(1.0, abs(ref["info"]["pobj"]))
    assert K.in_C(res["x"], lp.l, lp.u)
    print(f"N={N} precision {precision}: iterations {res['info']['iters']} vs oracle {ref['info']['iters']}")
