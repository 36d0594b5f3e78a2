"""The min-cost multicommodity-flow workload (random geometric k-NN digraph, 4 commodities,
shared arc capacities) on the CUDA path against the oracle: first iterates at small scale
and at the full size (1M nodes, 8M arcs, n = 32M, nnz = 96M; two iterations, the oracle
computing the same two), full solves at small scale in the FP64 and the FP32 switch forms."""
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


def _compare_trace(lp, N, tol=1e-11, **opts):
    ref = oracle.solve(lp, max_iter=N, trace_iters=N, **opts)
    lam = ref["info"]["lambda"]
    opts = dict(opts)
    opts["lambda_fixed"] = lam
    with hpr.Solver(lp, max_iter=N, trace_iters=N, **opts) as s:
        s.solve(1e-8)
        for k in range(N):
            g = s.trace(k)
            for key in ("x", "xhat", "xbar", "y", "ybar"):
                r_ = ref["trace"][key][k]
                assert rel(g[key], r_) <= tol, (k, key, rel(g[key], r_))


def test_mcf_first_100_iterates():
    _compare_trace(lpgen.mcf_lp(1, nodes=1000), 100)


def test_mcf_full_size_first_iterations():
    """Full size: 32M columns, 12M rows, 96M nonzeros, with lambda fixed (the oracle's
    power method would take hours here); the sliced-ELL layouts and grids are the
    ones the benchmark times."""
    lp = lpgen.mcf_lp(0)
    assert lp.nnz == 96_000_000
    _compare_trace(lp, 2, lambda_fixed=1.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_mcf_small_full_solve(precision):
    lp = lpgen.mcf_lp(0, nodes=300)
    ref = oracle.solve(lp, tol=1e-8, max_iter=200_000)
    assert ref["info"]["status"] == 0
    with hpr.Solver(lp, lambda_fixed=ref["info"]["lambda"], precision=precision) as s:
        res = s.solve(1e-8)
    assert res["status"] == hpr.HPR_OK
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    e = abs(res["info"]["primal_obj"] - ref["info"]["pobj"]) / abs(ref["info"]["pobj"])
    assert e <= 1e-7
    assert K.in_C(res["x"], lp.l, lp.u) and K.in_D(res["y"], lp.m1)
    print(f"precision {precision}: objective error vs FP64 oracle {e:.1e}, iterations "
          f"{res['info']['iters']} (FP32 {res['info']['iters_fp32']}) vs oracle {ref['info']['iters']}")
