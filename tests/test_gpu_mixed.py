"""The FP32 form (precision 1): FP32 matrix values and FP32 iterates x, x_hat, y with
double-float row accumulation, FP64 anchors / data / checks / power method, then FP64
iterates from the first check with KKT < switch_tol.  Its results are compared with the
FP64 oracle; the error of each stage is asserted and printed."""
import numpy as np
import pytest

from paper_2408_12179_b300 import hpr, lpgen
import oracle
from oracle import kkt as K

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hpr.load()


@pytest.mark.parametrize("name", ["tiny", "medium_1e-2"])
def test_fp32_phase_iterates_close_to_fp64_oracle(name):
    """Without the switch, the FP32-form iterates stay within FP32 rounding of the FP64
    oracle's over the first 100 iterations (relative error printed)."""
    lp = lpgen.planted_tiny(0) if name == "tiny" else lpgen.planted_medium(0, 0.01)
    N = 100
    ref = oracle.solve(lp, max_iter=N, trace_iters=N)
    lam = ref["info"]["lambda"]
    worst = 0.0
    with hpr.Solver(lp, max_iter=N, trace_iters=N, lambda_fixed=lam, precision=1, switch_tol=0.0) as s:
        info = s.solve(1e-8)["info"]
        assert info["iters_fp32"] == N
        for k in (0, 9, 49, 99):
            g = s.trace(k)
            for key in ("x", "y", "xbar", "ybar"):
                e = rel(g[key], ref["trace"][key][k])
                worst = max(worst, e)
                assert e <= 2e-5, (k, key, e)
    print(f"{name}: worst relative error of FP32-form iterates vs FP64 oracle over 100 iterations: {worst:.2e}")


@pytest.mark.parametrize("name", ["tiny", "medium_1e-2"])
def test_fp32_normal_iterations_close_to_fp64_oracle(name):
    """The FP32 form's normal iterations (FP32 epilogue arithmetic, no tracing: a traced
    iteration takes the FP64 check-mode epilogue) over 100 iterations without the switch:
    the w_bar returned at the cap against the FP64 oracle's, within FP32 rounding."""
    lp = lpgen.planted_tiny(0) if name == "tiny" else lpgen.planted_medium(0, 0.01)
    N = 100
    ref = oracle.solve(lp, max_iter=N)
    lam = ref["info"]["lambda"]
    res = hpr.solve(lp, tol=1e-12, max_iter=N, lambda_fixed=lam, precision=1, switch_tol=0.0, persistent=0)
    assert res["status"] == hpr.HPR_MAX_ITER and res["info"]["iters_fp32"] == N
    errs = {key: rel(res[key], ref[key]) for key in ("x", "y", "z")}
    print(f"{name}: FP32-form normal iterations, relative error of w_bar after {N} iterations: {errs}")
    for key in ("x", "y"):
        assert errs[key] <= 2e-5, (key, errs[key])


@pytest.mark.parametrize("seed", range(4))
def test_switch_form_solves_tiny(seed):
    lp = lpgen.planted_tiny(seed)
    ref = oracle.solve(lp, tol=1e-8, max_iter=200_000)
    res = hpr.solve(lp, tol=1e-8, precision=1)
    assert res["status"] == hpr.HPR_OK
    I = res["info"]
    assert 0 < I["iters_fp32"] < I["iters"]
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    e = abs(I["primal_obj"] - ref["info"]["pobj"]) / abs(ref["info"]["pobj"])
    assert e <= 1e-7
    assert K.in_C(res["x"], lp.l, lp.u) and K.in_D(res["y"], lp.m1)
    print(f"seed {seed}: objective error vs FP64 oracle {e:.1e}, iterations {I['iters']} "
          f"(FP32 {I['iters_fp32']}) vs oracle {ref['info']['iters']}")


def test_switch_form_solves_medium_small_scale():
    lp = lpgen.planted_medium(0, 0.01)
    ref = oracle.solve(lp, tol=1e-8, max_iter=400_000)
    res = hpr.solve(lp, tol=1e-8, precision=1)
    assert res["status"] == hpr.HPR_OK
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    e = abs(res["info"]["primal_obj"] - ref["info"]["pobj"]) / abs(ref["info"]["pobj"])
    assert e <= 1e-7
    print(f"medium/100: objective error vs FP64 oracle {e:.1e}; iterations {res['info']['iters']} "
          f"(FP32 {res['info']['iters_fp32']}) vs oracle {ref['info']['iters']}")


def test_switch_happens_at_first_check_below_tolerance():
    lp = lpgen.planted_tiny(5)
    with hpr.Solver(lp, precision=1, switch_tol=1.0) as s:
        res = s.solve(1e-8)
        checks = s.checks()
    first_check = [c for c in checks if int(c["kind"]) & 1][0]
    assert first_check["kkt"] < 1.0
    assert res["info"]["iters_fp32"] == int(first_check["k"]) + 1
    assert res["status"] == hpr.HPR_OK
