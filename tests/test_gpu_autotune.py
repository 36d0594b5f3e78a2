"""The layout autotuner and explicit layout parameters: whatever sliced-ELL layout a
context uses (lanes per row, work-unit size), its iterates equal the oracle's to 1e-11
over the first 100 iterations and its solves reach the oracle's objective."""
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


LAYOUTS = {
    "autotune": dict(autotune=1),
    "narrow": dict(sell_steps_a=16, sell_steps_t=16, unit_cost_a=32.0, unit_cost_t=32.0),
    "wide": dict(sell_steps_a=128, sell_steps_t=128, unit_cost_a=256.0, unit_cost_t=256.0),
}


@pytest.mark.parametrize("layout", list(LAYOUTS))
def test_layouts_keep_parity(layout):
    lp = lpgen.planted_medium(3, 0.01)
    N = 100
    ref = oracle.solve(lp, max_iter=N, trace_iters=N)
    with hpr.Solver(lp, max_iter=N, trace_iters=N, lambda_fixed=ref["info"]["lambda"], **LAYOUTS[layout]) as s:
        lay = s.layout()
        if layout != "autotune":
            assert lay["sell_steps"] == (LAYOUTS[layout]["sell_steps_a"], LAYOUTS[layout]["sell_steps_t"])
        assert all(v in (16, 24, 40, 64, 128) for v in lay["sell_steps"])
        s.solve(1e-8)
        for k in (0, 9, 49, 99):
            g = s.trace(k)
            for key in ("x", "xhat", "xbar", "y", "ybar"):
                assert rel(g[key], ref["trace"][key][k]) <= 1e-11, (layout, k, key)
    print(layout, lay)


def test_autotuned_solve_matches_oracle():
    lp = lpgen.mcf_lp(2, nodes=300)
    ref = oracle.solve(lp, tol=1e-8, max_iter=200_000)
    with hpr.Solver(lp, autotune=1, lambda_fixed=ref["info"]["lambda"]) as s:
        res = s.solve(1e-8)
        print("chosen layout", s.layout())
    assert res["status"] == hpr.HPR_OK
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    assert abs(res["info"]["primal_obj"] - ref["info"]["pobj"]) <= 1e-7 * abs(ref["info"]["pobj"])



@pytest.mark.parametrize("scale", [0.05, 0.5])
def test_default_layout_follows_phase_traffic(scale):
    """Without layout options a phase whose algorithmic traffic is below 40 MB gets the
    short-slice layout (16 steps, units of 32), a larger one the default (40, 64): at half
    scale the medium LP's x phase (Aᵀ) is above, its y phase (A) below."""
    lp = lpgen.planted_medium(0, scale)
    bx = 12 * lp.nnz + 60 * lp.n + 8 * lp.m
    by = 12 * lp.nnz + 8 * lp.n + 36 * lp.m
    with hpr.Solver(lp) as s:
        lay = s.layout()
    want = lambda b: (16, 32.0) if b < 40e6 else (40, 64.0)
    assert (lay["sell_steps"][0], lay["unit_cost"][0]) == want(by)
    assert (lay["sell_steps"][1], lay["unit_cost"][1]) == want(bx)
