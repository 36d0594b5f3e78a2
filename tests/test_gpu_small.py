"""The persistent single-CTA path (the whole solve in one CTA, iterates in shared memory)
against the oracle: the restart / sigma / termination decision sequence, the power method's
lambda, the final objective and an independently evaluated KKT residual, for the tiny
planted family, the Section 4.2 variants and a small QAP; and its microseconds per
iteration next to the multi-CTA graph path."""
import numpy as np
import pytest

from paper_2408_12179_b300 import hpr, lpgen

pytestmark = pytest.mark.gpu

import oracle
from oracle import kkt as K
from decisions import compare_decisions


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hpr.load()


def _check_sequence(gpu, orc, tol=1e-8, **kw):
    return compare_decisions(gpu, orc, tol, **kw)


@pytest.mark.parametrize("seed", range(4))
def test_persistent_tiny_matches_oracle(seed):
    lp = lpgen.planted_tiny(seed)
    ref = oracle.solve(lp, tol=1e-8, max_iter=200_000)
    with hpr.Solver(lp, persistent=2) as s:
        res = s.solve(1e-8)
        checks = s.checks()
    I = res["info"]
    assert res["status"] == hpr.HPR_OK and I["launches"] <= 3
    assert I["lambda"] == pytest.approx(ref["info"]["lambda"], rel=1e-10)
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    assert abs(I["primal_obj"] - ref["info"]["pobj"]) <= 1e-7 * abs(ref["info"]["pobj"])
    assert abs(ind["pobj"] - lp.planted_objective) <= 1e-7 * abs(lp.planted_objective)
    assert K.in_C(res["x"], lp.l, lp.u) and K.in_D(res["y"], lp.m1)
    _check_sequence(checks, ref["checks"])


@pytest.mark.parametrize("variant", [dict(halpern=0, reflect=0, restart=0, sigma_update=0),
                                     dict(halpern=1, reflect=0, restart=1, sigma_update=1)])
def test_persistent_variants_match_oracle(variant):
    lp = lpgen.planted_tiny(2)
    tol = 1e-6 if not variant["halpern"] else 1e-8
    ref = oracle.solve(lp, tol=tol, max_iter=400_000, **variant)
    with hpr.Solver(lp, persistent=2, max_iter=400_000, lambda_fixed=ref["info"]["lambda"], **variant) as s:
        res = s.solve(tol)
        checks = s.checks()
    assert res["status"] == hpr.HPR_OK
    assert abs(res["info"]["primal_obj"] - ref["info"]["pobj"]) <= 10 * tol * (1 + abs(ref["info"]["pobj"]))
    _check_sequence(checks, ref["checks"], tol=tol, restart=bool(variant["restart"]),
                    sigma_rule=bool(variant["sigma_update"]))


def test_persistent_qap():
    lp = lpgen.qap_lp(2, 6)
    ref = oracle.solve(lp, tol=1e-8, max_iter=400_000)
    with hpr.Solver(lp, persistent=2) as s:
        res = s.solve(1e-8)
    assert res["status"] == hpr.HPR_OK
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    assert abs(res["info"]["primal_obj"] - ref["info"]["pobj"]) <= 1e-7 * max(1.0, abs(ref["info"]["pobj"]))


def test_persistent_refused_when_it_cannot_run():
    lp = lpgen.planted_medium(0, 0.01)               # iterates beyond 200 KB of shared memory
    with hpr.Solver(lp, persistent=2) as s:
        with pytest.raises(hpr.HprError) as e:
            s.solve(1e-8)
        assert e.value.code == hpr.HPR_ERR_ARG
    with hpr.Solver(lpgen.planted_tiny(0), persistent=2, precision=1) as s:
        with pytest.raises(hpr.HprError):
            s.solve(1e-8)


def test_persistent_is_faster_per_iteration():
    """Iterations of the tiny planted LP cost a few microseconds on the multi-CTA graph path
    (two launches each) and well under that in the single CTA (printed)."""
    lp = lpgen.planted_tiny(0)
    out = {}
    for p in (0, 2):
        with hpr.Solver(lp, persistent=p, lambda_fixed=10.0, max_iter=30_000) as s:
            s.solve(1e-30)                            # warm-up (graph capture)
            I = s.solve(1e-30)["info"]
        out[p] = 1e6 * I["solve_time_s"] / I["iters"]
    print(f"us per iteration: multi-CTA graph path {out[0]:.2f}, single CTA {out[2]:.2f}")
    assert out[2] < out[0]


def test_default_path_choice():
    """persistent = 1 takes the single CTA for the tiny planted LP, the persistent cluster path
    for a medium planted LP at 1/200 scale (its FP64 work per iteration is beyond what one SM
    does faster, and it fits in the cluster's shared memory) and the multi-CTA path at 1/20
    scale (it does not fit); persistent = 2 still runs the 1/200 LP in one CTA, to the same
    iterates' quality (hpr_info.path names the path taken)."""
    with hpr.Solver(lpgen.planted_tiny(0), persistent=1) as s:
        I = s.solve(1e-8)["info"]
        assert I["launches"] <= 3 and I["path"] == 2 and I["path_ctas"] == 0
    lp = lpgen.planted_medium(0, 0.005)
    res = {}
    for p, path in ((1, 4), (2, 2), (0, 0)):
        with hpr.Solver(lp, persistent=p, max_iter=1500) as s:
            r = s.solve(1e-8)
        assert r["info"]["path"] == path and (r["info"]["launches"] <= 3) == (path != 0)
        assert (r["info"]["path_ctas"] > 1) == (path == 4)
        res[p] = r
    assert res[0]["info"]["iters"] == res[1]["info"]["iters"] == res[2]["info"]["iters"] == 1500
    assert res[2]["info"]["kkt"] == pytest.approx(res[1]["info"]["kkt"], rel=1e-3)
    with hpr.Solver(lpgen.planted_medium(0, 0.05), persistent=1, max_iter=300) as s:
        assert s.solve(1e-8)["info"]["path"] == 0
