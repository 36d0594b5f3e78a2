"""Checkpoint / resume (hpr_get_state, hpr_set_state) on the multi-CTA path: a solve stopped
by max_iter and resumed, in a fresh context of the same LP, from its checkpoint (the last
restart of Algorithm 2: anchor, sigma, counters, lambda) ends bit for bit where the
uninterrupted solve ends -- same iterations, restarts and w_bar -- in FP64 and in the FP32
form; misuse is refused."""
import numpy as np
import pytest

from paper_2408_12179_b300 import hpr, lpgen

pytestmark = pytest.mark.gpu

import oracle
from oracle import kkt as K


def _same(a, b):
    for key in ("iters", "restarts", "power_iters", "lambda", "primal_obj", "dual_obj", "kkt", "sigma"):
        assert a["info"][key] == b["info"][key], (key, a["info"][key], b["info"][key])
    for key in ("x", "y", "z"):
        assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("name,lp_fn,opts,cut", [
    ("tiny0", lambda: lpgen.planted_tiny(0), {}, 400),
    ("medium/200", lambda: lpgen.planted_medium(0, 0.005), {}, 10_000),
    ("tiny1 FP32 form", lambda: lpgen.planted_tiny(1), {"precision": 1}, 600),
])
def test_resume_replays_the_uninterrupted_solve(name, lp_fn, opts, cut):
    lp = lp_fn()
    with hpr.Solver(lp, persistent=0, **opts) as s:
        full = s.solve(1e-8)
    assert full["status"] == hpr.HPR_OK and full["info"]["iters"] > cut
    # (the cut solve also checks at its last iteration: cuts on the check schedule, or
    # where the residual is still above tol, stop with HPR_MAX_ITER)
    with hpr.Solver(lp, persistent=0, max_iter=cut, **opts) as s:
        part = s.solve(1e-8)
        blob = s.get_state()
    assert part["status"] == hpr.HPR_MAX_ITER and part["info"]["iters"] == cut
    with hpr.Solver(lp, persistent=1, **opts) as s:       # persistent 1: the resume takes the multi-CTA path
        s.set_state(blob)
        resumed = s.solve(1e-8)
        assert resumed["info"]["path"] == 0 and resumed["info"]["power_iters"] == full["info"]["power_iters"]
        _same(resumed, full)
        again = s.solve(1e-8)                                # the state is used once
        assert again["info"]["path"] in (0, 2, 4)
    ind = K.kkt(lp, resumed["x"], resumed["y"], resumed["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    print(f"{name}: stopped at {cut}, resumed to {resumed['info']['iters']} iterations, "
          f"{resumed['info']['restarts']} restarts, equal to the uninterrupted solve")


def test_state_misuse_is_refused():
    lp, other = lpgen.planted_tiny(0), lpgen.planted_tiny(1)
    with hpr.Solver(lp, persistent=0, max_iter=300) as s:
        with pytest.raises(hpr.HprError) as e:
            s.get_state()                                    # no solve yet
        assert e.value.code == hpr.HPR_ERR_STATE
        s.solve(1e-8)
        blob = s.get_state()
    with hpr.Solver(lp, persistent=2) as s:
        s.solve(1e-8)
        with pytest.raises(hpr.HprError) as e:
            s.get_state()                                    # anchors of a persistent path stay on chip
        assert e.value.code == hpr.HPR_ERR_STATE
    with hpr.Solver(other, persistent=0) as s:
        with pytest.raises(hpr.HprError) as e:
            s.set_state(blob)                                # another LP
        assert e.value.code == hpr.HPR_ERR_ARG
    with hpr.Solver(lp, persistent=0) as s:
        for bad in (blob[:100], b"x" * len(blob)):
            with pytest.raises(hpr.HprError) as e:
                s.set_state(bad)
            assert e.value.code == hpr.HPR_ERR_ARG
        s.set_state(blob)
        s.set_options(persistent=2)
        with pytest.raises(hpr.HprError) as e:
            s.solve(1e-8)                                    # a resume runs on the multi-CTA path only
        assert e.value.code == hpr.HPR_ERR_ARG
