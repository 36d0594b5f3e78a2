"""Comparison of the CUDA solver's check records with the oracle's (test helper).

Two things are checked over the WHOLE sequence of records of a solve:

1. the CUDA solver's own decisions follow the rules of Section 3.1 and Algorithm 3 from its
   own recorded values: criteria (restart_1)-(restart_3) with alpha = (0.2, 0.6, 0.2) tested
   after Algorithm 2 advances t and k, causes in the printed order, termination first, and
   sigma = Delta_x / Delta_y (eq. sigma_T1!=0) when Delta_x, Delta_y lie in (1e-16, 1e12) and
   err_d / err_p in (1e-8, 1e8), else 1;
2. the two solvers take the same decisions at the same checks, and their check values agree
   to a relative `tol_rel`, until the first check where they decide differently.  There the
   difference must be explained: for the criterion whose outcome differs, the two solvers'
   own values lie on opposite sides of its threshold, within `tol_rel` of it (the solvers
   round differently, so a near-tie may fall either way).  Records after that point are not
   compared (the runs have parted).

Returns the index of the first divergence (or the number of records compared).
"""
from __future__ import annotations

import pytest

ALPHA = (0.2, 0.6, 0.2)


def _margins(rec, R0, Rprev, alpha=ALPHA):
    """Signed distances to the thresholds of (restart_1), both parts of (restart_2) and
    (restart_3); a criterion holds when its margins are <= 0 (part b of (restart_2): < 0)."""
    a1, a2, a3 = alpha
    Rt = rec["Rt"]
    return dict(c1=Rt - a1 * R0, c2a=Rt - a2 * R0, c2b=Rprev - Rt,
                c3=a3 * (rec["k"] + 1) - (rec["t"] + 1))


def _cause(mg):
    if mg["c1"] <= 0:
        return 1
    if mg["c2a"] <= 0 and mg["c2b"] < 0:
        return 2
    if mg["c3"] <= 0:
        return 3
    return 0


def _walk(recs, tol, max_iter, restart=True):
    """Per record: (cause rebuilt from the rules, margins or None)."""
    out = []
    R0 = Rprev = None
    for c in recs:
        kind = int(c["kind"])
        if kind & 2:
            R0 = Rprev = c["Rt"]
        if not kind & 1:
            out.append((0, None))
            continue
        if c["kkt"] <= tol:
            out.append((-1, None))
            continue
        if kind & 2 or int(c["k"]) + 1 >= max_iter or not restart:   # no restart test at t = 0,
            # at the cap, or with the restarts switched off (Section 4.2 ablation)
            out.append((0, None))
            continue
        mg = _margins(c, R0, Rprev)
        out.append((_cause(mg), mg))
        Rprev = c["Rt"]
    return out


def _sigma_ok(c):
    Dx, Dy, ep, ed = c["Dx"], c["Dy"], c["err_p"], c["err_d"]
    rule = 1e-16 < Dx < 1e12 and 1e-16 < Dy < 1e12 and ep > 0 and 1e-8 < ed / ep < 1e8
    want = Dx / Dy if rule else 1.0
    return c["sigma_next"] == pytest.approx(want, rel=1e-12)


def compare_decisions(gpu, orc, tol, tol_rel=1e-6, sigma_rule=True, max_iter=1 << 62, restart=True):
    assert len(gpu) > 0 and len(orc) > 0
    gw = _walk(gpu, tol, max_iter, restart)
    for i, (c, (cause, _)) in enumerate(zip(gpu, gw)):      # 1. the GPU's own decisions
        assert int(c["cause"]) == cause, ("GPU decision against its own values", i, c)
        if cause > 0 and sigma_rule:
            assert _sigma_ok(c), ("GPU sigma", i, c)
    ow = _walk(orc, tol, max_iter, restart)
    n = min(len(gpu), len(orc))
    for i in range(n):                                       # 2. GPU against the oracle
        g, o = gpu[i], orc[i]
        assert (int(g["k"]), int(g["kind"]), int(g["r"]), int(g["t"])) == \
               (int(o["k"]), int(o["kind"]), int(o["r"]), int(o["t"])), (i, g, o)
        if int(g["cause"]) != int(o["cause"]):
            if -1 in (int(g["cause"]), int(o["cause"])):      # termination at a near-tie
                assert abs(o["kkt"] - tol) <= 2 * tol_rel * tol, ("termination decided differently", i, g, o)
                return i
            (_, gm), (_, om) = gw[i], ow[i]
            scale = max(abs(o["R0"]), abs(o["Rt"]), 1e-300)
            straddle = [key for key in gm
                        if (gm[key] <= 0) != (om[key] <= 0) and abs(om[key]) <= 2 * tol_rel * scale]
            assert straddle, ("divergence not at a near-tie", i, g, o)
            return i
        for key in ("err_p", "err_d", "pobj", "dobj", "Rt"):
            if int(g["kind"]) & 1 or key == "Rt":
                assert g[key] == pytest.approx(o[key], rel=tol_rel, abs=1e-13), (i, key, g[key], o[key])
        if int(g["kind"]) & 1:
            # the relative gap |dobj - pobj| / (1 + |pobj| + |dobj|) cancels: its disagreement is
            # bounded by the objectives' own disagreement (checked just above), not by its size
            den = 1.0 + abs(o["pobj"]) + abs(o["dobj"])
            bound = 2.0 * (abs(g["pobj"] - o["pobj"]) + abs(g["dobj"] - o["dobj"])) / den + 1e-13
            assert abs(g["err_gap"] - o["err_gap"]) <= bound, (i, "err_gap", g["err_gap"], o["err_gap"], bound)
        if int(g["cause"]) > 0:
            assert g["sigma_next"] == pytest.approx(o["sigma_next"], rel=tol_rel), (i, g, o)
    assert len(gpu) == len(orc), "one solver stopped earlier without a divergent decision"
    return n
