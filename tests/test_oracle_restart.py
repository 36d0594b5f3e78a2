"""Pins of the oracle's restart and sigma decisions (Section 3.1, Algorithm 2, Algorithm 3).

The paper prints no decision trace, so these tests rebuild every decision from quantities
that are pinned elsewhere or recomputed here, and from the paper's statement of the rules:

* the merit R~ = ||w - w_hat||_M is recomputed from the traced iterates with M built
  densely from its block definition (eq. def:M, T1 = lambda I - A A^*) wherever the run is
  traced, and equals the recorded value there;
* R~_{r,0} is the merit of the first iteration of inner loop r, and "R~ at the previous
  check" is the merit recorded at the previous check of the same inner loop: both are taken
  from the sequence of records, not from the oracle's internal variables;
* criteria (restart_1)-(restart_3) with alpha = (0.2, 0.6, 0.2) (Section 4.1), tested after
  Algorithm 2 has advanced t and k ("t = t + 1, k = k + 1" precedes "until one of the
  restart criteria holds"), so criterion 3 reads t+1 >= alpha3 (k+1) with the counters of
  the iteration that ends at the check; a restart's cause is the first criterion that holds
  in the order printed; termination is tested first;
* Algorithm 3 with eq. (sigma_T1!=0): Delta_x = ||x_bar - x0||, Delta_y = sqrt(lambda)
  ||y_bar - y0|| recomputed from the traced iterates and anchors.

The runs are chosen so that every discriminating situation occurs: a check between
alpha1 R~_0 and alpha2 R~_0 without a restart (an alpha1 / alpha2 swap restarts there),
criterion 2 alone (testing it against R~_{r,0} instead of the previous merit never fires),
criterion 3 alone where the pre-increment counters t >= alpha3 k would not fire, and two
criteria at once (the cause shows the order).  ``test_planted_misreadings_fail`` plants each
of those misreadings in a copy of the oracle's C source and checks that the decision
rebuild rejects it.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

from paper_2408_12179_b300 import lpgen

ALPHA = (0.2, 0.6, 0.2)
ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                          "hpr_oracle.c")

# (LP, check period, iterations traced): a medium planted LP at 1/500 scale (m = 400,
# n = 1,000, ~10k nonzeros) checked every 10 iterations shows every situation listed above;
# the tiny planted LP checked every 40 iterations has both criteria 1 and 3 at its first check
RUNS = {
    "medium/500": (lambda: lpgen.planted_medium(0, 0.002), 10, 1500),
    "tiny": (lambda: lpgen.planted_tiny(0), 40, 600),
}


def _scaled_A(orc, lp, res):
    import scipy.sparse as sp

    A = lp.A
    return sp.csr_matrix((res["scaled"]["As"], A.indices, A.indptr), shape=A.shape)


def _merit(A, sigma, lam, dy, dx):
    """2 ||(dy, dz, dx)||_M with M of eq. def:M (z block zero) built densely."""
    m, n = A.shape
    Ad = A.toarray()
    T1 = lam * np.eye(m) - Ad @ Ad.T
    M = np.zeros((m + n, m + n))
    M[:m, :m] = sigma * (Ad @ Ad.T) + sigma * T1
    M[:m, m:] = Ad
    M[m:, :m] = Ad.T
    M[m:, m:] = np.eye(n) / sigma
    d = np.concatenate([dy, dx])
    return 2.0 * math.sqrt(max(d @ M @ d, 0.0))


def rebuild_decisions(checks, alpha=ALPHA, tol=0.0):
    """Walk the oracle's check records and rebuild every decision from the rules of
    Section 3.1.  Returns (mismatches, events): a list of records whose restart, cause or
    counters disagree with the rules, and counts of the discriminating situations."""
    a1, a2, a3 = alpha
    bad, ev = [], dict(between=0, c2_alone=0, c3_alone_shifted=0, two_at_once=0, restarts=0)
    R0 = Rprev = None
    prev = None                   # (k, r, t, restarted) of the previous record
    for i, c in enumerate(checks):
        k, r, t, kind = int(c["k"]), int(c["r"]), int(c["t"]), int(c["kind"])
        if prev is not None:      # counters: a restart opens inner loop r+1 at the next iteration
            pk, pr, pt, restarted = prev
            if restarted and ((k, r, t) != (pk + 1, pr + 1, 0) or not kind & 2):
                bad.append((i, "no new inner loop after a restart", (k, r, t)))
            if not restarted and (r != pr or t - pt != k - pk):
                bad.append((i, "counters", (k, r, t), (pk, pr, pt)))
        if kind & 2:                               # first iteration of an inner loop
            if t != 0:
                bad.append((i, "R0 record with t != 0"))
            R0 = Rprev = c["Rt"]
            if c["R0"] != R0:
                bad.append((i, "R0 field"))
        prev = (k, r, t, False)
        if not kind & 1:
            continue
        if c["kkt"] <= tol:
            if c["cause"] != -1:
                bad.append((i, "termination"))
            break
        if kind & 2:                               # a check at t = 0 tests no criterion
            if c["cause"] != 0:
                bad.append((i, "restart at t = 0"))
            continue
        Rt = c["Rt"]
        h1 = Rt <= a1 * R0
        h2 = Rt <= a2 * R0 and Rt > Rprev
        h3 = (t + 1) >= a3 * (k + 1)
        cause = 1 if h1 else 2 if h2 else 3 if h3 else 0
        if int(c["cause"]) != cause:
            bad.append((i, "cause", int(c["cause"]), cause, k))
        if a1 * R0 < Rt <= a2 * R0 and not h2 and not h3:
            ev["between"] += 1
        if h2 and not h3:
            ev["c2_alone"] += 1
        if h3 and not h1 and not h2 and not (t >= a3 * k):
            ev["c3_alone_shifted"] += 1
        if int(h1) + int(h2) + int(h3) >= 2:
            ev["two_at_once"] += 1
        Rprev = Rt
        if cause:
            ev["restarts"] += 1
            prev = (k, r, t, True)
    return bad, ev


def _check_sigma_and_merit(orc, lp, res, traced):
    """Merit of every traced check against eq. def:M, sigma after every traced restart
    against Algorithm 3 with eq. (sigma_T1!=0), and the sigma of the next inner loop."""
    A = _scaled_A(orc, lp, res)
    lam = res["info"]["lambda"]
    tr = res["trace"]
    n, m = lp.n, lp.m
    x0, y0 = np.zeros(n), np.zeros(m)
    checked = restarts = 0
    for i, c in enumerate(res["checks"]):
        k = int(c["k"])
        if k >= traced - 1 or k >= res["info"]["iters"] - 1:
            break
        xprev = tr["x"][k - 1] if k > 0 else np.zeros(n)
        yprev = tr["y"][k - 1] if k > 0 else np.zeros(m)
        R = _merit(A, c["sigma"], lam, yprev - tr["ybar"][k], xprev - tr["xbar"][k])
        assert c["Rt"] == pytest.approx(R, rel=1e-8, abs=1e-14), (k, c["kind"])
        checked += 1
        if c["cause"] > 0:
            Dx = float(np.linalg.norm(tr["xbar"][k] - x0))
            Dy = math.sqrt(lam) * float(np.linalg.norm(tr["ybar"][k] - y0))
            ratio = c["err_d"] / c["err_p"] if c["err_p"] > 0 else math.inf
            ok = 1e-16 < Dx < 1e12 and 1e-16 < Dy < 1e12 and c["err_p"] > 0 and 1e-8 < ratio < 1e8
            assert c["sigma_next"] == pytest.approx(Dx / Dy if ok else 1.0, rel=1e-10), k
            nxt = res["checks"][i + 1]
            assert nxt["sigma"] == c["sigma_next"] and int(nxt["kind"]) & 2
            x0, y0 = tr["xbar"][k].copy(), tr["ybar"][k].copy()   # the new anchors
            restarts += 1
    return checked, restarts


@pytest.mark.parametrize("name", list(RUNS))
def test_restart_decisions_follow_section_3_1(orc, name):
    make, every, traced = RUNS[name]
    lp = make()
    res = orc.solve(lp, tol=1e-9, max_iter=20_000, check_every=every, trace_iters=traced)
    bad, ev = rebuild_decisions(res["checks"], tol=1e-9)
    assert not bad, bad[:5]
    checked, restarts = _check_sigma_and_merit(orc, lp, res, traced)
    assert checked >= 20 and restarts >= 3
    if name == "medium/500":
        assert ev["between"] >= 5 and ev["c2_alone"] >= 3 and ev["c3_alone_shifted"] >= 2, ev
    else:
        assert ev["two_at_once"] >= 1, ev


# ------------------------------------------------------------------ planted misreadings
# Each replaces the oracle's restart test by a plausible misreading of Section 3.1.
_CRIT = ("if (Rt <= O->alpha1 * R0) cause = 1;\n"
         "                else if (Rt <= O->alpha2 * R0 && Rt > Rprev) cause = 2;\n"
         "                else if ((double)(t + 1) >= O->alpha3 * (double)(k + 1)) cause = 3;")
MISREADINGS = {
    "alpha1 and alpha2 swapped": _CRIT.replace("alpha1", "ALPHA_A").replace("alpha2", "alpha1")
                                     .replace("ALPHA_A", "alpha2"),
    "criterion 2 against R~_{r,0}": _CRIT.replace("Rt > Rprev", "Rt > R0"),
    "criterion 3 before the counters advance": _CRIT.replace(
        "(double)(t + 1) >= O->alpha3 * (double)(k + 1)", "(double)t >= O->alpha3 * (double)k"),
    "criterion 3 tested first": (
        "if ((double)(t + 1) >= O->alpha3 * (double)(k + 1)) cause = 3;\n"
        "                else if (Rt <= O->alpha1 * R0) cause = 1;\n"
        "                else if (Rt <= O->alpha2 * R0 && Rt > Rprev) cause = 2;"),
}


def _build_mutant(tmp_path, name, text):
    src = open(ORACLE_SRC).read()
    assert src.count(_CRIT) == 1, "the oracle's restart test moved: update _CRIT"
    path = tmp_path / ("mut_%d.c" % list(MISREADINGS).index(name))
    path.write_text(src.replace(_CRIT, text))
    lib = tmp_path / (path.stem + ".so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-o", str(lib), str(path), "-lm"], check=True)
    return str(lib)


def test_planted_misreadings_fail(orc, tmp_path):
    """Every misreading above changes at least one rebuilt decision on one of the runs."""
    good = orc.lib()
    for name, text in MISREADINGS.items():
        mut = ctypes.CDLL(_build_mutant(tmp_path, name, text))
        mut.orc_hpr.argtypes = good.orc_hpr.argtypes
        mut.orc_hpr.restype = ctypes.c_int
        caught = False
        try:
            orc._lib = mut
            for key, (make, every, _) in RUNS.items():
                res = orc.solve(make(), tol=1e-9, max_iter=20_000, check_every=every)
                bad, _ = rebuild_decisions(res["checks"], tol=1e-9)
                caught = caught or bool(bad)
        finally:
            orc._lib = good
        assert caught, name
