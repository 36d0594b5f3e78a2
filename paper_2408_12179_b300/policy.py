"""The learned sigma policy: training data from HPR's own traces, training and evaluation.

At a restart where Algorithm 3 computes sigma = Delta_x / Delta_y, the policy may scale it
by 2^((a-2)/2), a = 0..4.  Its network (the CUDA kernels behind ``hpr.mlp_*``) maps 64
features of the last 16 checks (``Solver.policy_features``) to five predicted outcomes,
one per multiplier; the solver takes the smallest (``sigma_policy = 2``), and falls back to
Algorithm 3's value at the next restart whenever a learned choice was followed by a KKT
residual above the one at the decision.

Data: solves with ``sigma_policy = 1`` draw the multiplier at random (SplitMix64 from
``policy_seed``); every such restart becomes a sample (features, action, outcome) with
outcome = log10 KKT at the `horizon`-th periodic check after the decision (or at the end
of the solve) minus log10 KKT at the decision: lower is better.

``python -m paper_2408_12179_b300.policy eval weights.npy n_eval n_large margin...`` only
evaluates given weights, once per margin (``policy_margin``).
``python -m paper_2408_12179_b300.policy [n_train n_eval weights.npy n_large [large_scale]]``
trains on seeded small instances of the medium planted and multicommodity-flow families and
evaluates on held-out ones of the same sizes and on `n_large` held-out medium planted LPs
at scale `large_scale` (default 0.05: 25k columns) (one GPU), printing one JSON line with a
95% bootstrap interval of the geometric-mean iteration ratio.
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np

from . import hpr, lpgen

HORIZON = 8
FLOOR = 1e-12


def init_weights(seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, in the network's layout."""
    rng = np.random.default_rng([0x7EA1, seed])
    parts = []
    for rows, cols in ((64, 64), (64, 64), (64, 64), (5, 64)):
        parts.append((rng.standard_normal((rows, cols)) * math.sqrt(2.0 / cols)).ravel())
        parts.append(np.zeros(rows))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == hpr.mlp_param_count()
    return w


def samples_from_solve(solver, horizon: int = HORIZON):
    """(X, actions, outcomes) of the exploring restarts of the solver's last solve."""
    recs = solver.checks()
    checks = [i for i, r in enumerate(recs) if int(r["kind"]) & 1]
    X, A, Y = [], [], []
    for pos, i in enumerate(checks):
        r = recs[i]
        if int(r["cause"]) <= 0 or int(r["action"]) < 0:
            continue
        j = checks[min(pos + horizon, len(checks) - 1)]
        k0 = max(float(r["kkt"]), FLOOR)
        k1 = max(float(recs[j]["kkt"]), FLOOR)
        X.append(solver.policy_features(i))
        A.append(int(r["action"]))
        Y.append(math.log10(k1) - math.log10(k0))
    return X, A, Y


def collect(lps, seeds, max_iter=400_000, tol=1e-8):
    X, A, Y = [], [], []
    for lp in lps:
        with hpr.Solver(lp, sigma_policy=1, max_iter=max_iter) as s:
            for sd in seeds:
                s.set_options(policy_seed=int(sd))
                s.solve(tol)
                x, a, y = samples_from_solve(s)
                X += x
                A += a
                Y += y
    return np.array(X, np.float32).reshape(-1, 64), np.array(A, np.int32), np.array(Y, np.float32)


def train(X, A, Y, epochs=200, batch=128, lr=1e-3, seed=1):
    return hpr.mlp_train(init_weights(seed), X, A, Y, epochs=epochs, batch=batch, lr=lr, seed=seed)


def evaluate(lps, w, tol=1e-8, max_iter=2_000_000, margin=0.0):
    """Per LP: iterations and seconds with Algorithm 3 and with the learned policy."""
    rows = []
    for lp in lps:
        with hpr.Solver(lp, max_iter=max_iter, persistent=0) as s:   # both runs on the same path
            base = s.solve(tol)["info"]
            s.set_policy(w)
            s.set_options(sigma_policy=2, policy_margin=float(margin))
            pol = s.solve(tol)["info"]
        rows.append(dict(name=lp.name, rule_iters=int(base["iters"]), rule_s=base["solve_time_s"],
                         rule_status=int(base["status"]), policy_iters=int(pol["iters"]),
                         policy_s=pol["solve_time_s"], policy_status=int(pol["status"]),
                         decisions=int(pol["policy_decisions"]), fallbacks=int(pol["policy_fallbacks"])))
    return rows


def training_family(count, seed0=0):
    """Small instances of the medium planted family (scale 0.005-0.01) and the
    multicommodity-flow family (100-300 nodes), alternating."""
    out = []
    for i in range(count):
        if i % 2 == 0:
            out.append(lpgen.planted_medium(seed0 + i, 0.005 + 0.005 * ((i // 2) % 2)))
        else:
            out.append(lpgen.mcf_lp(seed0 + i, nodes=100 + 100 * ((i // 2) % 3)))
    return out


def summary(rows):
    ok = [r for r in rows if r["rule_status"] == 0 and r["policy_status"] == 0]
    logs = np.array([math.log(r["policy_iters"] / r["rule_iters"]) for r in ok])
    gm = math.exp(float(logs.mean())) if len(logs) else float("nan")
    ci = [float("nan"), float("nan")]
    if len(logs) > 1:                         # 95% bootstrap interval of the geometric mean
        rng = np.random.default_rng(0x5EED)
        means = rng.choice(logs, size=(2000, len(logs)), replace=True).mean(axis=1)
        ci = [math.exp(float(np.quantile(means, 0.025))), math.exp(float(np.quantile(means, 0.975)))]
    dec = sum(r["decisions"] for r in rows)
    fb = sum(r["fallbacks"] for r in rows)
    return dict(n=len(rows), converged_both=len(ok), iters_ratio_geomean=gm, iters_ratio_ci95=ci,
                time_rule_s=sum(r["rule_s"] for r in rows), time_policy_s=sum(r["policy_s"] for r in rows),
                worse=sum(r["policy_iters"] > r["rule_iters"] for r in ok), decisions=dec, fallbacks=fb,
                fallback_rate=fb / max(dec + fb, 1))


def main_eval(argv):
    """eval weights.npy n_eval n_large margin [margin ...]: held-out evaluation only."""
    hpr.load()
    w = np.load(argv[2])
    n_eval, n_large = int(argv[3]), int(argv[4])
    small = training_family(n_eval, 10_000)
    large = [lpgen.planted_medium(20_000 + i, 0.05) for i in range(n_large)]
    for mg in argv[5:]:
        rs, rl = evaluate(small, w, margin=float(mg)), evaluate(large, w, margin=float(mg))
        print(json.dumps(dict(margin=float(mg), small=summary(rs), large=summary(rl) if rl else None)), flush=True)


def main(argv):
    if len(argv) > 1 and argv[1] == "eval":
        return main_eval(argv)
    n_train = int(argv[1]) if len(argv) > 1 else 40
    n_eval = int(argv[2]) if len(argv) > 2 else 10
    n_large = int(argv[4]) if len(argv) > 4 else 0
    large_scale = float(argv[5]) if len(argv) > 5 else 0.05
    hpr.load()
    t0 = time.time()
    X, A, Y = collect(training_family(n_train, 0), seeds=(11, 12))
    t1 = time.time()
    w, hist = train(X, A, Y)
    t2 = time.time()
    held = training_family(n_eval, 10_000)
    rows = evaluate(held, w)
    large = (evaluate([lpgen.planted_medium(20_000 + i, large_scale) for i in range(n_large)], w)
             if n_large else [])
    t3 = time.time()
    print(json.dumps(dict(samples=int(len(Y)), n_train=n_train, large_scale=large_scale,
                          collect_s=t1 - t0, train_s=t2 - t1, eval_s=t3 - t2,
                          loss_first=float(hist[0]), loss_last=float(hist[-1]),
                          small=summary(rows), large=summary(large) if large else None,
                          rows=rows, large_rows=large)))
    if len(argv) > 3:                       # where to keep the trained weights
        np.save(argv[3], w)


if __name__ == "__main__":
    main(sys.argv)
