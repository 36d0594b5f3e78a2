"""Writes tests/golden/medium_lp_seed0.json: the oracle's solve of the medium sparse planted
LP (m = 200,000, n = 500,000, about 5.2M nonzeros, seed 0) to KKT <= 1e-8.

The stored primal / dual objectives and iteration count come from ``oracle.solve`` alone
(the plain FP64 CPU HPR-LP of Algorithm 2 with the preprocessing, power method and
termination test of Section 4.1) on the LP that ``lpgen.planted_medium(0, 1.0)`` generates;
nothing here touches the CUDA solver.  The planted optimal value <c, x*> of the same LP is
stored beside it, as a second, closed-form reference.

Run from the repository root (about an hour and a half on 8 host cores):

    python tests/golden/make_medium_solution.py
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import kkt as okkt  # noqa: E402
from paper_2408_12179_b300 import lpgen  # noqa: E402


def main() -> None:
    seed, scale, tol = 0, 1.0, 1e-8
    lp = lpgen.planted_medium(seed, scale)
    t0 = time.time()
    res = oracle.solve(lp, tol=tol, max_iter=3_000_000, checks_cap=100_000)
    secs = time.time() - t0
    info = res["info"]
    ind = okkt.kkt(lp, res["x"], res["y"], res["z"])
    out = {
        "_citation": "Algorithm 2 run to the termination test of Section 4.1 (relative KKT <= 1e-8, "
                     "checked every 150 iterations) by the FP64 CPU oracle; written by "
                     "tests/golden/make_medium_solution.py",
        "workload": "lpgen.planted_medium(seed=0, scale=1.0)",
        "m": lp.m, "n": lp.n, "nnz": lp.nnz,
        "tol": tol,
        "status": info["status"],
        "iters": info["iters"],
        "restarts": int(info["restarts"]),
        "lambda": info["lambda"],
        "power_iters": int(info["power_iters"]),
        "pobj": info["pobj"],
        "dobj": info["dobj"],
        "kkt": info["kkt"],
        "independent_kkt": ind["kkt"],
        "planted_objective": lp.planted_objective,
        "oracle_seconds": secs,
        "threads": os.environ.get("OMP_NUM_THREADS", str(os.cpu_count())),
    }
    path = os.path.join(HERE, "medium_lp_seed0.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
