"""The FP32 form against plain FP64 on the same instances: time and iterations to KKT <= tol.

``python -m paper_2408_12179_b300.forms N_SEEDS SCALE [TOL]`` solves seeded medium
planted LPs (seeds 0 .. N_SEEDS-1 at the given scale) on one GPU, each with
precision 0 and with precision 1 in the same context (power method included in both),
and prints one JSON line per instance and a summary line (geometric mean of the time
ratios, wins).
"""
from __future__ import annotations

import json
import math
import sys

from . import hpr, lpgen


def compare(lp, tol=1e-8, max_iter=3_000_000):
    row = {"name": lp.name}
    with hpr.Solver(lp, max_iter=max_iter, persistent=0) as s:
        for prec in (0, 1):
            s.set_options(precision=prec)
            I = s.solve(tol)["info"]
            row[f"p{prec}"] = dict(iters=int(I["iters"]), seconds=I["solve_time_s"], status=int(I["status"]),
                                   iters_fp32=int(I["iters_fp32"]), kkt=I["kkt"])
    return row


def main(argv):
    n = int(argv[1]) if len(argv) > 1 else 6
    scale = float(argv[2]) if len(argv) > 2 else 0.1
    tol = float(argv[3]) if len(argv) > 3 else 1e-8
    hpr.load()
    rows = []
    for seed in range(n):
        r = compare(lpgen.planted_medium(seed, scale), tol)
        rows.append(r)
        print(json.dumps(r), flush=True)
    ok = [r for r in rows if r["p0"]["status"] == 0 and r["p1"]["status"] == 0]
    ratios = [r["p1"]["seconds"] / r["p0"]["seconds"] for r in ok]
    gm = math.exp(sum(math.log(x) for x in ratios) / max(len(ratios), 1))
    print(json.dumps(dict(instances=len(rows), both_converged=len(ok), time_ratio_geomean=gm,
                          fp32_form_faster=sum(x < 1 for x in ratios),
                          total_fp64_s=sum(r["p0"]["seconds"] for r in ok),
                          total_fp32_form_s=sum(r["p1"]["seconds"] for r in ok))), flush=True)


if __name__ == "__main__":
    main(sys.argv)
