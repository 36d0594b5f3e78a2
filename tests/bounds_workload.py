"""Solves on every CUDA path with the solver library given on the command line (the normal
build or the bounds-checking build), printing one JSON line: a SHA-1 of each solve's
results and the library's count of out-of-range gather indices.  Run in a subprocess by
tests/test_gpu_bounds.py (a process loads one library).

With --plant, the bounds-checking build also runs the allocation-free power method on a
caller CSR whose first column index is one past the end: the kernel's check counts it and
reads index 0 instead (run on the bounds-checking build only)."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import scipy.sparse as sp  # noqa: E402


def digest(res):
    h = hashlib.sha1()
    for key in ("x", "y", "z"):
        h.update(np.ascontiguousarray(res[key]).tobytes())
    return h.hexdigest()[:16] + f":{int(res['info']['iters'])}:{int(res['info']['path'])}"


def noalloc(hpr, lp, plant):
    import torch

    A = sp.vstack([lp.A1, lp.A2]).tocsr()
    T = A.T.tocsr()
    dev = torch.device("cuda")

    def arrays(M):
        ci = M.indices.astype(np.int32).copy()
        if plant:
            ci[0] = M.shape[1]                       # one past the end of the gathered vector
        return (torch.tensor(M.indptr.astype(np.int32), device=dev), torch.tensor(ci, device=dev),
                torch.tensor(M.data, dtype=torch.float64, device=dev))

    a, t = arrays(A), arrays(T)
    u = torch.zeros(A.shape[0], dtype=torch.float64, device=dev)
    s = torch.zeros(A.shape[1], dtype=torch.float64, device=dev)
    lam, it = hpr.hpr_power_noalloc(A.shape[0], A.shape[1], tuple(x.data_ptr() for x in a),
                                    tuple(x.data_ptr() for x in t), 7, 2000, 1e-10, u.data_ptr(), s.data_ptr())
    torch.cuda.synchronize()
    return f"{lam!r}:{it}"


def main(argv):
    from paper_2408_12179_b300 import hpr, lpgen

    hpr.load(argv[1])
    plant = "--plant" in argv
    out = {}
    lps = {"tiny0": lpgen.planted_tiny(0), "ineq": lpgen.planted_tiny(3, m1=0, m2=90, n=170),
           "eq": lpgen.planted_tiny(4, m1=70, m2=0, n=190), "m200": lpgen.planted_medium(0, 0.005),
           "qap6": lpgen.qap_lp(2, 6)}
    for name, lp in lps.items():
        for p in (0, 2, 3, 4):
            try:
                out[f"{name}/p{p}"] = digest(hpr.solve(lp, tol=1e-8, max_iter=30_000, persistent=p))
            except hpr.HprError as e:                # the LP does not fit that path
                out[f"{name}/p{p}"] = f"refused {e.code}"
    out["tiny0/fp32"] = digest(hpr.solve(lps["tiny0"], tol=1e-8, max_iter=30_000, precision=1))
    for label, group, opts in (("small", [lpgen.planted_tiny(s) for s in (1, 2)], {}),
                               ("cluster", [lpgen.planted_medium(0, 0.001), lpgen.planted_medium(1, 0.002)], {}),
                               ("fused", [lpgen.planted_tiny(5), lpgen.mcf_lp(0, nodes=300)], {"persistent": 0})):
        solvers = [hpr.Solver(q, max_iter=30_000, **opts) for q in group]
        try:
            with hpr.Batch(solvers) as b:
                _, res = b.solve(1e-8)
            for i, r in enumerate(res):
                out[f"batch/{label}/{i}"] = digest(r)
        finally:
            for s_ in solvers:
                s_.close()
    out["noalloc"] = noalloc(hpr, lps["m200"], False)
    violations = hpr.bounds_violations()
    planted = None
    if plant:
        noalloc(hpr, lps["tiny0"], True)
        planted = hpr.bounds_violations() - violations
        out["after_plant"] = digest(hpr.solve(lps["tiny0"], tol=1e-8, max_iter=30_000, persistent=0))
    print(json.dumps({"results": out, "violations": violations, "planted": planted}), flush=True)


if __name__ == "__main__":
    main(sys.argv)
