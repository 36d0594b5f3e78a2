"""The batched solve (many LPs in lock step, normal iterations fused into shared launches)
through the C ABI.  Each LP's arithmetic is the same as in its own solve -- the same
layout, the same per-row operation order, the same per-context checks and reductions --
so every batched result must equal the context's solo result bit for bit, and (through
the solo path's parity) the oracle's to the usual tolerances, which is also checked."""
import numpy as np
import pytest

from paper_2408_12179_b300 import hpr, lpgen

pytestmark = pytest.mark.gpu

import oracle
from oracle import kkt as K


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hpr.load()


def _family(with_slow=True):
    """Uneven LPs: tiny, medium at 1/100, a 300-node multicommodity flow, an
    inequality-only LP, and (with_slow) four of the batched family, which need several
    hundred thousand iterations to 1e-8 and stop at the iteration cap here."""
    lps = [lpgen.planted_tiny(0), lpgen.planted_tiny(1, m1=10, m2=200, n=300, density=0.03),
           lpgen.planted_medium(2, 0.01), lpgen.mcf_lp(0, nodes=300),
           lpgen.planted_tiny(3, m1=0, m2=90, n=170)]
    if with_slow:
        lps += lpgen.batch_family(7, 4, 500, 2000)
    return lps


CAP = 20_000


def _solo(lp, **opts):
    with hpr.Solver(lp, persistent=0, **opts) as s:     # the multi-CTA path, as in a batch
        return s.solve(1e-8)


@pytest.mark.parametrize("precisions", ["fp64", "mixed"])
def test_batch_equals_solo_solves(precisions):
    lps = _family()
    prec = [0] * len(lps) if precisions == "fp64" else [i % 2 for i in range(len(lps))]
    solvers = [hpr.Solver(lp, precision=p, max_iter=CAP, persistent=0) for lp, p in zip(lps, prec)]
    try:
        with hpr.Batch(solvers) as b:
            status, res = b.solve(1e-8)
            st = b.stats()
        assert status == hpr.HPR_MAX_ITER            # the slow ones stop at the cap
        assert st["periods"] > 0 and st["fused_launches"] > 0
        print(precisions, [(lp.name or i, p, int(r["status"]), int(r["info"]["iters"]))
                           for i, (lp, p, r) in enumerate(zip(lps, prec, res))])
        assert sum(r["status"] == hpr.HPR_OK for r in res) >= 4   # converged LPs are compared too
        for lp, p, r in zip(lps, prec, res):
            solo = _solo(lp, precision=p, max_iter=CAP)
            assert r["status"] == solo["status"], lp.name
            assert r["info"]["iters"] == solo["info"]["iters"], lp.name
            assert r["info"]["restarts"] == solo["info"]["restarts"], lp.name
            for key in ("x", "y", "z"):
                assert np.array_equal(r[key], solo[key]), (lp.name, key)
    finally:
        for s in solvers:
            s.close()


def test_batch_results_match_oracle():
    lps = _family(with_slow=False)
    solvers = [hpr.Solver(lp) for lp in lps]
    try:
        with hpr.Batch(solvers) as b:
            status, res = b.solve(1e-8)
        assert status == hpr.HPR_OK
        for lp, r in zip(lps, res):
            ref = oracle.solve(lp, tol=1e-8, max_iter=400_000)
            ind = K.kkt(lp, r["x"], r["y"], r["z"])
            assert ind["kkt"] <= 1e-8 * (1 + 1e-6), lp.name
            assert abs(r["info"]["primal_obj"] - ref["info"]["pobj"]) <= 1e-7 * abs(ref["info"]["pobj"]), lp.name
            assert K.in_C(r["x"], lp.l, lp.u) and K.in_D(r["y"], lp.m1)
    finally:
        for s in solvers:
            s.close()


def test_batch_misuse_is_rejected():
    a = hpr.Solver(lpgen.planted_tiny(0))
    c = hpr.Solver(lpgen.planted_tiny(1), check_every=100)
    try:
        with pytest.raises(hpr.HprError):
            hpr.Batch([a, a])
        with hpr.Batch([a, c]) as b:
            with pytest.raises(hpr.HprError) as e:
                a.solve(1e-8)                         # a context in a batch is not solved alone
            assert e.value.code == hpr.HPR_ERR_STATE
            with pytest.raises(hpr.HprError):
                b.solve(1e-8)                         # different check periods
        # after the batch is gone the contexts work on their own again
        assert a.solve(1e-8)["status"] == hpr.HPR_OK
    finally:
        a.close()
        c.close()


def test_large_batch_lays_out_small_contexts_for_throughput():
    """Each LP's phases are small (short-slice layouts by default), but the batch's fused
    phases move more than 40 MB: the batch gives its contexts the default layout, and its
    results equal solo solves made with that layout, bit for bit."""
    lps = [lpgen.planted_medium(seed, 0.1) for seed in range(6)]
    assert sum(12 * lp.nnz + 60 * lp.n + 8 * lp.m for lp in lps) >= 40e6
    assert sum(12 * lp.nnz + 8 * lp.n + 36 * lp.m for lp in lps) >= 40e6
    cap = 600
    solvers = [hpr.Solver(lp, max_iter=cap) for lp in lps]
    try:
        assert all(s.layout()["sell_steps"] == (16, 16) for s in solvers)
        with hpr.Batch(solvers) as b:
            assert all(s.layout()["sell_steps"] == (40, 40) for s in solvers)
            assert all(s.layout()["unit_cost"] == (64.0, 64.0) for s in solvers)
            status, res = b.solve(1e-8)
        for lp, r in zip(lps, res):
            solo = _solo(lp, max_iter=cap, sell_steps_a=40, sell_steps_t=40, unit_cost_a=64.0, unit_cost_t=64.0)
            assert r["info"]["iters"] == solo["info"]["iters"], lp.name
            for key in ("x", "y", "z"):
                assert np.array_equal(r[key], solo[key]), (lp.name, key)
    finally:
        for s in solvers:
            s.close()


def test_batch_of_cluster_solves():
    """A batch whose LPs all take the persistent cluster path on their own runs as cluster
    launches (one per cluster size, one cluster per LP, on streams of their own) with no
    check period on the host; every result equals the LP's own default solve bit for bit.
    One LP that does not fit a cluster sends the whole batch to the fused path."""
    lps = [lpgen.planted_medium(0, 0.001), lpgen.planted_medium(1, 0.002), lpgen.planted_medium(2, 0.005),
           lpgen.qap_lp(2, 6), lpgen.planted_medium(4, 0.003)]
    solvers = [hpr.Solver(lp, max_iter=CAP) for lp in lps]
    try:
        with hpr.Batch(solvers) as b:
            status, res = b.solve(1e-8)
            st = b.stats()
        assert [int(r["info"]["path"]) for r in res] == [4] * len(lps)
        sizes = {int(r["info"]["path_ctas"]) for r in res}
        assert st["periods"] == 0 and st["fused_launches"] == len(sizes)
        for lp, r in zip(lps, res):
            with hpr.Solver(lp, max_iter=CAP) as s:
                solo = s.solve(1e-8)
            assert (solo["info"]["path"], solo["info"]["path_ctas"]) == (r["info"]["path"], r["info"]["path_ctas"])
            assert r["status"] == solo["status"] and r["info"]["iters"] == solo["info"]["iters"], lp.name
            for key in ("x", "y", "z"):
                assert np.array_equal(r[key], solo[key]), (lp.name, key)
        print("cluster sizes", sorted(sizes), "statuses", [int(r["status"]) for r in res])
    finally:
        for s in solvers:
            s.close()
    mixed = [hpr.Solver(lp, max_iter=300) for lp in (lps[0], lpgen.planted_medium(3, 0.05))]
    try:
        with hpr.Batch(mixed) as b:
            status, res = b.solve(1e-8)
            assert b.stats()["periods"] > 0
        assert [int(r["info"]["path"]) for r in res] == [0, 0]
    finally:
        for s in mixed:
            s.close()


def test_batch_of_single_cta_solves():
    """A batch whose LPs all take the persistent single-CTA path runs as one launch, one CTA
    per LP; each result equals that LP's own single-CTA solve bit for bit."""
    lps = [lpgen.planted_tiny(seed) for seed in range(12)] + [lpgen.planted_tiny(3, m1=0, m2=90, n=170)]
    solvers = [hpr.Solver(lp) for lp in lps]
    try:
        with hpr.Batch(solvers) as b:
            status, res = b.solve(1e-8)
            st = b.stats()
        assert status == hpr.HPR_OK and st["fused_launches"] == 1 and st["periods"] == 0
        for lp, r in zip(lps, res):
            with hpr.Solver(lp, persistent=2) as s:
                solo = s.solve(1e-8)
            assert r["info"]["iters"] == solo["info"]["iters"], lp.name
            assert r["info"]["lambda"] == solo["info"]["lambda"], lp.name
            for key in ("x", "y", "z"):
                assert np.array_equal(r[key], solo[key]), (lp.name, key)
    finally:
        for s in solvers:
            s.close()
