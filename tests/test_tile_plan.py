"""The gather-tiled layout of the x phase (hpr_tile_plan, host only, no GPU): its invariants,
and a plain simulation of k_tile_part / k_tile_epi on it that must reproduce the CSR
product row by row.

The simulation follows the kernels' data flow, not their arithmetic order: each slice's
stored entries are multiplied with the block's entries of x and summed per sub-row, each
sub-row's sum goes to its slot, and each row adds its slots in block order.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2408_12179_b300 import hpr


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hpr.load()


def _matrix(seed, rows, cols, density, long_row=False, empty=False):
    rng = np.random.default_rng(seed)
    M = sp.random(rows, cols, density=density, random_state=rng, data_rvs=rng.standard_normal, format="lil")
    if long_row:
        M[rows // 3, :] = rng.standard_normal(cols)      # a row longer than a slice's steps
    if empty:
        M[1, :] = 0.0                                      # a row with no entry: no slot
    M = M.tocsr()
    M.eliminate_zeros()
    M.sort_indices()
    return M


def _simulate(M, L, x):
    """Row sums in row_order through the layout, checking on the way that every slot is
    written once and that a row's slots come in block order."""
    nsub = L["oslot"].size
    P = np.full(nsub, np.nan)
    writer = np.full(nsub, -1)
    written = np.zeros(nsub, int)
    val = np.where(L["src"] >= 0, M.data[np.maximum(L["src"], 0)], 0.0)
    nblk = L["bstart"].size - 1
    for b in range(nblk):
        g0, g1 = L["bstart"][b], L["bstart"][b + 1]
        for u in range(L["ustart"][b], L["ustart"][b + 1]):
            for s in range(L["wstart"][u], L["wstart"][u + 1]):
                r0, base, steps, w = (int(v) for v in L["smeta"][s])
                lg, nrows = w & 0xFF, w >> 8
                ent = base + np.arange(steps * 32)
                c = L["col"][ent].astype(np.int64)
                assert np.all(c < g1 - g0), "column offset outside its block"
                assert np.all(c[L["src"][ent] < 0] == 0), "padding must point at offset 0"
                prod = (val[ent] * x[g0 + c]).reshape(steps, 32)
                lane = prod.sum(axis=0)                     # per lane over the steps
                per_row = lane.reshape(32 >> lg, 1 << lg).sum(axis=1)
                for q in range(nrows):
                    slot = L["oslot"][r0 + q]
                    P[slot] = per_row[q]
                    writer[slot] = b
                    written[slot] += 1
    assert np.all(written == 1), "every slot is written exactly once"
    sp_ = L["slot_ptr"]
    sums = np.array([P[sp_[r]:sp_[r + 1]].sum() for r in range(M.shape[0])])
    for r in range(M.shape[0]):                             # a row's slots in block order
        assert np.all(np.diff(writer[sp_[r]:sp_[r + 1]]) > 0)
    return sums


CASES = [
    dict(seed=0, rows=700, cols=2000, density=0.01, tile_len=64),
    dict(seed=1, rows=1500, cols=900, density=0.004, tile_len=1000, long_row=True, empty=True),
    dict(seed=2, rows=300, cols=5000, density=0.02, tile_len=28928),
    dict(seed=3, rows=2000, cols=300, density=0.006, tile_len=2, grid=400),
    dict(seed=4, rows=64, cols=3001, density=0.05, tile_len=101, long_row=True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"seed{c['seed']}-tile{c['tile_len']}")
def test_tile_plan_reproduces_the_product(case):
    M = _matrix(case["seed"], case["rows"], case["cols"], case["density"], case.get("long_row", False),
                case.get("empty", False))
    grid = case.get("grid", 148)
    L = hpr.tile_plan(M, case["tile_len"], grid)
    bs = L["bstart"]
    nblk = bs.size - 1
    tl = case["tile_len"] & ~1
    # blocks: cover the columns, start even, at most tile_len long, balanced CTAs
    assert bs[0] == 0 and bs[-1] == M.shape[1] and np.all(np.diff(bs) > 0)
    assert np.all(bs[:-1] % 2 == 0) and np.all(np.diff(bs) <= tl)
    assert nblk >= -(-M.shape[1] // tl) and nblk <= grid
    assert L["cta_blk"].size == grid and np.all(np.diff(L["cta_blk"]) >= 0)
    assert np.array_equal(np.unique(L["cta_blk"]), np.arange(nblk))
    # units: runs of slices, each block's own, none empty
    assert np.all(np.diff(L["wstart"]) > 0) and L["wstart"][-1] == L["smeta"].shape[0]
    assert L["ustart"][0] == 0 and L["ustart"][-1] == L["wstart"].size - 1
    # every stored nonzero exactly once
    src = L["src"][L["src"] >= 0]
    assert np.array_equal(np.sort(src), np.arange(M.nnz))
    # slots: one per (row, block holding an entry of the row)
    order = L["row_order"]
    blocks_of_row = [np.unique(np.searchsorted(bs, M.indices[M.indptr[o]:M.indptr[o + 1]], side="right") - 1)
                     for o in order]
    assert np.array_equal(np.diff(L["slot_ptr"]), [b.size for b in blocks_of_row])
    assert L["slot_ptr"][-1] == L["oslot"].size
    x = np.random.default_rng(case["seed"] + 100).standard_normal(M.shape[1])
    got = _simulate(M, L, x)
    ref = (M @ x)[order]
    scale = np.abs(M)[order] @ np.abs(x)
    assert np.all(np.abs(got - ref) <= 1e-13 * np.maximum(scale, 1e-300)), np.max(np.abs(got - ref))


def test_tile_plan_rejects_what_it_cannot_lay_out():
    M = _matrix(5, 100, 5000, 0.01)
    with pytest.raises(hpr.HprError) as e:                # 2500 blocks of 2 columns > 148 CTAs
        hpr.tile_plan(M, 2, 148)
    assert e.value.code == hpr.HPR_ERR_ARG
    for bad in (dict(tile_len=1), dict(tile_len=70000), dict(grid=0)):
        args = dict(tile_len=64, grid=148)
        args.update(bad)
        with pytest.raises(hpr.HprError) as e:
            hpr.tile_plan(M, **args)
        assert e.value.code == hpr.HPR_ERR_ARG
