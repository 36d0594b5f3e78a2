"""The sliced-ELL layout of the hot path's SpMV phases, inspected on the host through
hpr_layout_plan (no GPU): every nonzero is stored exactly once at the position the layout
defines, padding is zero, rows are ordered by decreasing length (stably), each 32-row group
takes the fewest lanes per row that keep its longest row within the step bound, and the
work units split exactly the groups whose cost exceeds the unit size."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2408_12179_b300 import hpr


def _matrix(seed, rows=300, cols=2000):
    """Rows of very uneven lengths: empty rows, short ones, ones around the step bounds
    (16, 40 steps of one lane) and a few beyond 32 lanes x 40 steps."""
    rng = np.random.default_rng(seed)
    lens = rng.choice([0, 1, 2, 3, 5, 9, 16, 17, 40, 41, 64, 100, 700, 1300, 1500],
                      size=rows, p=[.06, .2, .12, .1, .1, .1, .06, .06, .05, .05, .04, .03, .01, .01, .01])
    indptr = np.zeros(rows + 1, np.int64)
    indptr[1:] = np.cumsum(lens)
    indices = np.concatenate([np.sort(rng.choice(cols, size=k, replace=False)) for k in lens]).astype(np.int32)
    data = rng.standard_normal(indptr[-1])
    return sp.csr_matrix((data, indices, indptr), shape=(rows, cols))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hpr.load()


PARAMS = [(40, 64.0), (16, 32.0), (8, 16.0), (128, 256.0), (1, 4.0)]


@pytest.mark.parametrize("steps,cost", PARAMS)
@pytest.mark.parametrize("seed", [0, 1])
def test_every_entry_stored_once_where_the_layout_says(seed, steps, cost):
    M = _matrix(seed)
    P = hpr.layout_plan(M, steps, cost)
    order, srow, sptr, slg, col, src = (P[k] for k in ("row_order", "srow", "sptr", "slg", "col", "src"))
    seen = np.zeros(M.nnz, np.int64)
    for s in range(len(slg)):
        L = 1 << int(slg[s])
        r0, r1 = int(srow[s]), int(srow[s + 1])
        width = int(sptr[s + 1] - sptr[s])
        assert width % 32 == 0
        for k in range(width // 32):
            for lane in range(32):
                at = int(sptr[s]) + 32 * k + lane
                q, e = lane // L, k * L + lane % L
                if src[at] < 0:                      # padding: past the row's end or past the slice's rows
                    assert col[at] == 0
                    assert q >= r1 - r0 or e >= M.indptr[order[r0 + q] + 1] - M.indptr[order[r0 + q]]
                    continue
                row = int(order[r0 + q])
                assert src[at] == M.indptr[row] + e             # the e-th entry of its row
                assert col[at] == M.indices[src[at]]
                seen[src[at]] += 1
    assert np.all(seen == 1)


@pytest.mark.parametrize("seed", [0, 1])
def test_rows_by_decreasing_length_stably(seed):
    M = _matrix(seed)
    order = hpr.layout_plan(M)["row_order"]
    lens = np.diff(M.indptr)
    assert sorted(order) == list(range(M.shape[0]))
    expect = sorted(range(M.shape[0]), key=lambda i: (-lens[i], i))
    assert list(order) == expect


@pytest.mark.parametrize("steps,cost", PARAMS)
def test_lanes_and_work_units(steps, cost):
    M = _matrix(2)
    P = hpr.layout_plan(M, steps, cost)
    order, srow, sptr, slg, wstart = (P[k] for k in ("row_order", "srow", "sptr", "slg", "wstart"))
    lens = np.diff(M.indptr)[order]
    rows = M.shape[0]
    # slices of each 32-row group, and the group's lanes per row
    groups, s = [], 0
    for g0 in range(0, rows, 32):
        g1 = min(rows, g0 + 32)
        lg = 0
        while lg < 5 and -(-int(lens[g0]) // (1 << lg)) > steps:
            lg += 1
        L, per = 1 << lg, 32 >> lg
        first = s
        for r in range(g0, g1, per):
            assert srow[s] == r and srow[s + 1] == min(g1, r + per) and slg[s] == lg
            assert (sptr[s + 1] - sptr[s]) // 32 == -(-int(lens[r]) // L)      # steps of the slice
            s += 1
        groups.append((first, s))
    assert s == len(slg)
    # work units: a group whole when its cost fits, else one unit per slice
    cost_of = lambda sl: (sptr[sl + 1] - sptr[sl]) // 32 + 2 + int(slg[sl]) + 8.0 * (srow[sl + 1] - srow[sl]) / 32
    want = []
    for a, b in groups:
        if sum(cost_of(sl) for sl in range(a, b)) <= cost:
            want.append(a)
        else:
            want.extend(range(a, b))
    assert list(wstart) == want + [len(slg)]


def test_bad_input_rejected():
    M = _matrix(0, rows=40)
    for steps, cost in [(0, 64.0), (5000, 64.0), (40, 0.0), (40, -1.0)]:
        with pytest.raises(hpr.HprError):
            hpr.layout_plan(M, steps, cost)
    bad = M.copy()
    bad.indices[3] = M.shape[1] + 5
    with pytest.raises(hpr.HprError):
        hpr.layout_plan(bad)
