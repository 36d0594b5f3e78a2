"""Seeded synthetic LP generators shared by the CUDA path's tests/bench and the oracle.

This module builds problem DATA only: it holds none of the solver's arithmetic
(no scaling, no projections, no iteration).  Every instance is the LP of Section 1,
eq. (1):

    min <c, x>   s.t.  A1 x = b1,  A2 x >= b2,  l <= x <= u,

returned as an :class:`LP` whose constraint blocks are SciPy CSR matrices with sorted,
duplicate-free column indices.

Planted optimum.  For the "planted" families an optimal primal-dual triple
(x*, y*, z*) is fixed first and the data are derived from it so that it satisfies the
KKT system of Section 2 (eq. KKT): A1 x* = b1, A2 x* - b2 = s >= 0 with y2* >= 0 and
y2*_i s_i = 0, z* in -N_C(x*) (z*_j > 0 only at an active lower bound, < 0 only at an
active upper bound) and c = A^T y* + z*.  The optimal value is then <c, x*>.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class LP:
    A1: sp.csr_matrix
    A2: sp.csr_matrix
    b1: np.ndarray
    b2: np.ndarray
    c: np.ndarray
    l: np.ndarray
    u: np.ndarray
    x_star: np.ndarray | None = None
    y_star: np.ndarray | None = None
    z_star: np.ndarray | None = None
    name: str = ""

    @property
    def m1(self) -> int:
        return self.A1.shape[0]

    @property
    def m2(self) -> int:
        return self.A2.shape[0]

    @property
    def m(self) -> int:
        return self.m1 + self.m2

    @property
    def n(self) -> int:
        return self.A1.shape[1]

    @property
    def nnz(self) -> int:
        return self.A1.nnz + self.A2.nnz

    @property
    def A(self) -> sp.csr_matrix:
        """A = [A1; A2] in CSR (rows 0..m1-1 are the equalities)."""
        return sp.vstack([self.A1, self.A2], format="csr")

    @property
    def b(self) -> np.ndarray:
        return np.concatenate([self.b1, self.b2])

    @property
    def planted_objective(self) -> float | None:
        if self.x_star is None:
            return None
        return float(np.dot(self.c, self.x_star))


def _canonical(M: sp.spmatrix) -> sp.csr_matrix:
    M = sp.csr_matrix(M, dtype=np.float64)
    M.sum_duplicates()
    M.sort_indices()
    M.eliminate_zeros()
    M.indices = M.indices.astype(np.int32, copy=False)
    M.indptr = M.indptr.astype(np.int64, copy=False)
    return M


def _plant_boxed_primal(rng, n_cols, lo, hi):
    """x* and z* for boxed columns [lo, hi]: 30% at a bound (half lower, half upper),
    the rest strictly inside; z* complementary to the active bound."""
    x = rng.uniform(lo + 0.05 * (hi - lo), hi - 0.05 * (hi - lo), n_cols)
    z = np.zeros(n_cols)
    at_bound = rng.random(n_cols) < 0.3
    at_upper = at_bound & (rng.random(n_cols) < 0.5)
    at_lower = at_bound & ~at_upper
    x[at_lower] = lo
    x[at_upper] = hi
    z[at_lower] = rng.uniform(0.1, 1.0, at_lower.sum())
    z[at_upper] = -rng.uniform(0.1, 1.0, at_upper.sum())
    return x, z


def _plant_rows(rng, A1, A2, x, z):
    """y*, slack s and the right-hand sides / cost for a planted optimum."""
    m1, m2 = A1.shape[0], A2.shape[0]
    y1 = rng.standard_normal(m1)
    tight = rng.random(m2) < 0.5
    y2 = np.where(tight, rng.uniform(0.1, 1.0, m2), 0.0)
    s = np.where(tight, 0.0, rng.uniform(0.1, 1.0, m2))
    b1 = A1 @ x
    b2 = A2 @ x - s
    c = A1.T @ y1 + A2.T @ y2 + z
    return np.concatenate([y1, y2]), b1, b2, c


def planted_tiny(seed: int, m1: int = 40, m2: int = 60, n: int = 200, density: float = 0.05) -> LP:
    """Tiny planted LP: each entry nonzero with probability `density`, values N(0,1);
    l = 0, u = 10 on the first half of the columns and +inf on the rest; 30% of x* at a
    bound (boxed columns: half at l, half at u; unbounded columns: at l)."""
    rng = np.random.default_rng([0x71A7, seed])
    m = m1 + m2
    mask = rng.random((m, n)) < density
    vals = rng.standard_normal((m, n))
    dense = np.where(mask, vals, 0.0)
    A1 = _canonical(sp.csr_matrix(dense[:m1]))
    A2 = _canonical(sp.csr_matrix(dense[m1:]))
    l = np.zeros(n)
    u = np.full(n, np.inf)
    nb = n // 2
    u[:nb] = 10.0
    x, z = _plant_boxed_primal(rng, n, 0.0, 10.0)
    # unbounded columns: active bound can only be the lower one
    free_up = np.arange(n) >= nb
    moved = free_up & (x == 10.0)
    x[moved] = 0.0
    z[moved] = -z[moved]
    y, b1, b2, c = _plant_rows(rng, A1, A2, x, z)
    return LP(A1, A2, b1, b2, c, l, u, x, y, z, name=f"tiny-{seed}")


def _zipf_counts(rng, n, s, cap, target_nnz, m):
    counts = np.minimum(rng.zipf(s, n), cap).astype(np.float64)
    counts *= target_nnz / counts.sum()
    base = np.floor(counts)
    counts = base + (rng.random(n) < (counts - base))
    counts = np.maximum(counts, 1).astype(np.int64)
    return np.minimum(counts, m)


def _rows_without_replacement(rng, counts, m):
    """For column j draw counts[j] distinct row indices uniformly from [0, m)."""
    cols = np.repeat(np.arange(counts.size, dtype=np.int64), counts)
    rows = rng.integers(0, m, cols.size)
    while True:
        key = cols * m + rows
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(ks.size, dtype=bool)
        dup[1:] = ks[1:] == ks[:-1]
        if not dup.any():
            return rows, cols
        idx = order[dup]
        rows[idx] = rng.integers(0, m, idx.size)


def planted_sparse(seed: int, m: int = 200_000, n: int = 500_000, nnz: float = 5e6,
                   zipf_s: float = 1.5, cap: int = 2000, free_frac: float = 0.2) -> LP:
    """Medium sparse planted LP (50% equalities): power-law column counts (Zipf(s)
    capped at `cap`, then scaled to about `nnz` in total with stochastic rounding and
    a floor of 1), rows of a column uniform without replacement, values
    +-10^U(-3,3); `free_frac` of the columns free (z* = 0, x* ~ N(0,1)), the rest boxed
    [0, 10] with the tiny family's x*/z* rule."""
    rng = np.random.default_rng([0x5A25E, seed])
    m1 = m // 2
    counts = _zipf_counts(rng, n, zipf_s, cap, nnz, m)
    rows, cols = _rows_without_replacement(rng, counts, m)
    vals = rng.choice([-1.0, 1.0], rows.size) * 10.0 ** rng.uniform(-3.0, 3.0, rows.size)
    A = _canonical(sp.csr_matrix((vals, (rows, cols)), shape=(m, n)))
    A1 = _canonical(A[:m1])
    A2 = _canonical(A[m1:])
    free = rng.random(n) < free_frac
    l = np.where(free, -np.inf, 0.0)
    u = np.where(free, np.inf, 10.0)
    x, z = _plant_boxed_primal(rng, n, 0.0, 10.0)
    x[free] = rng.standard_normal(free.sum())
    z[free] = 0.0
    y, b1, b2, c = _plant_rows(rng, A1, A2, x, z)
    return LP(A1, A2, b1, b2, c, l, u, x, y, z, name=f"sparse-{seed}-m{m}-n{n}")


def planted_medium(seed: int, scale: float = 1.0) -> LP:
    """The medium sparse planted LP (m = 200k, n = 500k, nnz ~ 5M) scaled by `scale`
    in rows, columns and nonzeros."""
    m = max(4, int(round(200_000 * scale)))
    n = max(4, int(round(500_000 * scale)))
    nnz = 5e6 * scale
    cap = max(2, min(2000, m))
    return planted_sparse(seed, m=m + (m % 2), n=n, nnz=nnz, cap=cap)


def batch_family(seed: int, count: int, m_lo: int = 500, m_hi: int = 50_000) -> list[LP]:
    """Uneven LPs for a batched solve: m log-uniform in [m_lo, m_hi] (rounded to even),
    n = 2.5 m, density log-uniform in [0.1%, 1%], each built like the medium planted LP
    (Zipf(1.5) column counts capped at min(2000, m), values +-10^U(-3,3), 20% free
    columns, planted optimum) with nnz = density * m * n."""
    rng = np.random.default_rng([0xBA7C, seed])
    out = []
    for i in range(count):
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        m += m % 2
        n = int(round(2.5 * m))
        density = math.exp(rng.uniform(math.log(1e-3), math.log(1e-2)))
        lp = planted_sparse(seed * 1_000_003 + i, m=m, n=n, nnz=density * m * n, cap=max(2, min(2000, m)))
        lp.name = f"batch-{seed}-{i}-m{m}"
        out.append(lp)
    return out


def micro_lp(seed: int, n: int = 5, m1: int = 1, m2: int = 3) -> LP:
    """Micro LP with finite bounds and a dense A, feasible by construction (the
    right-hand sides are taken at a random point of the box).  No optimum is planted:
    these are solved by vertex enumeration in the tests."""
    rng = np.random.default_rng([0x31C0, seed])
    m = m1 + m2
    A = np.round(rng.uniform(-3, 3, (m, n)), 1)
    A[A == 0] = 0.5
    l = np.round(rng.uniform(-2, 0, n), 1)
    u = np.round(l + rng.uniform(1, 4, n), 1)
    x0 = rng.uniform(l, u)
    r = A @ x0
    b1 = r[:m1]
    b2 = r[m1:] - rng.uniform(0, 1, m2)
    c = np.round(rng.uniform(-2, 2, n), 1)
    return LP(_canonical(A[:m1]), _canonical(A[m1:]), b1, b2, c, l, u, name=f"micro-{seed}")


def simplex_lp(costs) -> LP:
    """min <c,x> s.t. sum(x) = 1, x >= 0: the optimum is min_i c_i (closed form)."""
    c = np.asarray(costs, dtype=np.float64)
    n = c.size
    A1 = _canonical(np.ones((1, n)))
    A2 = _canonical(sp.csr_matrix((0, n)))
    return LP(A1, A2, np.ones(1), np.zeros(0), c, np.zeros(n), np.full(n, np.inf), name="simplex")


def knapsack_lp(a, cost, beta, ub) -> LP:
    """Continuous covering knapsack: min <c,x> s.t. <a,x> >= beta, 0 <= x <= ub with
    a, c > 0.  The optimum is the greedy fill by increasing c_j / a_j (closed form)."""
    a = np.asarray(a, dtype=np.float64)
    n = a.size
    A1 = _canonical(sp.csr_matrix((0, n)))
    A2 = _canonical(a[None, :])
    return LP(A1, A2, np.zeros(0), np.array([float(beta)]), np.asarray(cost, dtype=np.float64),
              np.zeros(n), np.asarray(ub, dtype=np.float64), name="knapsack")


def knapsack_optimum(a, cost, beta, ub) -> float:
    """Greedy value of :func:`knapsack_lp` (fill cheapest c/a first)."""
    a = np.asarray(a, float)
    cost = np.asarray(cost, float)
    ub = np.asarray(ub, float)
    need = float(beta)
    val = 0.0
    for j in np.argsort(cost / a, kind="stable"):
        if need <= 0:
            break
        take = min(ub[j], need / a[j])
        val += cost[j] * take
        need -= a[j] * take
    return val


def mcf_lp(seed: int, nodes: int = 1_000_000, k_out: int = 8, commodities: int = 4) -> LP:
    """Min-cost multicommodity flow on a random geometric k-nearest-neighbour digraph.

    Nodes are uniform in the unit square and numbered along a Morton (Z-order) curve;
    each node has arcs to its `k_out` nearest neighbours.  Variables f_{a,k} >= 0 (one
    per arc and commodity, commodity-major); equality rows are node x commodity flow
    conservation (entries +-1), inequality rows are the shared capacities
    -sum_k f_{a,k} >= -cap_a.  Costs U[1,100], capacities U[1,50].  Supplies are
    balanced and feasible by construction: a random flow f0 puts U(0, 1/4) * cap_a of
    every commodity on every arc (so the shared capacities hold) and b1 = A1 f0."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng([0x3CF, seed])
    pts = rng.random((nodes, 2))
    q = np.minimum((pts * 65536).astype(np.uint64), 65535)

    def spread(v):
        v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF)
        v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F)
        v = (v | (v << np.uint64(2))) & np.uint64(0x33333333)
        v = (v | (v << np.uint64(1))) & np.uint64(0x55555555)
        return v

    morton = spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1))
    pts = pts[np.argsort(morton, kind="stable")]
    tree = cKDTree(pts)
    _, nbr = tree.query(pts, k=k_out + 1)
    tail = np.repeat(np.arange(nodes, dtype=np.int64), k_out)
    head = nbr[:, 1:].reshape(-1).astype(np.int64)
    narcs = tail.size
    cap = rng.uniform(1.0, 50.0, narcs)
    cost = rng.uniform(1.0, 100.0, narcs)
    # random feasible flow: the node imbalances of f0 define the supplies
    f0 = rng.uniform(0.0, 0.25, (commodities, narcs)) * cap[None, :]
    n = narcs * commodities
    kk = np.repeat(np.arange(commodities, dtype=np.int64), narcs)
    arc = np.tile(np.arange(narcs, dtype=np.int64), commodities)
    var = np.arange(n, dtype=np.int64)
    # node-arc incidence per commodity: +1 at the tail (outflow), -1 at the head
    rows_eq = np.concatenate([kk * nodes + np.tile(tail, commodities), kk * nodes + np.tile(head, commodities)])
    cols_eq = np.concatenate([var, var])
    vals_eq = np.concatenate([np.ones(n), -np.ones(n)])
    A1 = _canonical(sp.csr_matrix((vals_eq, (rows_eq, cols_eq)), shape=(nodes * commodities, n)))
    A2 = _canonical(sp.csr_matrix((-np.ones(n), (arc, var)), shape=(narcs, n)))
    x0 = f0.reshape(-1)
    b1 = A1 @ x0
    b2 = -cap
    c = np.tile(cost, commodities)
    return LP(A1, A2, b1, b2, c, np.zeros(n), np.full(n, np.inf), name=f"mcf-{seed}-{nodes}")


def qap_matrices(seed: int, N: int):
    """Random QAP data: flows a (symmetric, integers 0..9, zero diagonal) and distances b
    (Manhattan distances between N distinct points of an N x N grid)."""
    rng = np.random.default_rng([0x0A9, seed])
    f = rng.integers(0, 10, (N, N)).astype(np.float64)
    a = np.triu(f, 1)
    a = a + a.T
    cells = rng.choice(N * N, N, replace=False)
    px, py = cells // N, cells % N
    b = (np.abs(px[:, None] - px[None, :]) + np.abs(py[:, None] - py[None, :])).astype(np.float64)
    return a, b


def qap_lp(seed: int, N: int) -> LP:
    """Adams-Johnson linearisation of the QAP min sum a_ik b_jl x_ij x_kl, in the form the
    paper prints for its QAP experiment: variables x_kl (N^2, in [0, 1]) then s_ijkl
    (N^4, >= 0, index ((i N + j) N + k) N + l); equality rows sum_i s_ijkl = x_kl (j, k, l),
    sum_j s_ijkl = x_kl (i, k, l), s_ijkl = s_klij for each unordered pair
    (i, j) != (k, l), sum_j x_ij = 1 (i) and sum_i x_ij = 1 (j); cost a_ik b_jl on s_ijkl.
    The flow and distance matrices are random (qap_matrices), not QAPLIB's."""
    a, b = qap_matrices(seed, N)
    N2, N4 = N * N, N ** 4
    i, j, k, l = (v.ravel() for v in np.meshgrid(*(np.arange(N),) * 4, indexing="ij"))
    sv = N2 + ((i * N + j) * N + k) * N + l
    xkl = k * N + l
    rows, cols, vals = [], [], []
    # sum_i s_ijkl - x_kl = 0, one row per (j, k, l)
    r1 = (j * N + k) * N + l
    rows += [r1, np.arange(N ** 3)]
    cols += [sv, (np.arange(N ** 3) % N2)]
    vals += [np.ones(N4), -np.ones(N ** 3)]
    # sum_j s_ijkl - x_kl = 0, one row per (i, k, l)
    r2 = N ** 3 + (i * N + k) * N + l
    rows += [r2, N ** 3 + np.arange(N ** 3)]
    cols += [sv, (np.arange(N ** 3) % N2)]
    vals += [np.ones(N4), -np.ones(N ** 3)]
    # s_ijkl - s_klij = 0 for (i, j) < (k, l)
    p_ij, p_kl = i * N + j, k * N + l
    keep = p_ij < p_kl
    nsym = int(keep.sum())
    r3 = 2 * N ** 3 + np.arange(nsym)
    rows += [r3, r3]
    cols += [sv[keep], N2 + ((k[keep] * N + l[keep]) * N + i[keep]) * N + j[keep]]
    vals += [np.ones(nsym), -np.ones(nsym)]
    # assignment rows
    base = 2 * N ** 3 + nsym
    ii, jj = np.divmod(np.arange(N2), N)
    rows += [base + ii, base + N + jj]
    cols += [np.arange(N2), np.arange(N2)]
    vals += [np.ones(N2), np.ones(N2)]
    m = base + 2 * N
    n = N2 + N4
    A1 = _canonical(sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(m, n)))
    A2 = _canonical(sp.csr_matrix((0, n)))
    b1 = np.concatenate([np.zeros(2 * N ** 3 + nsym), np.ones(2 * N)])
    c = np.concatenate([np.zeros(N2), a[i, k] * b[j, l]])
    lo = np.zeros(n)
    up = np.concatenate([np.ones(N2), np.full(N4, np.inf)])
    return LP(A1, A2, b1, np.zeros(0), c, lo, up, name=f"qap-{seed}-N{N}")


def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """Reference values of the counter-based generator used by both solvers for the
    power-method start vector (SplitMix64, Steele, Lea & Flood, OOPSLA 2014): the i-th
    output mixes seed + (i+1) * 0x9E3779B97F4A7C15; U = (out >> 11) * 2^-53.
    Provided for tests only; each solver implements the generator itself."""
    mask = (1 << 64) - 1
    out = np.empty(count)
    for i in range(count):
        z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z ^= z >> 31
        out[i] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out
