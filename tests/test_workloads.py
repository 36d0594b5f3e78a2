"""The seeded workloads are reproducible and have the sizes the measurements quote: the
benchmark LP (medium planted, seed 0), the QAP linearisation at N = 20 and 30, the
multicommodity-flow LP at 1/100 scale, and the tiny planted family's planted optimum."""
import numpy as np
import pytest

from paper_2408_12179_b300 import lpgen


def test_benchmark_lp_sizes_and_reproducibility():
    a = lpgen.planted_medium(0, 1.0)
    assert (a.m, a.m1, a.n, a.nnz) == (200_000, 100_000, 500_000, 5_248_615)
    b = lpgen.planted_medium(0, 1.0)
    for key in ("b1", "b2", "c", "l", "u"):
        assert np.array_equal(getattr(a, key), getattr(b, key), equal_nan=True), key
    assert np.array_equal(a.A1.indices, b.A1.indices) and np.array_equal(a.A2.data, b.A2.data)
    free = np.isneginf(a.l) & np.isposinf(a.u)
    assert abs(free.mean() - 0.2) < 0.01                    # 20% free columns
    assert np.all(a.l[~free] == 0.0) and np.all(a.u[~free] == 10.0)
    v = np.abs(np.concatenate([a.A1.data, a.A2.data]))
    assert v.min() >= 1e-3 * (1 - 1e-12) and v.max() <= 1e3 * (1 + 1e-12)   # +-10^U(-3,3)


@pytest.mark.parametrize("N,n,m,nnz", [(20, 160_400, 95_840, 496_400), (30, 810_900, 458_610, 2_484_900)])
def test_qap_sizes(N, n, m, nnz):
    lp = lpgen.qap_lp(0, N)
    assert (lp.n, lp.m, lp.nnz) == (n, m, nnz)


def test_mcf_structure():
    lp = lpgen.mcf_lp(0, nodes=10_000)
    # 4 commodities on 8 out-arcs per node: n = 32 * nodes flows, m1 = 4 * nodes conservation
    # rows, m2 = 8 * nodes capacity rows, 3 nonzeros per flow column
    assert (lp.n, lp.m1, lp.m2, lp.nnz) == (320_000, 40_000, 80_000, 960_000)
    assert np.all(lp.l == 0.0) and np.all(np.isposinf(lp.u))


@pytest.mark.parametrize("seed", range(3))
def test_tiny_planted_point_is_feasible_and_complementary(seed):
    lp = lpgen.planted_tiny(seed)
    x, y, z = lp.x_star, lp.y_star, lp.z_star
    assert np.allclose(lp.A1 @ x, lp.b1) and np.all(lp.A2 @ x >= lp.b2 - 1e-12)
    assert np.allclose(lp.A1.T @ y[:lp.m1] + lp.A2.T @ y[lp.m1:] + z, lp.c)
    assert np.all(y[lp.m1:] >= 0.0)
    slack = lp.A2 @ x - lp.b2
    assert np.allclose(slack * y[lp.m1:], 0.0, atol=1e-12)   # complementary slackness
    assert np.all((z <= 1e-15) | (np.abs(x - lp.l) < 1e-12))
    assert np.all((z >= -1e-15) | (np.abs(x - lp.u) < 1e-12))


def test_batch_family_ranges():
    """The batched family: m in [m_lo, m_hi] (even), n = 2.5 m, density in [0.1%, 1%] up to the
    stochastic rounding of the column counts, planted optimum feasible; reproducible."""
    lps = lpgen.batch_family(0, 24, 500, 5000)
    again = lpgen.batch_family(0, 24, 500, 5000)
    for lp, lp2 in zip(lps, again):
        assert 500 <= lp.m <= 5002 and lp.m % 2 == 0 and lp.n == int(round(2.5 * lp.m))
        dens = lp.nnz / (lp.m * lp.n)
        assert 0.8e-3 <= dens <= 1.2e-2, (lp.name, dens)
        assert lp.nnz == lp2.nnz and np.array_equal(lp.c, lp2.c)
        assert np.allclose(lp.A1 @ lp.x_star, lp.b1) and np.all(lp.A2 @ lp.x_star >= lp.b2 - 1e-9)
    ms = np.log([lp.m for lp in lps])
    assert ms.max() - ms.min() > 1.0             # spread over the log-uniform range
