"""The allocation-free power method (hpr_power_noalloc) against hpr_power.

hpr_power_noalloc serves callers that may not allocate device memory themselves; it
keeps its partial sums in a fixed array inside the library instead.  This checks that it
returns the same lambda as the context-based power method on the same scaled matrix,
to the 1e-10 relative tolerance used for lambda elsewhere, on two calls in a row (the
second call starts from whatever the first left in the shared array).  The file is named
so that pytest collects it last.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2408_12179_b300 import hpr, lpgen

pytestmark = pytest.mark.gpu


def _device_csr(torch, M):
    M = sp.csr_matrix(M)
    rp = torch.tensor(M.indptr.astype(np.int32), device="cuda")
    ci = torch.tensor(M.indices.astype(np.int32), device="cuda")
    v = torch.tensor(M.data.astype(np.float64), device="cuda")
    return (rp, ci, v), tuple(t.data_ptr() for t in (rp, ci, v))


@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_power_noalloc_matches_hpr_power(name):
    torch = pytest.importorskip("torch")
    lp = lpgen.planted_tiny(3) if name == "tiny" else lpgen.planted_medium(1, 0.02)
    with hpr.Solver(lp) as s:
        lam_ref, it_ref = s.power()
        sc = s.scaling()
    A = lp.A
    As = sp.csr_matrix((sc["As"], A.indices, A.indptr), shape=A.shape)
    keepA, pA = _device_csr(torch, As)
    keepT, pT = _device_csr(torch, As.T.tocsr())
    u = torch.empty(lp.m, dtype=torch.float64, device="cuda")
    sv = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    seed = hpr.hpr_default_options().seed
    for _ in range(2):
        u.fill_(np.nan)
        lam, it = hpr.hpr_power_noalloc(lp.m, lp.n, pA, pT, seed, 5000, 1e-10,
                                        u.data_ptr(), sv.data_ptr())
        torch.cuda.synchronize()
        assert lam == pytest.approx(lam_ref, rel=1e-10)
        assert abs(it - it_ref) <= 1
        uu = u.cpu().numpy()
        assert np.linalg.norm(uu) == pytest.approx(1.0, rel=1e-12)
        # s = A^T u of the last step, and lambda its squared norm up to the last update
        assert np.all(np.isfinite(sv.cpu().numpy()))


def test_power_noalloc_rejects_bad_sizes():
    with pytest.raises(hpr.HprError) as e:
        hpr.hpr_power_noalloc(0, 5, (1, 1, 1), (1, 1, 1), 0, 10, 1e-10, 1, 1)
    assert e.value.code == hpr.HPR_ERR_ARG
    with pytest.raises(hpr.HprError) as e:
        hpr.hpr_power_noalloc(2 ** 31, 5, (1, 1, 1), (1, 1, 1), 0, 10, 1e-10, 1, 1)
    assert e.value.code == hpr.HPR_ERR_ARG
