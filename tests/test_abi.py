"""The C-ABI library: builds, exports every symbol include/hpr.h declares, matches the
header's struct layouts, and rejects bad input on the host (no GPU needed: validation
runs before any device call)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2408_12179_b300 import build, hpr, lpgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hpr.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return hpr.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hpr_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (hpr_\w+)", out))
    decl = declared_functions()
    assert decl, "no declarations parsed"
    missing = [f for f in decl if f not in exported]
    assert not missing, missing
    assert set(decl) == set(hpr.SIGNATURES)


def test_struct_layouts_match_header(tmp_path):
    import ctypes

    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "hpr.h"\n'
                   'int main(){printf("%zu %zu %zu %zu %zu\\n", sizeof(hpr_options), sizeof(hpr_info),'
                   ' sizeof(hpr_check_record), sizeof(hpr_csr), offsetof(hpr_options, cuda_stream));}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(hpr.hpr_options), ctypes.sizeof(hpr.hpr_info),
                   ctypes.sizeof(hpr.hpr_check_record), ctypes.sizeof(hpr.hpr_csr),
                   hpr.hpr_options.cuda_stream.offset]


def test_default_options_are_the_papers(lib):
    o = hpr.hpr_default_options()
    assert (o.tol, o.check_every, o.alpha1, o.alpha2, o.alpha3, o.sigma0, o.ruiz_iters, o.pc_alpha) == \
        (1e-8, 150, 0.2, 0.6, 0.2, 1.0, 10, 1.0)


def _tiny():
    return lpgen.planted_tiny(0)


def _create(lp, **kw):
    d = dict(A1=lp.A1, A2=lp.A2, b1=lp.b1, b2=lp.b2, c=lp.c, l=lp.l, u=lp.u)
    d.update(kw)
    return hpr.hpr_create(d["A1"], d["A2"], d["b1"], d["b2"], d["c"], d["l"], d["u"],
                          hpr.hpr_default_options())


@pytest.mark.parametrize("case", ["nan_value", "unsorted", "duplicate", "l_gt_u", "l_inf",
                                  "u_minf", "nan_c", "col_range"])
def test_invalid_input_rejected(lib, case):
    lp = _tiny()
    A1 = lp.A1.copy()
    kw = {}
    if case == "nan_value":
        A1.data[0] = np.nan
        kw["A1"] = A1
    elif case in ("unsorted", "duplicate"):
        row = int(np.argmax(np.diff(A1.indptr) >= 2))
        p = A1.indptr[row]
        if case == "unsorted":
            A1.indices[p], A1.indices[p + 1] = A1.indices[p + 1], A1.indices[p]
        else:
            A1.indices[p + 1] = A1.indices[p]
        kw["A1"] = A1
    elif case == "l_gt_u":
        l = lp.l.copy(); l[3] = 20.0
        kw["l"] = l
    elif case == "l_inf":
        l = lp.l.copy(); l[150] = np.inf
        kw["l"] = l
    elif case == "u_minf":
        u = lp.u.copy(); u[4] = -np.inf; l = lp.l.copy(); l[4] = -np.inf
        kw["u"], kw["l"] = u, l
    elif case == "nan_c":
        c = lp.c.copy(); c[7] = np.nan
        kw["c"] = c
    elif case == "col_range":
        A1.indices[-1] = lp.n + 5
        kw["A1"] = A1
    with pytest.raises(hpr.HprError) as e:
        _create(lp, **kw)
    assert e.value.code == hpr.HPR_ERR_ARG


def test_zero_matrix_rejected(lib):
    lp = _tiny()
    Z1 = sp.csr_matrix((lp.m1, lp.n))
    Z2 = sp.csr_matrix(([0.0], ([0], [0])), shape=(lp.m2, lp.n))
    with pytest.raises(hpr.HprError) as e:
        _create(lp, A1=lpgen._canonical(Z1), A2=Z2)
    assert e.value.code == hpr.HPR_ERR_ZERO_MATRIX


def test_status_strings(lib):
    assert hpr.hpr_status_str(0) == "HPR_OK"
    assert hpr.hpr_status_str(-5) == "HPR_ERR_DEVICE_TIMEOUT"
    assert hpr.hpr_status_str(99) == "HPR_UNKNOWN"


@pytest.mark.parametrize("bad", [dict(sell_steps_a=-1), dict(sell_steps_t=5000), dict(unit_cost_t=-2.0),
                                 dict(autotune=2), dict(halpern=3), dict(reflect=-1), dict(precision=2),
                                 dict(gather_tiles=3), dict(gather_tiles=-1), dict(tile_len=1),
                                 dict(tile_len=70000)])
def test_invalid_options_rejected(lib, bad):
    lp = _tiny()
    with pytest.raises(hpr.HprError) as e:
        hpr.Solver(lp, **bad)
    assert e.value.code == hpr.HPR_ERR_ARG


def test_sizes_beyond_32_bit_indices_rejected_before_reading(lib):
    """A block declaring 2^31 nonzeros is refused from its sizes alone (the 32-bit index
    layout cannot hold it); the arrays behind it are never read."""
    import ctypes
    rp = np.array([0, 1 << 31], dtype=np.int64)
    ci = np.zeros(1, dtype=np.int32)
    va = np.ones(1)
    B = hpr.hpr_csr(1, 4, 1 << 31, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                    ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), va.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    out = ctypes.c_void_p()
    b = np.zeros(1)
    v4 = np.zeros(4)
    u4 = np.ones(4)
    code = lib.hpr_create(ctypes.byref(out), ctypes.byref(B), None, b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          None, v4.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          v4.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          u4.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    assert code == hpr.HPR_ERR_ARG
    assert "2^31" in hpr.hpr_last_error(None)


def test_power_noalloc_rejects_sizes_beyond_its_bound(lib):
    """hpr_power_noalloc accepts m, n in [1, 2^31 - 2] (its kernels step with 64-bit
    counters, so no row or entry index wraps below that bound) and refuses anything
    outside from the sizes alone, before touching the device pointers."""
    for m, n in ((2 ** 31 - 1, 5), (5, 2 ** 31 - 1), (0, 5), (5, -1)):
        with pytest.raises(hpr.HprError) as e:
            hpr.hpr_power_noalloc(m, n, (1, 1, 1), (1, 1, 1), 0, 10, 1e-10, 1, 1)
        assert e.value.code == hpr.HPR_ERR_ARG
        assert "2^31 - 2" in hpr.hpr_last_error(None)


def test_normal_build_checks_no_bounds(lib):
    """The normal build counts nothing (-1) and needs no device to say so; the bounds-checking
    build, when built, exports the same entry points."""
    assert hpr.bounds_violations() == -1
    from paper_2408_12179_b300 import build as solver_build
    if not os.path.exists(solver_build.LIB_CHECKED):
        pytest.skip("the bounds-checking build is not built")
    checked = ctypes.CDLL(solver_build.LIB_CHECKED)
    for name in declared_functions():
        getattr(checked, name)
