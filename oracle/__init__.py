"""HPR-LP oracle -- TEST INFRASTRUCTURE ONLY.

A plain FP64 CPU implementation of HPR-LP (arXiv 2408.12179) used to check the CUDA
solver.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the solver package never does.

``solve`` runs the C implementation in ``hpr_oracle.c`` (preprocessing of Section 4.1,
power method, Algorithm 2 with the closed forms of Section 3.3, restart criteria of
Section 3.1, Algorithm 3 and the termination test of Section 4.1).  ``kkt`` (module
``oracle.kkt``) is a second, independent evaluation of the termination quantities on the
original LP, written in numpy.

Parity pins: see the test-suite (``tests/test_oracle_*.py``).  Every function here is
pinned; the restart / sigma decision sequence, for which the paper prints no trace, is
rebuilt check by check from the rules of Section 3.1 and Algorithm 3
(``tests/test_oracle_restart.py``, which also plants misreadings of the rules in a copy of
the C source and checks that the rebuild rejects each one).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

OI = ["status", "iters", "restarts", "sigma", "lambda", "power_iters", "pobj", "dobj",
      "err_p", "err_d", "err_gap", "kkt", "beta_b", "beta_c", "n_checks", "seconds"]
OC = ["k", "r", "t", "sigma", "err_p", "err_d", "err_gap", "kkt", "pobj", "dobj",
      "Rt", "R0", "cause", "sigma_next", "kind", "Dx", "Dy"]

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)


class _LP(ctypes.Structure):
    _fields_ = [("m1", ctypes.c_int64), ("m2", ctypes.c_int64), ("n", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("row_ptr", _I64), ("col_idx", _I32), ("val", _D),
                ("b", _D), ("c", _D), ("l", _D), ("u", _D)]


class _Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int64),
                ("check_every", ctypes.c_int64), ("alpha1", ctypes.c_double),
                ("alpha2", ctypes.c_double), ("alpha3", ctypes.c_double),
                ("sigma0", ctypes.c_double), ("ruiz_iters", ctypes.c_int64),
                ("pc_alpha", ctypes.c_double), ("power_max_iter", ctypes.c_int64),
                ("power_tol", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("lambda_fixed", ctypes.c_double), ("restart", ctypes.c_int64),
                ("sigma_update", ctypes.c_int64), ("trace_iters", ctypes.c_int64),
                ("halpern", ctypes.c_int64), ("reflect", ctypes.c_int64)]


class _Out(ctypes.Structure):
    _fields_ = [("x", _D), ("y", _D), ("z", _D), ("info", _D), ("trace", _D),
                ("checks", _D), ("checks_cap", ctypes.c_int64), ("Dr", _D), ("Dc", _D),
                ("As_val", _D), ("bs", _D), ("cs", _D), ("ls", _D), ("us", _D)]


DEFAULTS = dict(tol=1e-8, max_iter=100_000, check_every=150, alpha1=0.2, alpha2=0.6,
                alpha3=0.2, sigma0=1.0, ruiz_iters=10, pc_alpha=1.0, power_max_iter=5000,
                power_tol=1e-10, seed=0x48505221, lambda_fixed=0.0, restart=1,
                sigma_update=1, trace_iters=0, halpern=1, reflect=1)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _lib.orc_hpr.argtypes = [ctypes.POINTER(_LP), ctypes.POINTER(_Opts), ctypes.POINTER(_Out)]
        _lib.orc_hpr.restype = ctypes.c_int
        _lib.orc_scale.argtypes = [ctypes.POINTER(_LP), ctypes.c_int64, ctypes.c_double,
                                   _D, _D, _D, _D, _D, _D, _D, _D]
        _lib.orc_scale.restype = ctypes.c_int
        _lib.orc_power.argtypes = [ctypes.c_int64, ctypes.c_int64, _I64, _I32, _D,
                                   ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, _I64]
        _lib.orc_power.restype = ctypes.c_double
    return _lib


def _p(a, t=_D):
    return a.ctypes.data_as(t) if a is not None else ctypes.cast(None, t)


class _Problem:
    """Keeps the contiguous arrays of an LP alive while C holds pointers to them."""

    def __init__(self, lp):
        A = lp.A
        self.m1, self.m2, self.n = lp.m1, lp.m2, lp.n
        self.rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(A.indices, dtype=np.int32)
        self.v = np.ascontiguousarray(A.data, dtype=np.float64)
        self.b = np.ascontiguousarray(lp.b, dtype=np.float64)
        self.c = np.ascontiguousarray(lp.c, dtype=np.float64)
        self.l = np.ascontiguousarray(lp.l, dtype=np.float64)
        self.u = np.ascontiguousarray(lp.u, dtype=np.float64)
        self.s = _LP(self.m1, self.m2, self.n, self.v.size, _p(self.rp, _I64), _p(self.ci, _I32),
                     _p(self.v), _p(self.b), _p(self.c), _p(self.l), _p(self.u))


def scale(lp, ruiz_iters=10, pc_alpha=1.0):
    """Preprocessing of Section 4.1.  Returns dict(As (CSR values of A), Dr, Dc, bs, cs,
    ls, us, beta_b, beta_c)."""
    P = _Problem(lp)
    m, n = lp.m, lp.n
    out = dict(As=np.empty(P.v.size), Dr=np.empty(m), Dc=np.empty(n), bs=np.empty(m),
               cs=np.empty(n), ls=np.empty(n), us=np.empty(n))
    beta = np.empty(2)
    lib().orc_scale(ctypes.byref(P.s), ruiz_iters, pc_alpha, _p(out["As"]), _p(out["Dr"]),
                    _p(out["Dc"]), _p(out["bs"]), _p(out["cs"]), _p(out["ls"]), _p(out["us"]),
                    _p(beta))
    out["beta_b"], out["beta_c"] = float(beta[0]), float(beta[1])
    return out


def power(A, seed=DEFAULTS["seed"], max_iter=5000, tol=1e-10):
    """lambda_1(A A^T) by the power method of the oracle.  Returns (lambda, iterations)."""
    import scipy.sparse as sp

    A = sp.csr_matrix(A)
    rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.indices, dtype=np.int32)
    v = np.ascontiguousarray(A.data, dtype=np.float64)
    it = np.zeros(1, dtype=np.int64)
    lam = lib().orc_power(A.shape[0], A.shape[1], _p(rp, _I64), _p(ci, _I32), _p(v),
                          seed, max_iter, tol, _p(it, _I64))
    return float(lam), int(it[0])


def solve(lp, checks_cap=100_000, **opts):
    """Run the oracle HPR-LP on `lp`.  Keyword options as in DEFAULTS.  Returns a dict:
    x, y, z (original space), info (dict), checks (list of dicts), and when requested
    trace (dict of arrays, shape (trace_iters, .)) and the scaled data."""
    o = dict(DEFAULTS)
    o.update(opts)
    P = _Problem(lp)
    m, n = lp.m, lp.n
    O = _Opts(**{k: o[k] for k, _ in _Opts._fields_})
    res = dict(x=np.empty(n), y=np.empty(m), z=np.empty(n), info=np.zeros(len(OI)))
    tr_n = int(o["trace_iters"])
    trace = np.zeros((tr_n, 3 * n + 2 * m)) if tr_n > 0 else None
    checks = np.zeros((checks_cap, len(OC)))
    scal = dict(Dr=np.empty(m), Dc=np.empty(n), As=np.empty(P.v.size), bs=np.empty(m),
                cs=np.empty(n), ls=np.empty(n), us=np.empty(n))
    out = _Out(_p(res["x"]), _p(res["y"]), _p(res["z"]), _p(res["info"]), _p(trace),
               _p(checks), checks_cap, _p(scal["Dr"]), _p(scal["Dc"]), _p(scal["As"]),
               _p(scal["bs"]), _p(scal["cs"]), _p(scal["ls"]), _p(scal["us"]))
    lib().orc_hpr(ctypes.byref(P.s), ctypes.byref(O), ctypes.byref(out))
    info = {k: float(v) for k, v in zip(OI, res["info"])}
    info["status"] = int(info["status"])
    info["iters"] = int(info["iters"])
    nchk = min(int(info["n_checks"]), checks_cap)
    res["info"] = info
    res["checks"] = [dict(zip(OC, row)) for row in checks[:nchk]]
    res["scaled"] = scal
    if trace is not None:
        k = min(tr_n, info["iters"])
        res["trace"] = dict(xbar=trace[:k, :n], xhat=trace[:k, n:2 * n], x=trace[:k, 2 * n:3 * n],
                            ybar=trace[:k, 3 * n:3 * n + m], y=trace[:k, 3 * n + m:])
    return res
