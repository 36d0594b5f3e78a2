"""ctypes binding of the C ABI in ``include/hpr.h`` (same names, argument marshalling only).

Every step of the method runs in the CUDA library ``libhpr_b300.so``; this module only
converts numpy / SciPy inputs into the C structures and copies results out.  Importing
it does not need a GPU; calling into it without the built library raises.

    from paper_2408_12179_b300 import hpr
    res = hpr.solve(lp, tol=1e-8)          # lp: lpgen.LP or any object with A1, A2, b1, ...
    res["x"], res["y"], res["z"], res["info"]
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhpr_b300.so")

HPR_OK, HPR_MAX_ITER, HPR_TIME_LIMIT = 0, 1, 2
HPR_ERR_ARG, HPR_ERR_ZERO_MATRIX, HPR_ERR_NOMEM, HPR_ERR_CUDA = -1, -2, -3, -4
HPR_ERR_DEVICE_TIMEOUT, HPR_ERR_NUMERIC, HPR_ERR_STATE, HPR_ERR_NO_DEVICE = -5, -6, -7, -8

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)


class hpr_csr(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", _I64), ("col_idx", _I32), ("val", _D)]


class hpr_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int64),
                ("time_limit_s", ctypes.c_double), ("check_every", ctypes.c_int64),
                ("alpha1", ctypes.c_double), ("alpha2", ctypes.c_double),
                ("alpha3", ctypes.c_double), ("sigma0", ctypes.c_double),
                ("ruiz_iters", ctypes.c_int64), ("pc_alpha", ctypes.c_double),
                ("power_max_iter", ctypes.c_int64), ("power_tol", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("lambda_fixed", ctypes.c_double),
                ("restart", ctypes.c_int64), ("sigma_update", ctypes.c_int64),
                ("trace_iters", ctypes.c_int64), ("use_graph", ctypes.c_int64),
                ("verbose", ctypes.c_int64), ("cuda_stream", ctypes.c_void_p),
                ("precision", ctypes.c_int64), ("switch_tol", ctypes.c_double),
                ("halpern", ctypes.c_int64), ("reflect", ctypes.c_int64),
                ("autotune", ctypes.c_int64), ("sell_steps_a", ctypes.c_int64),
                ("sell_steps_t", ctypes.c_int64), ("unit_cost_a", ctypes.c_double),
                ("unit_cost_t", ctypes.c_double), ("sigma_policy", ctypes.c_int64),
                ("policy_seed", ctypes.c_uint64), ("policy_margin", ctypes.c_double),
                ("persistent", ctypes.c_int64), ("pdl", ctypes.c_int64),
                ("gather_tiles", ctypes.c_int64), ("tile_len", ctypes.c_int64)]


class hpr_info(ctypes.Structure):
    _fields_ = [("primal_obj", ctypes.c_double), ("dual_obj", ctypes.c_double),
                ("err_p", ctypes.c_double), ("err_d", ctypes.c_double),
                ("err_gap", ctypes.c_double), ("kkt", ctypes.c_double),
                ("sigma", ctypes.c_double), ("lambda", ctypes.c_double),
                ("solve_time_s", ctypes.c_double), ("power_time_s", ctypes.c_double),
                ("time_to_1e4_s", ctypes.c_double), ("iters_to_1e4", ctypes.c_int64),
                ("iters", ctypes.c_int64), ("restarts", ctypes.c_int64),
                ("power_iters", ctypes.c_int64), ("n_checks", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("status", ctypes.c_int64),
                ("iters_fp32", ctypes.c_int64),
                ("policy_decisions", ctypes.c_int64), ("policy_fallbacks", ctypes.c_int64),
                ("power_rel_change", ctypes.c_double), ("path", ctypes.c_int64), ("path_ctas", ctypes.c_int64),
                ("x_tiles", ctypes.c_int64)]


class hpr_check_record(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("r", ctypes.c_int64), ("t", ctypes.c_int64),
                ("kind", ctypes.c_int64), ("cause", ctypes.c_int64),
                ("sigma", ctypes.c_double), ("err_p", ctypes.c_double),
                ("err_d", ctypes.c_double), ("err_gap", ctypes.c_double),
                ("kkt", ctypes.c_double), ("pobj", ctypes.c_double), ("dobj", ctypes.c_double),
                ("Rt", ctypes.c_double), ("R0", ctypes.c_double), ("sigma_next", ctypes.c_double),
                ("Dx", ctypes.c_double), ("Dy", ctypes.c_double), ("elapsed_s", ctypes.c_double),
                ("action", ctypes.c_int64), ("sigma_rule", ctypes.c_double)]


# every symbol the header declares, with (restype, argtypes)
SIGNATURES = {
    "hpr_default_options": (ctypes.c_int, [ctypes.POINTER(hpr_options)]),
    "hpr_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(hpr_csr),
                                  ctypes.POINTER(hpr_csr), _D, _D, _D, _D, _D,
                                  ctypes.POINTER(hpr_options)]),
    "hpr_set_options": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(hpr_options)]),
    "hpr_power": (ctypes.c_int, [ctypes.c_void_p, _D, _I64]),
    "hpr_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "hpr_get": (ctypes.c_int, [ctypes.c_void_p, _D, _D, _D, ctypes.POINTER(hpr_info)]),
    "hpr_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "hpr_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "hpr_get_scaling": (ctypes.c_int, [ctypes.c_void_p, _D, _D, _D, _D, _D, _D, _D, _D]),
    "hpr_get_checks": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(hpr_check_record),
                                      ctypes.c_int64, _I64]),
    "hpr_get_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _D, _D, _D, _D, _D]),
    "hpr_time_iteration": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _D, _D, _D]),
    "hpr_power_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, _D, _I64]),
    "hpr_get_layout": (ctypes.c_int, [ctypes.c_void_p, _I64, _D, _I64]),
    "hpr_memory_probe": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, _D, _D]),
    "hpr_fp64_probe": (ctypes.c_int, [ctypes.c_void_p, _D]),
    "hpr_bounds_violations": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64)]),
    "hpr_layout_plan": (ctypes.c_int, [ctypes.POINTER(hpr_csr), ctypes.c_int64, ctypes.c_double, _I64, _I64,
                                       _I64, _I32, _I32, _I32, ctypes.POINTER(ctypes.c_uint8), _I32, _I32,
                                       _I32]),
    "hpr_tile_plan": (ctypes.c_int, [ctypes.POINTER(hpr_csr), ctypes.c_int64, ctypes.c_int64, _I64, _I32, _I32,
                                     _I32, _I32, _I32, _I32, _I32, _I32, ctypes.POINTER(ctypes.c_uint16), _I32]),
    "hpr_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "hpr_batch_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "hpr_batch_stats": (ctypes.c_int, [ctypes.c_void_p, _D, _I64, _I64]),
    "hpr_batch_destroy": (None, [ctypes.c_void_p]),
    "hpr_set_policy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hpr_policy_features": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "hpr_mlp_param_count": (ctypes.c_int, []),
    "hpr_mlp_infer": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "hpr_mlp_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, _D]),
    "hpr_mlp_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_uint64, ctypes.c_void_p]),
    "hpr_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "hpr_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "hpr_destroy": (None, [ctypes.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA solver library not built: {path} is missing "
                               "(run python -m paper_2408_12179_b300.build)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class HprError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{hpr_status_str(code)}: {msg}")
        self.code = code


def hpr_status_str(code: int) -> str:
    return load().hpr_status_str(int(code)).decode()


def hpr_last_error(ctx) -> str:
    return load().hpr_last_error(ctx).decode()


def hpr_default_options(**overrides) -> hpr_options:
    o = hpr_options()
    load().hpr_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(a, t=_D):
    return a.ctypes.data_as(t) if a is not None else ctypes.cast(None, t)


def _block(M, n):
    """(hpr_csr, keep-alive tuple) for a SciPy CSR block (or None)."""
    if M is None or M.shape[0] == 0:
        return hpr_csr(0, n, 0, None, None, None), ()
    rp = np.ascontiguousarray(M.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(M.indices, dtype=np.int32)
    v = np.ascontiguousarray(M.data, dtype=np.float64)
    return hpr_csr(M.shape[0], M.shape[1], v.size, _ptr(rp, _I64), _ptr(ci, _I32), _ptr(v)), (rp, ci, v)


def layout_plan(M, steps_max=40, unit_cost=64.0):
    """The sliced-ELL layout hpr_create builds for the rows of the SciPy CSR matrix M (host
    only, no GPU): dict of numpy arrays row_order, srow, sptr, slg, col, src, wstart."""
    lib = load()
    B, keep = _block(M, M.shape[1])
    ns, ne, nu = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib.hpr_layout_plan(ctypes.byref(B), int(steps_max), float(unit_cost), ctypes.byref(ns), ctypes.byref(ne),
                               ctypes.byref(nu), None, None, None, None, None, None, None))
    out = dict(row_order=np.zeros(M.shape[0], np.int32), srow=np.zeros(ns.value + 1, np.int32),
               sptr=np.zeros(ns.value + 1, np.int32), slg=np.zeros(ns.value, np.uint8),
               col=np.zeros(ne.value, np.int32), src=np.zeros(ne.value, np.int32),
               wstart=np.zeros(nu.value + 1, np.int32))
    _check(lib.hpr_layout_plan(ctypes.byref(B), int(steps_max), float(unit_cost), None, None, None,
                               _ptr(out["row_order"], _I32), _ptr(out["srow"], _I32), _ptr(out["sptr"], _I32),
                               _ptr(out["slg"], ctypes.POINTER(ctypes.c_uint8)), _ptr(out["col"], _I32),
                               _ptr(out["src"], _I32), _ptr(out["wstart"], _I32)))
    del keep
    return out


def tile_plan(M, tile_len, grid=148):
    """The gather-tiled layout of the x phase for the rows of the SciPy CSR matrix M (host
    only, no GPU; see hpr_tile_plan in include/hpr.h): dict of numpy arrays row_order, bstart,
    ustart, cta_blk, wstart, smeta (slices x 4), oslot, slot_ptr, col (uint16), src."""
    lib = load()
    B, keep = _block(M, M.shape[1])
    sz = np.zeros(6, np.int64)
    _check(lib.hpr_tile_plan(ctypes.byref(B), int(tile_len), int(grid), _ptr(sz, _I64), None, None, None, None,
                             None, None, None, None, None, None))
    nblk, ns, ne, nsub, nu, g = (int(v) for v in sz)
    out = dict(row_order=np.zeros(M.shape[0], np.int32), bstart=np.zeros(nblk + 1, np.int32),
               ustart=np.zeros(nblk + 1, np.int32), cta_blk=np.zeros(g, np.int32),
               wstart=np.zeros(nu + 1, np.int32), smeta=np.zeros((ns, 4), np.int32),
               oslot=np.zeros(nsub, np.int32), slot_ptr=np.zeros(M.shape[0] + 1, np.int32),
               col=np.zeros(ne, np.uint16), src=np.zeros(ne, np.int32))
    _check(lib.hpr_tile_plan(ctypes.byref(B), int(tile_len), int(grid), None, _ptr(out["row_order"], _I32),
                             _ptr(out["bstart"], _I32), _ptr(out["ustart"], _I32), _ptr(out["cta_blk"], _I32),
                             _ptr(out["wstart"], _I32), _ptr(out["smeta"], _I32), _ptr(out["oslot"], _I32),
                             _ptr(out["slot_ptr"], _I32), _ptr(out["col"], ctypes.POINTER(ctypes.c_uint16)),
                             _ptr(out["src"], _I32)))
    del keep
    return out


def _check(code, ctx=None):
    if code < 0:
        raise HprError(code, hpr_last_error(ctx))
    return code


def hpr_create(A1, A2, b1, b2, c, l, u, options: hpr_options | None = None):
    """Create a solver context from host data (SciPy CSR blocks and numpy vectors).
    Returns an opaque handle for the other calls; raises HprError on failure."""
    lib = load()
    n = (A1 if A1 is not None and A1.shape[0] else A2).shape[1]
    s1, k1 = _block(A1, n)
    s2, k2 = _block(A2, n)
    vecs = [np.ascontiguousarray(v, dtype=np.float64) if v is not None else None
            for v in (b1, b2, c, l, u)]
    h = ctypes.c_void_p()
    code = lib.hpr_create(ctypes.byref(h), ctypes.byref(s1), ctypes.byref(s2),
                          *[_ptr(v) if v is not None and v.size else _ptr(np.zeros(1)) for v in vecs],
                          ctypes.byref(options) if options is not None else None)
    if code < 0:
        raise HprError(code, lib.hpr_last_error(None).decode())
    del k1, k2
    return h


def hpr_set_options(ctx, options: hpr_options):
    return _check(load().hpr_set_options(ctx, ctypes.byref(options)), ctx)


def hpr_power(ctx):
    lam = ctypes.c_double()
    it = ctypes.c_int64()
    _check(load().hpr_power(ctx, ctypes.byref(lam), ctypes.byref(it)), ctx)
    return lam.value, it.value


def hpr_solve(ctx, tol: float) -> int:
    return _check(load().hpr_solve(ctx, float(tol)), ctx)


def _info_dict(I: hpr_info) -> dict:
    return {name: getattr(I, name) for name, _ in hpr_info._fields_}


def hpr_get(ctx, n: int, m: int):
    x, y, z = np.empty(n), np.empty(m), np.empty(n)
    I = hpr_info()
    _check(load().hpr_get(ctx, _ptr(x), _ptr(y), _ptr(z), ctypes.byref(I)), ctx)
    return x, y, z, _info_dict(I)


def hpr_get_scaling(ctx, n: int, m: int, nnz: int):
    out = dict(Dr=np.empty(m), Dc=np.empty(n), As=np.empty(nnz), bs=np.empty(m),
               cs=np.empty(n), ls=np.empty(n), us=np.empty(n))
    beta = np.empty(2)
    _check(load().hpr_get_scaling(ctx, _ptr(out["Dr"]), _ptr(out["Dc"]), _ptr(out["As"]),
                                  _ptr(out["bs"]), _ptr(out["cs"]), _ptr(out["ls"]),
                                  _ptr(out["us"]), _ptr(beta)), ctx)
    out["beta_b"], out["beta_c"] = float(beta[0]), float(beta[1])
    return out


def hpr_get_checks(ctx):
    cnt = ctypes.c_int64()
    _check(load().hpr_get_checks(ctx, None, 0, ctypes.byref(cnt)), ctx)
    arr = (hpr_check_record * max(cnt.value, 1))()
    _check(load().hpr_get_checks(ctx, arr, cnt.value, ctypes.byref(cnt)), ctx)
    return [{name: getattr(r, name) for name, _ in hpr_check_record._fields_} for r in arr[:cnt.value]]


def hpr_get_trace(ctx, k: int, n: int, m: int):
    out = dict(xbar=np.empty(n), xhat=np.empty(n), x=np.empty(n), ybar=np.empty(m), y=np.empty(m))
    _check(load().hpr_get_trace(ctx, int(k), _ptr(out["xbar"]), _ptr(out["xhat"]), _ptr(out["x"]),
                                _ptr(out["ybar"]), _ptr(out["y"])), ctx)
    return out


def hpr_time_iteration(ctx, reps: int):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().hpr_time_iteration(ctx, int(reps), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), ctx)
    return a.value, b.value, c.value


def bounds_violations() -> int:
    """Out-of-range gather indices counted by the bounds-checking build (-1: normal build)."""
    c = ctypes.c_int64()
    _check(load().hpr_bounds_violations(ctypes.byref(c)), None)
    return int(c.value)


def fp64_probe(stream=None):
    """FP64 warp instructions per second of the whole GPU, in 1e9/s (see hpr_fp64_probe in
    include/hpr.h)."""
    r = ctypes.c_double()
    _check(load().hpr_fp64_probe(stream, ctypes.byref(r)), None)
    return r.value


def memory_probe(read_bytes=72_000_000, gather_len=1 << 18, stream=None):
    """(read-only stream GB/s, random-gather rate in 1e9/s) measured by the library's probe
    kernels (see hpr_memory_probe in include/hpr.h)."""
    r, g = ctypes.c_double(), ctypes.c_double()
    _check(load().hpr_memory_probe(int(read_bytes), int(gather_len), stream, ctypes.byref(r), ctypes.byref(g)), None)
    return r.value, g.value


def hpr_power_noalloc(m, n, A_ptrs, At_ptrs, seed, max_iter, tol, u_ptr, s_ptr, stream=None):
    """Allocation-free power method on device CSR arrays given as raw device addresses
    (A_ptrs / At_ptrs = (row_ptr, col_idx, val)); u_ptr (m doubles) and s_ptr (n) are
    device output buffers.  Returns (lambda, iterations).

    stream: a cudaStream_t handle.  When None and torch is loaded, torch's current CUDA
    stream is used, so that buffers filled on it are ready before the call reads them;
    without torch, None is the legacy default stream and the caller orders its own streams."""
    if stream is None:
        import sys
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
            stream = torch.cuda.current_stream().cuda_stream
    lam = ctypes.c_double()
    it = ctypes.c_int64()
    code = load().hpr_power_noalloc(int(m), int(n), *A_ptrs, *At_ptrs, int(seed), int(max_iter),
                                    float(tol), u_ptr, s_ptr, stream, ctypes.byref(lam),
                                    ctypes.byref(it))
    _check(code, None)
    return lam.value, it.value


def _f32(a, cols=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def mlp_param_count():
    return int(load().hpr_mlp_param_count())


def mlp_infer(w, X):
    """Outputs (n x 5) of the sigma policy network for the rows of X (n x 64)."""
    w, X = _f32(w), _f32(X, 64)
    Q = np.empty((X.shape[0], 5), np.float32)
    _check(load().hpr_mlp_infer(w.ctypes.data, X.shape[0], X.ctypes.data, Q.ctypes.data), None)
    return Q


def mlp_grad(w, X, act, y):
    """(loss, gradient) of the network's regression loss on the GPU."""
    w, X, y = _f32(w), _f32(X, 64), _f32(y)
    act = np.ascontiguousarray(act, dtype=np.int32)
    g = np.empty(w.size, np.float32)
    loss = ctypes.c_double()
    _check(load().hpr_mlp_grad(w.ctypes.data, X.shape[0], X.ctypes.data, act.ctypes.data, y.ctypes.data,
                               g.ctypes.data, ctypes.byref(loss)), None)
    return loss.value, g


def mlp_train(w, X, act, y, epochs=50, batch=256, lr=1e-3, seed=1):
    """Trains on the GPU; returns (weights, per-epoch losses)."""
    w, X, y = _f32(w).copy(), _f32(X, 64), _f32(y)
    act = np.ascontiguousarray(act, dtype=np.int32)
    hist = np.zeros(max(int(epochs), 1))
    _check(load().hpr_mlp_train(w.ctypes.data, X.shape[0], X.ctypes.data, act.ctypes.data, y.ctypes.data,
                                int(epochs), int(batch), float(lr), int(seed), hist.ctypes.data), None)
    return w, hist[:int(epochs)]


def hpr_destroy(ctx):
    if ctx is not None and ctx.value:
        load().hpr_destroy(ctx)


class Solver:
    """Context manager around one hpr_ctx for an LP object (fields A1, A2, b1, b2, c, l, u)."""

    def __init__(self, lp, **opts):
        self.n, self.m, self.nnz = lp.n, lp.m, lp.nnz
        self.options = hpr_default_options(**opts)
        self.ctx = hpr_create(lp.A1, lp.A2, lp.b1, lp.b2, lp.c, lp.l, lp.u, self.options)

    def set_options(self, **opts):
        for k, v in opts.items():
            setattr(self.options, k, v)
        hpr_set_options(self.ctx, self.options)

    def power(self):
        return hpr_power(self.ctx)

    def solve(self, tol=None):
        status = hpr_solve(self.ctx, self.options.tol if tol is None else tol)
        x, y, z, info = hpr_get(self.ctx, self.n, self.m)
        return dict(x=x, y=y, z=z, info=info, status=status)

    def scaling(self):
        return hpr_get_scaling(self.ctx, self.n, self.m, self.nnz)

    def checks(self):
        return hpr_get_checks(self.ctx)

    def trace(self, k):
        return hpr_get_trace(self.ctx, k, self.n, self.m)

    def get_state(self) -> bytes:
        """The checkpoint of the last solve (hpr_get_state): an opaque blob."""
        need = ctypes.c_int64()
        _check(load().hpr_get_state(self.ctx, None, 0, ctypes.byref(need)), self.ctx)
        buf = ctypes.create_string_buffer(need.value)
        _check(load().hpr_get_state(self.ctx, buf, need.value, ctypes.byref(need)), self.ctx)
        return buf.raw

    def set_state(self, blob: bytes):
        """The next solve starts from this checkpoint (hpr_set_state)."""
        _check(load().hpr_set_state(self.ctx, blob, len(blob)), self.ctx)

    def result(self):
        """(x, y, z, info) of the last solve (e.g. one run through a Batch)."""
        x, y, z, info = hpr_get(self.ctx, self.n, self.m)
        return dict(x=x, y=y, z=z, info=info, status=int(info["status"]))

    def set_policy(self, w):
        """Policy network weights for sigma_policy = 2 (None removes them)."""
        if w is None:
            _check(load().hpr_set_policy(self.ctx, None), self.ctx)
            return
        self._policy_w = np.ascontiguousarray(w, dtype=np.float32)
        _check(load().hpr_set_policy(self.ctx, self._policy_w.ctypes.data), self.ctx)

    def policy_features(self, rec):
        out = np.empty(64, np.float32)
        _check(load().hpr_policy_features(self.ctx, int(rec), out.ctypes.data), self.ctx)
        return out

    def layout(self):
        """Sliced-ELL layout parameters of A and A^T: dict of (A, A^T) pairs."""
        st = (ctypes.c_int64 * 2)()
        uc = (ctypes.c_double * 2)()
        un = (ctypes.c_int64 * 2)()
        _check(load().hpr_get_layout(self.ctx, st, uc, un), self.ctx)
        return dict(sell_steps=tuple(st), unit_cost=tuple(uc), units=tuple(un))

    def time_iteration(self, reps=50):
        return hpr_time_iteration(self.ctx, reps)

    def close(self):
        hpr_destroy(self.ctx)
        self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Context manager solving several Solver contexts in lock step with fused launches
    (hpr_batch_*).  The solvers stay owned by the caller and must outlive the batch."""

    def __init__(self, solvers, stream=None):
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.ctx.value for s in self.solvers])
        out = ctypes.c_void_p()
        code = load().hpr_batch_create(ctypes.byref(out), len(self.solvers), arr, stream)
        _check(code, None)
        self.b = out

    def solve(self, tol=1e-8):
        """Returns the batch status and the per-LP results."""
        status = load().hpr_batch_solve(self.b, float(tol))
        if status < 0:
            _check(status, None)
        return status, [s.result() for s in self.solvers]

    def stats(self):
        t = ctypes.c_double()
        p = ctypes.c_int64()
        f = ctypes.c_int64()
        _check(load().hpr_batch_stats(self.b, ctypes.byref(t), ctypes.byref(p), ctypes.byref(f)), None)
        return dict(solve_time_s=t.value, periods=p.value, fused_launches=f.value)

    def close(self):
        if self.b is not None and self.b.value:
            load().hpr_batch_destroy(self.b)
        self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve(lp, tol=1e-8, **opts):
    """One-shot solve: returns dict(x, y, z, info, status) in the original space."""
    with Solver(lp, **opts) as s:
        return s.solve(tol)
