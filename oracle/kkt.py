"""Independent evaluation of the termination quantities -- TEST INFRASTRUCTURE ONLY.

Written separately from the oracle solver's own check (numpy, not C) so that a
mistake in one does not hide in the other.  Follows the stopping criteria of
Section 4.1 on the ORIGINAL problem of eq. (1):

    err_p = ||Pi_D(b - A x)|| / (1 + ||b||),   D = R^{m1} x R^{m2}_+
    err_d = ||c - A^T y - z|| / (1 + ||c||)
    pobj  = <c, x>,   dobj = <b, y> - delta_C^*(-z)
    gap   = |dobj - pobj| / (1 + |pobj| + |dobj|)

with delta_C^*(-z) = sup_{l <= x <= u} <-z, x> = -sum_{z_j>0} z_j l_j - sum_{z_j<0} z_j u_j
(a zero z_j contributes nothing even where its bound is infinite).
"""
from __future__ import annotations

import numpy as np


def support_term(z, l, u):
    """<b,y> - delta_C^*(-z) minus <b,y>: the bound part of the dual objective."""
    z = np.asarray(z, float)
    pos = z > 0
    neg = z < 0
    return float(np.sum(z[pos] * np.asarray(l)[pos]) + np.sum(z[neg] * np.asarray(u)[neg]))


def kkt(lp, x, y, z):
    A = lp.A
    b = lp.b
    r = b - A @ x
    r[lp.m1:] = np.maximum(r[lp.m1:], 0.0)
    err_p = float(np.linalg.norm(r) / (1.0 + np.linalg.norm(b)))
    err_d = float(np.linalg.norm(lp.c - A.T @ y - z) / (1.0 + np.linalg.norm(lp.c)))
    pobj = float(lp.c @ x)
    dobj = float(b @ y) + support_term(z, lp.l, lp.u)
    gap = abs(dobj - pobj) / (1.0 + abs(pobj) + abs(dobj))
    return dict(err_p=err_p, err_d=err_d, err_gap=gap, pobj=pobj, dobj=dobj,
                kkt=max(err_p, err_d, gap))


def in_C(x, l, u):
    return bool(np.all(x >= l) and np.all(x <= u))


def in_D(y, m1):
    return bool(np.all(np.asarray(y)[m1:] >= 0.0))
