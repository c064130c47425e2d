"""Feasibility of a plan's constraint set, by linear programming.

TEST INFRASTRUCTURE ONLY: tests/ use it to decide whether the half-spaces of
a plan (Fig. 2's dose and cDL rows and the LETd rows (L - Lambda D) w <= 0,
with w >= 0) have a common point, which tells whether a feasibility-seeking
run that still violates rows is slow or faces an empty set.  Nothing in the
CUDA library imports it.

The LP (a library primitive, scipy's HiGHS) minimises the total violation:
    minimise sum_r s_r  over w >= 0, s >= 0
    subject to  a_r . w - s_r <= b_r   (upper rows)
               -a_r . w - s_r <= -b_r  (lower rows)
Its optimum is 0 exactly when the set is non-empty; the returned w is then
a feasible point up to the solver's tolerance.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog

from .fredopt_oracle import Rows, violations


def min_total_violation(R: Rows, method: str = "highs-ipm"):
    """(smallest achievable sum of row violations, a minimising w >= 0)."""
    m, n = R.A.shape
    if m == 0:
        return 0.0, np.zeros(n)
    sign = np.where(R.upper, 1.0, -1.0)
    A = sp.diags(sign) @ sp.csr_matrix(R.A)
    A_ub = sp.hstack([A, -sp.eye(m)]).tocsr()
    c = np.concatenate([np.zeros(n), np.ones(m)])
    res = linprog(c, A_ub=A_ub, b_ub=sign * R.b, bounds=(0, None), method=method)
    if res.status != 0:
        raise RuntimeError(f"LP failed: {res.message}")
    return float(res.fun), res.x[:n]


def is_feasible(R: Rows, tol: float = 1e-7):
    """(True if some w >= 0 meets every row to within `tol`, that w, its
    largest row violation)."""
    f, w = min_total_violation(R)
    v = float(violations(R, w).max()) if R.A.shape[0] else 0.0
    return v <= tol, w, v
