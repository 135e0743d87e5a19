"""Oracle for the differentiation layer: LP optimal-value gradients and the
implicit-function adjoint of a strictly convex QP's solution.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper differentiates QPs by unrolling the iteration and LPs through
surrogate losses (Sec. 3.4); the layer built here differentiates the optimum
itself, which the paper does not state, so these are definitions written out:

* LP value v(c, lc, uc, l, u) = min c^T x: by the envelope theorem its gradient
  at a primal-dual optimum (x*, y*) with reduced costs lam* = c - A^T y* is
      dv/dc = x*,  dv/dlc = y*^+,  dv/duc = -y*^-,  dv/dl = lam*^+,  dv/du = -lam*^-.
* QP solution x*(c, b, D) for Q = diag(D) + F F^T (or a general sparse Q, D
  then standing for Q's diagonal), equality rows A x = b and box bounds.  On the free set F (variables strictly inside their bounds, plus
  bound variables whose multiplier is at most delta' in magnitude) and the
  active rows R (equalities and inequality rows with y_i != 0), x* solves
      Q_FF x_F - A_RF^T y_R = -c_F - Q_FB x_B,   A_RF x_F = b_R - A_RB x_B.
  For a loss L with g = dL/dx*, the adjoint system
      [[Q_FF, A_RF^T], [A_RF, 0]] [w; v] = [g_F; 0]
  gives dL/dc_F = -w, dL/db_R = v, dL/dD_j = -w_j x*_j (j in F), and zero for
  the other entries.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .pdhg import Problem


def lp_value_gradient(p: Problem, x, y):
    """Gradients of the LP optimal value at the optimum (x, y)."""
    lam = p.c - p.A.T @ y
    return dict(c=np.asarray(x, dtype=np.float64).copy(), lc=np.maximum(y, 0.0),
                uc=-np.maximum(-y, 0.0), l=np.maximum(lam, 0.0), u=-np.maximum(-lam, 0.0))


def active_sets(p: Problem, x, y, tol_x=1e-9, tol_lam=1e-9):
    """Free variables and active rows at (x, y), thresholds as in the module
    docstring: |x - bound| > tol_x (1 + |bound|) is free; a variable at a bound
    whose multiplier is at most tol_lam (1 + ||c||_inf) is free too."""
    lam = p.qx(x) + p.c - p.A.T @ y
    near_l = np.isfinite(p.l) & (x - p.l <= tol_x * (1 + np.abs(p.l)))
    near_u = np.isfinite(p.u) & (p.u - x <= tol_x * (1 + np.abs(p.u)))
    weak = np.abs(lam) <= tol_lam * (1 + np.max(np.abs(p.c), initial=0.0))
    free = ~(near_l | near_u) | weak
    eq = np.isfinite(p.lc) & np.isfinite(p.uc) & (p.lc == p.uc)
    rows = eq | (y != 0.0)
    return free, rows


def qp_adjoint(p: Problem, x, y, g, free=None, rows=None):
    """(dL/dc, dL/db, dL/dD) for Q = diag(D) + F F^T via a direct sparse solve
    of the adjoint saddle system."""
    if free is None or rows is None:
        free, rows = active_sets(p, x, y)
    Fi = np.flatnonzero(free)
    Ri = np.flatnonzero(rows)
    if hasattr(p.Q, "D"):
        Ff = p.Q.F[Fi]
        QFF = sp.diags(p.Q.D[Fi]) + Ff @ Ff.T
    else:  # a general sparse Q; dD is then the gradient of Q's diagonal
        QFF = p.Q.Q[Fi][:, Fi]
    ARF = p.A[Ri][:, Fi]
    K = sp.bmat([[QFF, ARF.T], [ARF, None]], format="csc")
    rhs = np.concatenate([g[Fi], np.zeros(len(Ri))])
    sol = spla.spsolve(K, rhs)
    w = sol[:len(Fi)]
    v = sol[len(Fi):]
    dc = np.zeros(p.n)
    dc[Fi] = -w
    db = np.zeros(p.m)
    db[Ri] = v
    dD = np.zeros(p.n)
    dD[Fi] = -w * x[Fi]
    return dc, db, dD
