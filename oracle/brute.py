"""Brute-force checkers that pin the oracle's converged answers.

TEST INFRASTRUCTURE ONLY.  These do not follow the paper's method at all: they
solve tiny instances of problem (1) exactly by enumeration, so that a mistake in
the PDHG oracle (a dropped term, a wrong sign, a transposed operand) shows up as
a different optimum.

* ``lp_vertex_enumeration``: a bounded feasible LP attains its optimum at a
  vertex, i.e. at a point where n linearly independent constraints are active.
  Enumerate every choice of active inequalities that completes the equalities to
  n constraints, solve, keep the feasible points, return the best.
* ``qp_active_set_enumeration``: for a strictly convex QP with box bounds and
  equality rows, enumerate the 3^n patterns (at lower, at upper, free), solve
  the equality-constrained KKT system of each, and keep the unique pattern whose
  solution is primal feasible with correctly signed bound multipliers.
"""
from __future__ import annotations

import itertools

import numpy as np


def _constraint_system(A, lc, uc, l, u):
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    E, e, G, h = [], [], [], []
    for i in range(m):
        if np.isfinite(lc[i]) and np.isfinite(uc[i]) and lc[i] == uc[i]:
            E.append(A[i]); e.append(lc[i])
            continue
        if np.isfinite(uc[i]):
            G.append(A[i]); h.append(uc[i])
        if np.isfinite(lc[i]):
            G.append(-A[i]); h.append(-lc[i])
    I = np.eye(n)
    for j in range(n):
        if np.isfinite(u[j]):
            G.append(I[j]); h.append(u[j])
        if np.isfinite(l[j]):
            G.append(-I[j]); h.append(-l[j])
    E = np.array(E).reshape(-1, n); e = np.array(e)
    G = np.array(G).reshape(-1, n); h = np.array(h)
    return E, e, G, h


def lp_vertex_enumeration(A, c, lc, uc, l, u, tol=1e-9, chunk=20000):
    """Exact optimum of a bounded, feasible LP by enumerating vertices.
    Returns (best value, best x)."""
    E, e, G, h = _constraint_system(A, lc, uc, l, u)
    n = len(c)
    k = n - E.shape[0]
    if k < 0:
        raise ValueError("more equalities than variables")
    best_val, best_x = np.inf, None
    combos = itertools.combinations(range(G.shape[0]), k)
    while True:
        block = list(itertools.islice(combos, chunk))
        if not block:
            break
        idx = np.array(block, dtype=np.int64).reshape(len(block), k)
        M = np.concatenate([np.broadcast_to(E, (len(block),) + E.shape), G[idx]], axis=1)
        rhs = np.concatenate([np.broadcast_to(e, (len(block), E.shape[0])), h[idx]], axis=1)
        sv = np.linalg.svd(M, compute_uv=False)
        ok = sv[:, -1] > 1e-9 * np.maximum(sv[:, 0], 1.0)
        if not ok.any():
            continue
        X = np.linalg.solve(M[ok], rhs[ok][..., None])[..., 0]
        feas = np.all(X @ G.T <= h + tol * (1 + np.abs(h)), axis=1)
        if E.shape[0]:
            feas &= np.all(np.abs(X @ E.T - e) <= tol * (1 + np.abs(e)), axis=1)
        if not feas.any():
            continue
        vals = X[feas] @ c
        j = int(np.argmin(vals))
        if vals[j] < best_val:
            best_val, best_x = float(vals[j]), X[feas][j]
    return best_val, best_x


def qp_active_set_enumeration(Q, c, A_eq, b_eq, l, u, tol=1e-9):
    """Exact solution of  min 1/2 x^T Q x + c^T x  s.t.  A_eq x = b_eq,
    l <= x <= u  (Q positive definite, finite box).  Returns (x, y, value) with
    y the multipliers of A_eq x = b_eq in the convention Q x + c - A^T y = lam,
    lam >= 0 at a lower bound and <= 0 at an upper bound."""
    Q = np.asarray(Q, dtype=np.float64)
    A = np.asarray(A_eq, dtype=np.float64).reshape(-1, len(c))
    n = len(c)
    m = A.shape[0]
    found = []
    for pattern in itertools.product((0, 1, 2), repeat=n):  # 0 free, 1 at l, 2 at u
        pat = np.array(pattern)
        F = np.flatnonzero(pat == 0)
        B = np.flatnonzero(pat != 0)
        xB = np.where(pat[B] == 1, l[B], u[B])
        nf = len(F)
        K = np.zeros((nf + m, nf + m))
        K[:nf, :nf] = Q[np.ix_(F, F)]
        K[:nf, nf:] = -A[:, F].T
        K[nf:, :nf] = A[:, F]
        rhs = np.concatenate([-c[F] - Q[np.ix_(F, B)] @ xB, b_eq - A[:, B] @ xB])
        try:
            sol = np.linalg.solve(K, rhs)
        except np.linalg.LinAlgError:
            continue
        if not np.all(np.isfinite(sol)):
            continue
        x = np.empty(n)
        x[F] = sol[:nf]
        x[B] = xB
        y = sol[nf:]
        if np.any(x < l - tol) or np.any(x > u + tol):
            continue
        if np.max(np.abs(A @ x - b_eq), initial=0.0) > 1e-7:
            continue
        lam = Q @ x + c - A.T @ y
        at_l = B[pat[B] == 1]
        at_u = B[pat[B] == 2]
        if np.any(lam[at_l] < -tol) or np.any(lam[at_u] > tol):
            continue
        found.append((x, y, float(0.5 * x @ Q @ x + c @ x)))
    if not found:
        raise ValueError("no KKT point found (infeasible?)")
    return min(found, key=lambda t: t[2])
