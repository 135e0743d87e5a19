"""Pins of the differentiation oracle: central finite differences (h = 1e-6) of
the optimal value (LP, solved by HiGHS) and of the QP loss (solved by the
oracle to 1e-11), on small non-degenerate instances."""
import numpy as np
import pytest
from scipy.optimize import linprog

from oracle import adjoint as AD
from oracle import pdhg as O
from synth import instance_seed, lp_instance, qp_instance


def _lp_value(p):
    eq = np.isfinite(p.uc) & (p.lc == p.uc)
    res = linprog(p.c, A_ub=-p.A[~eq], b_ub=-p.lc[~eq], A_eq=p.A[eq], b_eq=p.lc[eq],
                  bounds=list(zip(p.l, p.u)), method="highs")
    return res.fun if res.status == 0 else None


def test_lp_value_gradient_matches_finite_differences():
    # a non-degenerate vertex: 10 equality rows + 6 tight inequality rows + 24
    # variables at a bound = n = 40 active constraints, strictly complementary,
    # so both the primal and the dual optimum are unique
    d = lp_instance(20, 40, seed=instance_seed(404), density=0.3, variant="nondegenerate",
                    tight_frac=0.6)
    p = O.problem_from_arrays(d)
    r = O.solve_lp(p, O.Options(eps_abs=1e-11, eps_rel=1e-11, iteration_limit=10**6))
    assert r.status == "optimal"
    gr = AD.lp_value_gradient(p, r.x, r.y)
    h = 1e-6
    rng = np.random.default_rng(0)
    for j in rng.choice(p.n, 8, replace=False):
        cp, cm = p.c.copy(), p.c.copy()
        cp[j] += h
        cm[j] -= h
        fd = (_lp_value(O.Problem(p.A, cp, p.lc, p.uc, p.l, p.u))
              - _lp_value(O.Problem(p.A, cm, p.lc, p.uc, p.l, p.u))) / (2 * h)
        assert fd == pytest.approx(gr["c"][j], abs=1e-5)
    tested = 0
    for i in range(p.m):
        lp_, lm_, up_, um_ = p.lc.copy(), p.lc.copy(), p.uc.copy(), p.uc.copy()
        lp_[i] += h
        up_[i] += h
        lm_[i] -= h
        um_[i] -= h
        vp = _lp_value(O.Problem(p.A, p.c, lp_, up_, p.l, p.u))
        vm = _lp_value(O.Problem(p.A, p.c, lm_, um_, p.l, p.u))
        if vp is None or vm is None:  # a row whose moves the fixed bounds cannot absorb
            continue
        assert (vp - vm) / (2 * h) == pytest.approx(gr["lc"][i] + gr["uc"][i], abs=1e-5)
        tested += 1
    assert tested >= 10
    # envelope theorem: at an upper bound the value falls with u at rate lam^-
    at_u = np.flatnonzero(np.abs(r.x - p.u) < 1e-9)
    j = at_u[0]
    up, um = p.u.copy(), p.u.copy()
    up[j] += h
    um[j] -= h
    fd = (_lp_value(O.Problem(p.A, p.c, p.lc, p.uc, p.l, up))
          - _lp_value(O.Problem(p.A, p.c, p.lc, p.uc, p.l, um))) / (2 * h)
    assert fd == pytest.approx(gr["u"][j], abs=1e-5)


def _qp_loss(p, xt, opts):
    r = O.solve_qp(p, opts)
    assert r.status == "optimal"
    return 0.5 * float(np.sum((r.x - xt) ** 2))


def test_qp_adjoint_matches_finite_differences():
    d = qp_instance(50, 25, seed=instance_seed(202), a_density=0.04, f_cols=32, f_density=0.04,
                    min_row=2)
    p = O.problem_from_arrays(d)
    xt = d["x_target"]
    opts = O.Options(eps_abs=1e-11, eps_rel=1e-11, iteration_limit=10**6)
    r = O.solve_qp(p, opts)
    free, rows = AD.active_sets(p, r.x, r.y, 1e-7, 1e-7)
    # non-degenerate: every bound variable has a clearly nonzero multiplier
    lam = p.qx(r.x) + p.c - p.A.T @ r.y
    assert np.all(np.abs(lam[~free]) > 1e-6)
    dc, db, dD = AD.qp_adjoint(p, r.x, r.y, r.x - xt, free, rows)
    h = 1e-6
    rng = np.random.default_rng(1)

    def fd(make):
        return (_qp_loss(make(+h), xt, opts) - _qp_loss(make(-h), xt, opts)) / (2 * h)

    for j in rng.choice(p.n, 6, replace=False):
        def mk(s, j=j):
            c = p.c.copy()
            c[j] += s
            return O.Problem(p.A, c, p.lc, p.uc, p.l, p.u, p.Q)
        assert fd(mk) == pytest.approx(dc[j], rel=1e-4, abs=1e-6)
    for i in rng.choice(p.m, 4, replace=False):
        def mk(s, i=i):
            lo, hi = p.lc.copy(), p.uc.copy()
            lo[i] += s
            hi[i] += s
            return O.Problem(p.A, p.c, lo, hi, p.l, p.u, p.Q)
        assert fd(mk) == pytest.approx(db[i], rel=1e-4, abs=1e-6)
    for j in rng.choice(np.flatnonzero(free), 4, replace=False):
        def mk(s, j=j):
            D = p.Q.D.copy()
            D[j] += s
            return O.Problem(p.A, p.c, p.lc, p.uc, p.l, p.u, O.DiagLowRankQ(D, p.Q.F))
        assert fd(mk) == pytest.approx(dD[j], rel=1e-4, abs=1e-6)


def test_sparse_q_adjoint_matches_finite_differences():
    """A general sparse Q: dL/dc and the gradient of Q's diagonal against central
    differences of converged oracle solves."""
    import scipy.sparse as sp
    from synth import qp_sparse_q_instance
    d = qp_sparse_q_instance(50, 25, seed=instance_seed(204), a_density=0.04, b_density=0.04,
                             min_row=2)
    p = O.problem_from_arrays(d)
    xt = d["x_target"]
    opts = O.Options(eps_abs=1e-11, eps_rel=1e-11, iteration_limit=10**6)
    r = O.solve_qp(p, opts)
    free, rows = AD.active_sets(p, r.x, r.y, 1e-7, 1e-7)
    lam = p.qx(r.x) + p.c - p.A.T @ r.y
    assert np.all(np.abs(lam[~free]) > 1e-6)
    dc, db, dD = AD.qp_adjoint(p, r.x, r.y, r.x - xt, free, rows)
    h = 1e-6
    rng = np.random.default_rng(3)

    def fd(make):
        return (_qp_loss(make(+h), xt, opts) - _qp_loss(make(-h), xt, opts)) / (2 * h)

    for j in rng.choice(p.n, 4, replace=False):
        def mk(s, j=j):
            c = p.c.copy()
            c[j] += s
            return O.Problem(p.A, c, p.lc, p.uc, p.l, p.u, p.Q)
        assert fd(mk) == pytest.approx(dc[j], rel=1e-4, abs=1e-6)
    for j in rng.choice(np.flatnonzero(free), 3, replace=False):
        def mk(s, j=j):
            e = np.zeros(p.n)
            e[j] = s
            return O.Problem(p.A, p.c, p.lc, p.uc, p.l, p.u,
                             O.SparseQ(p.Q.Q + sp.diags(e)))
        assert fd(mk) == pytest.approx(dD[j], rel=1e-4, abs=1e-6)
