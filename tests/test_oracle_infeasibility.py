"""Pins of the oracle's infeasibility detection (LP) against closed forms, a
library LP solver's classification and the defining conditions of Farkas
certificates on constructions whose infeasibility is known by hand."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg as O
from synth import instance_seed, lp_instance

INF = np.inf


def _p(A, c, lc, uc, l, u):
    return O.Problem(sp.csr_matrix(np.asarray(A, dtype=np.float64)), np.asarray(c, float),
                     np.asarray(lc, float), np.asarray(uc, float), np.asarray(l, float),
                     np.asarray(u, float))


def test_two_contradicting_equalities_separate_by_a_hyperplane():
    # x1 + x2 = 1 and x1 + x2 = 2 on the box [0, 10]^2.  y certifies infeasibility
    # iff the hyperplane it defines separates: min over the row values s = (1, 2)
    # of y^T s exceeds max over the box of y^T A x, i.e.
    #     y1 + 2 y2 > 20 max(y1 + y2, 0).
    p = _p([[1, 1], [1, 1]], [1, 1], [1, 2], [1, 2], [0, 0], [10, 10])
    r = O.solve_lp(p)
    assert r.status == "primal_infeasible"
    y = r.certificate / np.linalg.norm(r.certificate)
    assert y[0] + 2 * y[1] > 20 * max(y[0] + y[1], 0.0) + 1e-3


def test_inequality_above_the_box_is_primal_infeasible():
    # x1 + x2 >= 3 with 0 <= x <= 1: a certificate is any y1 > 0 (the row's
    # multiplier), since 3 y1 - (u1 + u2) y1 = y1 > 0 for the free reduced costs.
    p = _p([[1, 1]], [1, -1], [3], [INF], [0, 0], [1, 1])
    r = O.solve_lp(p)
    assert r.status == "primal_infeasible"
    assert r.certificate[0] > 0


def test_unbounded_ray_along_the_diagonal():
    # min -x1 s.t. x1 - x2 = 0, x >= 0: the recession directions with A dx = 0 and
    # dx >= 0 are t (1, 1), and c^T dx = -t < 0.
    p = _p([[1, -1]], [-1, 0], [0], [0], [0, 0], [INF, INF])
    r = O.solve_lp(p)
    assert r.status == "dual_infeasible"
    d = r.certificate / np.linalg.norm(r.certificate)
    np.testing.assert_allclose(d, np.array([1.0, 1.0]) / np.sqrt(2), atol=1e-6)


def test_unbounded_with_an_inequality_row():
    # min -x1 - x2 s.t. x1 - x2 >= -1, x >= 0: rays need dx >= 0, dx1 - dx2 >= 0,
    # and -dx1 - dx2 < 0.
    p = _p([[1, -1]], [-1, -1], [-1], [INF], [0, 0], [INF, INF])
    r = O.solve_lp(p)
    assert r.status == "dual_infeasible"
    d = r.certificate / np.max(np.abs(r.certificate))
    assert d.min() >= -1e-7 and d[0] - d[1] >= -1e-7 and d.sum() > 0


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_random_lp_with_a_contradicting_copy_row(seed):
    """A feasible random LP plus a copy of its equality row 0 shifted up by one:
    infeasible by construction; HiGHS classifies it the same way; the returned
    dual ray meets the Farkas conditions (A^T y in the reduced-cost cone up to
    1e-8 of its positive objective)."""
    from scipy.optimize import linprog
    d = lp_instance(30, 60, seed=instance_seed(seed), density=0.2)
    p0 = O.problem_from_arrays(d)
    A = sp.vstack([p0.A, p0.A[0]]).tocsr()
    p = O.Problem(A, p0.c, np.append(p0.lc, p0.uc[0] + 1.0), np.append(p0.uc, INF), p0.l, p0.u)
    r = O.solve_lp(p)
    assert r.status == "primal_infeasible"
    # the library's classification of the same LP: status 2 = infeasible
    Ad = A.toarray()
    eq = np.isfinite(p.lc) & np.isfinite(p.uc) & (p.lc == p.uc)
    ge = ~eq & np.isfinite(p.lc)
    res = linprog(p.c, A_ub=-Ad[ge], b_ub=-p.lc[ge], A_eq=Ad[eq], b_eq=p.lc[eq],
                  bounds=list(zip(p.l, p.u)), method="highs")
    assert res.status == 2
    # Farkas conditions of the certificate, checked directly
    y = r.certificate
    assert np.all(y[~np.isfinite(p.uc)] >= 0) and np.all(y[~np.isfinite(p.lc)] <= 0)
    lam = -(A.T @ y)                 # every column has finite l and u here: lam is free
    obj = (np.where(np.isfinite(p.lc), p.lc, 0) @ np.maximum(y, 0)
           - np.where(np.isfinite(p.uc), p.uc, 0) @ np.maximum(-y, 0)
           + p.l @ np.maximum(lam, 0) - p.u @ np.maximum(-lam, 0))
    assert obj > 0
    # weak duality: a feasible x would give 0 <= y^T (A x) - ... contradiction; the
    # certificate's objective must exceed what any point of the box can reach
    assert obj > 1e-6 * np.linalg.norm(y)


def test_feasible_instances_are_never_reported_infeasible():
    for i in range(4):
        d = lp_instance(20, 40, seed=instance_seed(100 + i), density=0.3,
                        variant="nondegenerate")
        r = O.solve_lp(O.problem_from_arrays(d), O.Options(eps_abs=1e-8, eps_rel=1e-8))
        assert r.status == "optimal"
        assert r.kkt["primal_obj"] == pytest.approx(d["opt_value"], rel=1e-6, abs=1e-6)
