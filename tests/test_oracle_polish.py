"""Pins of the oracle's feasibility polishing (Sec. 3.3): the primal phase
lands on the constraint set from an infeasible start, leaves an exact optimum
(from HiGHS) where it is, and the dual phase brings the dual residual of a
point with one-sided bounds to the polishing tolerance."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

from oracle import pdhg as O
from synth import instance_seed, lp_instance

INF = np.inf


def test_primal_phase_reaches_the_line_inside_the_box():
    # x1 + x2 = 1 on [0, 1]^2 from the infeasible (0.6, 0.6)
    p = O.Problem(sp.csr_matrix(np.array([[1.0, 1.0]])), np.array([1.0, 2.0]), np.array([1.0]),
                  np.array([1.0]), np.zeros(2), np.ones(2))
    xp, yp, rp, rd = O.polish_lp(p, np.array([0.6, 0.6]), np.zeros(1))
    assert abs(xp.sum() - 1.0) <= 1e-6 * 2
    assert np.all(xp >= -1e-12) and np.all(xp <= 1 + 1e-12)


def test_an_exact_optimum_is_left_in_place():
    d = lp_instance(30, 60, seed=instance_seed(404), density=0.2, variant="nondegenerate")
    p = O.problem_from_arrays(d)
    A = p.A.toarray()
    eq = p.lc == p.uc
    res = linprog(p.c, A_ub=-A[~eq], b_ub=-p.lc[~eq], A_eq=A[eq], b_eq=p.lc[eq],
                  bounds=list(zip(p.l, p.u)), method="highs")
    assert res.status == 0
    x = np.clip(res.x, p.l, p.u)
    xp, _, rp, _ = O.polish_lp(p, x, np.zeros(p.m))
    assert rp.iterations == 64                 # done at the first check
    np.testing.assert_allclose(xp, x, atol=1e-8)


def test_dual_phase_meets_the_tolerance_with_one_sided_bounds():
    # the literal construction (c = A_eq^T y0, x0 inside the box) stays bounded
    # without upper bounds: c^T x = y0^T b_eq on the feasible set
    d = lp_instance(40, 80, seed=instance_seed(405), density=0.1)
    p0 = O.problem_from_arrays(d)
    # lower bounds only: Lambda_j = R+, so c - A^T y must be >= 0
    p = O.Problem(p0.A, p0.c, p0.lc, p0.uc, p0.l, np.full(p0.n, INF))
    r = O.solve_lp(p, O.Options(eps_abs=1e-3, eps_rel=1e-3, iteration_limit=50000))
    assert r.status == "optimal"
    k0 = O.kkt(p, r.x, r.y)
    xp, yp, rp, rd = O.polish_lp(p, r.x, r.y)
    k1 = O.kkt(p, xp, yp)
    assert k1["dual_res"] <= 1e-6 * (1 + k1["c_norm"])
    assert k1["primal_res"] <= 1e-6 * (1 + k1["b_norm"])
    assert k1["dual_res"] <= k0["dual_res"] + 1e-12
