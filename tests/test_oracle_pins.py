"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
hand-derived worked examples (tests/golden), algebraic identities of eqs. (3)-(6),
projection invariants of the dual cone Y (Sec. 2), brute-force vertex and
active-set enumeration, a library LP solver (HiGHS via scipy), closed forms of
the constructed instances, and SVD norms."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import brute
from oracle import pdhg as O
from synth import instance_seed, lp_instance, qp_instance, random_state


def _f(v):
    return np.array([float(t) for t in v], dtype=np.float64)


@pytest.fixture(scope="module")
def worked(golden_dir):
    with open(os.path.join(golden_dir, "worked_2x3.json")) as fh:
        g = json.load(fh)
    pr = g["problem"]
    p = O.Problem(sp.csr_matrix(np.array(pr["A"], dtype=float)), _f(pr["c"]), _f(pr["lc"]),
                  _f(pr["uc"]), _f(pr["l"]), _f(pr["u"]))
    return g, p


# ---------------------------------------------------------------- worked example

def test_pdhg_step_worked_example(worked):
    g, p = worked
    w = g["pdhg_lp"]
    x_hat, y_hat, xbar = O.pdhg_step_lp(p, _f(w["x"]), _f(w["y"]), w["tau"], w["sigma"])
    np.testing.assert_allclose(x_hat, w["x_hat"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(xbar, w["xbar"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(y_hat, w["y_hat"], rtol=0, atol=1e-15)


def test_halpern_worked_example(worked):
    g, p = worked
    w = g["pdhg_lp"]
    x_hat, y_hat = _f(w["x_hat"]), _f(w["y_hat"])
    h = g["halpern_k1_gamma1"]
    xn = O.halpern(x_hat, _f(w["x"]), _f(h["x_anchor"]), h["k"], h["gamma"])
    yn = O.halpern(y_hat, _f(w["y"]), _f(h["y_anchor"]), h["k"], h["gamma"])
    np.testing.assert_allclose(xn, h["x_next"], rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(yn, h["y_next"], rtol=1e-15, atol=1e-15)
    h2 = g["halpern_k0_gamma_half"]
    xn2 = O.halpern(x_hat, _f(w["x"]), _f(h2["x_anchor"]), h2["k"], h2["gamma"])
    np.testing.assert_allclose(xn2, h2["x_next"], rtol=1e-15, atol=1e-15)


def test_apdhg_worked_example(worked):
    g, p = worked
    w = g["apdhg_qp_k1"]
    pq = O.Problem(p.A, p.c, p.lc, p.uc, p.l, p.u, O.SparseQ(sp.diags(_f(w["Q_diag"]))))
    xn, yn, xa, ya, xref = O.apdhg_step_qp(pq, _f(w["x"]), _f(w["y"]), _f(w["xavg"]),
                                           _f(w["yavg"]), w["k"], w["tau"], w["sigma"])
    for got, key in ((xn, "x_next"), (yn, "y_next"), (xa, "xavg_next"), (ya, "yavg_next"),
                     (xref, "xref")):
        np.testing.assert_allclose(got, w[key], rtol=1e-14, atol=1e-15)


def test_kkt_worked_example(worked):
    g, p = worked
    k = g["kkt"]
    pk = O.Problem(p.A, p.c, p.lc, p.uc, _f(k["l"]), _f(k["u"]))
    info = O.kkt(pk, _f(k["x"]), _f(k["y"]))
    for key, val in k["lp"].items():
        assert info[key] == pytest.approx(val, rel=1e-14, abs=1e-15), key
    pq = O.Problem(p.A, p.c, p.lc, p.uc, _f(k["l"]), _f(k["u"]),
                   O.SparseQ(sp.diags(_f(k["qp_Q_diag"]))))
    info = O.kkt(pq, _f(k["x"]), _f(k["y"]))
    for key, val in k["qp"].items():
        assert info[key] == pytest.approx(val, rel=1e-14, abs=1e-15), key


# ---------------------------------------------------------------- identities

def _mixed_bounds_problem(seed, m=30, n=50):
    rng = np.random.default_rng(seed)
    A = sp.random(m, n, density=0.2, random_state=rng, data_rvs=rng.standard_normal, format="csr")
    c = rng.standard_normal(n)
    kinds_r = rng.integers(0, 4, size=m)  # 0 eq, 1 only lower, 2 only upper, 3 free
    b = rng.standard_normal(m)
    lc = np.where(kinds_r == 0, b, np.where(kinds_r == 1, b - 1, -np.inf))
    uc = np.where(kinds_r == 0, b, np.where(kinds_r == 2, b + 1, np.inf))
    lc[kinds_r == 3] = -np.inf
    kinds_c = rng.integers(0, 4, size=n)  # 0 box, 1 lower, 2 upper, 3 free
    l = np.where((kinds_c == 0) | (kinds_c == 1), -1.0, -np.inf)
    u = np.where((kinds_c == 0) | (kinds_c == 2), 1.0, np.inf)
    return O.Problem(A, c, lc, uc, l, u)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_projections_land_in_X_and_Y(seed):
    p = _mixed_bounds_problem(seed)
    st = random_state(p.n, p.m, seed=seed)
    x = st["x"] * 3
    y = st["y"] * 3
    x_hat, y_hat, _ = O.pdhg_step_lp(p, x, y, 0.3, 0.7)
    assert np.all(x_hat >= p.l) and np.all(x_hat <= p.u)
    fl, fu = np.isfinite(p.lc), np.isfinite(p.uc)
    # Y_i: {0} if both infinite, R- if only uc finite, R+ if only lc finite.
    # Eq. (3) as written, y - sigma s - sigma proj(y/sigma - s), cancels to the
    # boundary of Y only up to rounding, hence the slack.
    slack = 1e-12 * (np.abs(y) + 0.7 * np.abs(p.A @ (2 * x_hat - x)) + 1.0)
    assert np.all(np.abs(y_hat[~fl & ~fu]) <= slack[~fl & ~fu])
    assert np.all(y_hat[~fl & fu] <= slack[~fl & fu])
    assert np.all(y_hat[fl & ~fu] >= -slack[fl & ~fu])
    # the primal projection is idempotent
    np.testing.assert_array_equal(O.clamp(x_hat, p.l, p.u), x_hat)


def test_halpern_k0_gamma1_returns_pdhg_point():
    rng = np.random.default_rng(5)
    z, zh = rng.standard_normal(7), rng.standard_normal(7)
    np.testing.assert_allclose(O.halpern(zh, z, z, 0, 1.0), zh, rtol=0, atol=1e-15)


def test_apdhg_first_step_is_plain_pdhg_and_average_resets():
    d = qp_instance(40, 10, seed=instance_seed(11), a_density=0.2, f_density=0.2, min_row=2)
    p = O.problem_from_arrays(d)
    st = random_state(p.n, p.m, seed=3)
    xn, yn, xa, ya, _ = O.apdhg_step_qp(p, st["x"], st["y"], st["xbar"], st["ybar"], 0, 0.1, 0.2)
    # beta_0 = 1: x_md = x, so the primal step is eq. (5)
    x_ref = O.clamp(st["x"] - 0.1 * (p.Q.matvec(st["x"]) + p.c - p.A.T @ st["y"]), p.l, p.u)
    np.testing.assert_allclose(xn, x_ref, rtol=0, atol=1e-14)
    # theta_0 = 1: the averages restart at the new iterate
    np.testing.assert_array_equal(xa, xn)
    np.testing.assert_array_equal(ya, yn)


def test_fixed_point_iff_kkt():
    """At the constructed optimum (x0, y0) of a nondegenerate LP the PDHG map
    is stationary and the KKT error vanishes; a perturbed point is neither."""
    d = lp_instance(40, 80, seed=instance_seed(21), density=0.1, variant="nondegenerate")
    p = O.problem_from_arrays(d)
    x0, y0 = d["x0"], d["y0"]
    x_hat, y_hat, _ = O.pdhg_step_lp(p, x0, y0, 0.05, 0.05)
    np.testing.assert_allclose(x_hat, x0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(y_hat, y0, rtol=0, atol=1e-12)
    info = O.kkt(p, x0, y0)
    assert info["rel_kkt"] < 1e-13
    assert info["primal_obj"] == pytest.approx(d["opt_value"], rel=1e-13)
    xp = x0 + 0.01
    x_hat2, _, _ = O.pdhg_step_lp(p, xp, y0, 0.05, 0.05)
    assert np.max(np.abs(x_hat2 - xp)) > 1e-6
    assert O.kkt(p, xp, y0)["rel_kkt"] > 1e-5


def test_bound_vector_and_primal_weight():
    lc = np.array([1.0, -np.inf, -3.0, -np.inf, 2.0])
    uc = np.array([1.0, 4.0, np.inf, np.inf, -5.0])
    np.testing.assert_array_equal(O.bound_vector(lc, uc), [1.0, 4.0, -3.0, 0.0, -5.0])
    assert O.initial_primal_weight(np.array([3.0, 4.0]), np.array([0.0, 2.0])) == 2.5
    assert O.initial_primal_weight(np.zeros(2), np.array([0.0, 2.0])) == 1.0


# ---------------------------------------------------------------- scaling

def test_pock_chambolle_hand_example():
    A = sp.csr_matrix(np.array([[1.0, -3.0], [0.0, 4.0]]))
    Dr, Dc = O.scaling_factors(A, ruiz_iters=0, pock_chambolle=True)
    np.testing.assert_allclose(Dr, [1 / 2.0, 1 / 2.0])      # row sums 4, 4
    np.testing.assert_allclose(Dc, [1.0, 1 / math.sqrt(7)])  # column sums 1, 7


def test_ruiz_equilibrates():
    d = lp_instance(60, 90, seed=instance_seed(31), density=0.1)
    p = O.problem_from_arrays(d)
    p.A.data *= np.exp(3 * np.random.default_rng(0).standard_normal(p.A.nnz))
    Dr, Dc = O.scaling_factors(p.A, ruiz_iters=40, pock_chambolle=False)
    K = abs(sp.diags(Dr) @ p.A @ sp.diags(Dc)).tocsr()
    rmax = K.max(axis=1).toarray().ravel()
    cmax = K.max(axis=0).toarray().ravel()
    nz_r = np.diff(p.A.indptr) > 0
    nz_c = np.bincount(p.A.indices, minlength=p.n) > 0
    assert np.all(np.abs(rmax[nz_r] - 1) < 1e-3)
    assert np.all(np.abs(cmax[nz_c] - 1) < 1e-3)
    # empty rows/columns keep factor 1
    assert np.all(Dr[~nz_r] == 1.0) and np.all(Dc[~nz_c] == 1.0)


def test_scaling_preserves_the_optimum():
    d = lp_instance(30, 60, seed=instance_seed(41), density=0.15, variant="nondegenerate")
    p = O.problem_from_arrays(d)
    Dr, Dc = O.scaling_factors(p.A)
    ps = O.scale_problem(p, Dr, Dc)
    # the constructed optimum maps to an optimum of the scaled problem
    xs, ys = d["x0"] / Dc, d["y0"] / Dr
    assert O.kkt(ps, xs, ys)["rel_kkt"] < 1e-13
    assert float(ps.c @ xs) == pytest.approx(d["opt_value"], rel=1e-13)


# ---------------------------------------------------------------- norms

def test_splitmix64_reference_sequence():
    """The power iteration's start vector uses SplitMix64 (Steele, Lea and Flood,
    2014): seeded with 0, the generator's first outputs are the published
    E220A8397B1DCDAF, 6E789E6AA1B965F4, 06C45D188009454F (output k mixes the
    state k * 0x9E3779B97F4A7C15)."""
    golden = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [O._splitmix64((k * golden) & ((1 << 64) - 1)) for k in range(3)]
    assert got == want
    # the start vector: unit norm, entries of both signs in balance (2u - 1, u uniform)
    v = O.power_start(10000)
    assert np.linalg.norm(v) == pytest.approx(1.0, rel=1e-14)
    assert 0.48 < float(np.mean(v > 0)) < 0.52


def test_power_norm_matches_svd():
    d = lp_instance(80, 120, seed=instance_seed(51), density=0.1)
    A = O.problem_from_arrays(d).A
    s = np.linalg.norm(A.toarray(), 2)
    nu, _ = O.power_norm_A(A, max_iter=5000, tol=1e-14)
    assert nu == pytest.approx(s, rel=1e-8)
    nu_default, _ = O.power_norm_A(A)
    assert abs(nu_default - s) / s < 2e-2
    Q = O.DiagLowRankQ(np.linspace(0.1, 1, 120),
                       sp.random(120, 4, density=0.3, random_state=1, format="csr"))
    ev = np.linalg.eigvalsh(Q.dense())[-1]
    nq, _ = O.power_norm_Q(Q, 120, max_iter=5000, tol=1e-14)
    assert nq == pytest.approx(ev, rel=1e-8)


# ---------------------------------------------------------------- converged LP

@pytest.mark.parametrize("seed,m,n", [(61, 3, 6), (62, 4, 8), (63, 4, 8), (64, 5, 10)])
def test_lp_matches_vertex_enumeration(seed, m, n):
    variant = "nondegenerate" if seed % 2 else "literal"
    d = lp_instance(m, n, seed=instance_seed(seed), density=0.6, variant=variant, min_row=2)
    p = O.problem_from_arrays(d)
    r = O.solve_lp(p, O.Options(eps_abs=1e-10, eps_rel=1e-10, iteration_limit=500000))
    assert r.status == "optimal"
    best, _ = brute.lp_vertex_enumeration(p.A.toarray(), p.c, p.lc, p.uc, p.l, p.u)
    assert r.kkt["primal_obj"] == pytest.approx(best, rel=1e-7, abs=1e-7)
    assert best == pytest.approx(d["opt_value"], rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("variant", ["literal", "nondegenerate"])
def test_lp_200x400_matches_highs_and_closed_form(variant):
    from scipy.optimize import linprog
    d = lp_instance(200, 400, seed=instance_seed(1), density=0.02, variant=variant)
    p = O.problem_from_arrays(d)
    r = O.solve_lp(p, O.Options(eps_abs=1e-8, eps_rel=1e-8, iteration_limit=400000))
    assert r.status == "optimal" and r.kkt["rel_kkt"] <= 1e-8
    eq = np.isfinite(p.uc)
    ref = linprog(p.c, A_ub=-p.A[~eq], b_ub=-p.lc[~eq], A_eq=p.A[eq], b_eq=p.lc[eq],
                  bounds=list(zip(p.l, p.u)), method="highs")
    assert ref.status == 0
    assert r.kkt["primal_obj"] == pytest.approx(ref.fun, rel=1e-7)
    assert r.kkt["primal_obj"] == pytest.approx(d["opt_value"], rel=1e-7)
    # strong duality at the returned point
    assert r.kkt["gap"] <= 1e-8 * (1 + abs(r.kkt["primal_obj"]) + abs(r.kkt["dual_obj"]))


def test_lp_10x20_slice_closed_form_and_duality():
    d = lp_instance(10, 20, seed=instance_seed(71), density=0.3, variant="nondegenerate",
                    min_row=2)
    p = O.problem_from_arrays(d)
    r = O.solve_lp(p, O.Options(eps_abs=1e-9, eps_rel=1e-9, iteration_limit=500000))
    assert r.status == "optimal"
    assert r.kkt["primal_obj"] == pytest.approx(d["opt_value"], rel=1e-7)
    assert abs(r.kkt["primal_obj"] - r.kkt["dual_obj"]) < 1e-6


# ---------------------------------------------------------------- converged QP

@pytest.mark.parametrize("seed,n,m", [(81, 6, 2), (82, 8, 3)])
def test_qp_matches_active_set_enumeration(seed, n, m):
    d = qp_instance(n, m, seed=instance_seed(seed), a_density=0.6, f_cols=3, f_density=0.5,
                    min_row=2)
    p = O.problem_from_arrays(d)
    r = O.solve_qp(p, O.Options(eps_abs=1e-10, eps_rel=1e-10, iteration_limit=2000000))
    assert r.status == "optimal"
    x, y, val = brute.qp_active_set_enumeration(p.Q.dense(), p.c, p.A.toarray(), p.lc, p.l, p.u)
    np.testing.assert_allclose(r.x, x, rtol=0, atol=1e-6)
    assert r.kkt["primal_obj"] == pytest.approx(val, rel=1e-8, abs=1e-8)


def _sparse_psd_q(n, seed):
    """Q = B B^T + diag(U[0.1, 1]) with B n x n at 30% density: sparse, symmetric,
    positive definite, with off-diagonal entries of both signs."""
    rng = np.random.default_rng(seed)
    B = sp.random(n, n, density=0.3, random_state=rng, data_rvs=rng.standard_normal)
    return sp.csr_matrix(B @ B.T + sp.diags(rng.uniform(0.1, 1.0, n)))


@pytest.mark.parametrize("seed,n,m", [(83, 6, 2), (84, 8, 3)])
def test_sparse_q_qp_matches_active_set_enumeration(seed, n, m):
    """A general sparse Q (SparseQ): its diagonal joins the scaling, its norm the
    step sizes and its product the iteration and the KKT test."""
    d = qp_instance(n, m, seed=instance_seed(seed), a_density=0.6, f_cols=3, f_density=0.5,
                    min_row=2)
    p0 = O.problem_from_arrays(d)
    p = O.Problem(p0.A, p0.c, p0.lc, p0.uc, p0.l, p0.u, O.SparseQ(_sparse_psd_q(n, seed)))
    r = O.solve_qp(p, O.Options(eps_abs=1e-10, eps_rel=1e-10, iteration_limit=2000000))
    assert r.status == "optimal"
    x, y, val = brute.qp_active_set_enumeration(p.Q.dense(), p.c, p.A.toarray(), p.lc, p.l, p.u)
    np.testing.assert_allclose(r.x, x, rtol=0, atol=1e-6)
    assert r.kkt["primal_obj"] == pytest.approx(val, rel=1e-8, abs=1e-8)


def test_box_qp_diagonal_closed_form():
    rng = np.random.default_rng(9)
    n = 30
    D = rng.uniform(0.1, 1.0, n)
    c = 2 * rng.standard_normal(n)
    l, u = -np.ones(n), np.ones(n)
    p = O.Problem(sp.csr_matrix((0, n)), c, np.zeros(0), np.zeros(0), l, u,
                  O.DiagLowRankQ(D, sp.csr_matrix((n, 1))))
    r = O.solve_qp(p, O.Options(eps_abs=1e-11, eps_rel=1e-11, iteration_limit=200000))
    np.testing.assert_allclose(r.x, np.clip(-c / D, l, u), rtol=0, atol=1e-8)


# ---------------------------------------------------------------- the checkers themselves

@pytest.mark.parametrize("seed", [71, 72, 73])
def test_vertex_enumeration_agrees_with_highs(seed):
    """The brute-force LP checker against HiGHS on tiny LPs with equality, one- and
    two-sided rows and finite boxes (an independent solver pins the checker)."""
    from scipy.optimize import linprog
    rng = np.random.default_rng(seed)
    m, n = 3, 5
    A = rng.normal(size=(m, n))
    x0 = rng.uniform(0, 1, n)
    ax = A @ x0
    lc = np.array([ax[0], ax[1] - 0.5, -np.inf])
    uc = np.array([ax[0], np.inf, ax[2] + 0.5])
    l, u = np.zeros(n), np.full(n, 2.0)
    c = rng.normal(size=n)
    best, _ = brute.lp_vertex_enumeration(A, c, lc, uc, l, u)
    A_ub = np.vstack([-A[1:2], A[2:3]])
    b_ub = np.array([-lc[1], uc[2]])
    ref = linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=A[0:1], b_eq=lc[0:1],
                  bounds=list(zip(l, u)), method="highs")
    assert ref.status == 0
    assert best == pytest.approx(ref.fun, rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("seed", [91, 92])
def test_active_set_enumeration_agrees_with_slsqp(seed):
    """The brute-force QP checker against SciPy's SLSQP on tiny strictly convex QPs
    with an equality row and a box."""
    from scipy.optimize import minimize
    rng = np.random.default_rng(seed)
    n = 5
    B = rng.normal(size=(n, n))
    Q = B @ B.T + 0.5 * np.eye(n)
    c = 3.0 * rng.normal(size=n)
    A = rng.normal(size=(1, n))
    b = A @ rng.uniform(-0.5, 0.5, n)
    l, u = -np.ones(n), np.ones(n)
    x, _, val = brute.qp_active_set_enumeration(Q, c, A, b, l, u)
    f = lambda z: 0.5 * z @ Q @ z + c @ z  # noqa: E731
    r = minimize(f, np.zeros(n), jac=lambda z: Q @ z + c, method="SLSQP",
                 bounds=list(zip(l, u)),
                 constraints=[dict(type="eq", fun=lambda z: A @ z - b, jac=lambda z: A)],
                 options=dict(ftol=1e-14, maxiter=1000))
    assert r.success
    np.testing.assert_allclose(x, r.x, atol=1e-6)
    assert val == pytest.approx(f(r.x), rel=1e-9, abs=1e-9)


def test_restart_rule_and_primal_weight_update_by_hand():
    """The restart rule (sufficient 0.2, necessary 0.8 with no progress, artificial
    0.36 of all iterations) and the smoothed primal-weight update, on hand inputs."""
    o = O.Options()
    assert O._restart_decision(1.0, None, None, 1, 64, o)  # the first check always restarts
    assert O._restart_decision(0.19, 1.0, 0.5, 10, 1000, o)  # sufficient decay
    assert not O._restart_decision(0.21, 1.0, 0.5, 10, 1000, o)  # progress, not enough
    assert O._restart_decision(0.7, 1.0, 0.6, 10, 1000, o)  # necessary + no progress
    assert not O._restart_decision(0.7, 1.0, 0.8, 10, 1000, o)  # still progressing
    assert O._restart_decision(0.9, 1.0, 0.8, 360, 1000, o)  # artificial: k >= 0.36 t
    assert not O._restart_decision(0.9, 1.0, 0.8, 359, 1000, o)
    # omega <- exp(0.5 log(dy/dx) + 0.5 log omega): the geometric mean of dy/dx and omega
    assert O._update_weight(2.0, 1.0, 8.0, o) == pytest.approx(4.0, rel=1e-15)
    assert O._update_weight(2.0, 0.0, 8.0, o) == 2.0  # a zero move keeps omega


@pytest.mark.parametrize("kind", ["bernoulli", "zipf", "empty_rows_cols", "qp_diag"])
def test_pock_chambolle_bound_against_svd(kind):
    """After the Pock-Chambolle round (alpha = 1) the scaled matrix has
    ||A~||_2 <= 1 (Schur's test with weights sqrt(r_i), sqrt(c_j)); the batch path
    uses that bound in place of the power iteration (power_max_iter = 0).  Pinned
    against the exact 2-norm (SVD), for LPs and for a QP whose scaled diagonal
    Q~_jj joins the column sums (which only enlarges c_j)."""
    rng = np.random.default_rng({"bernoulli": 1, "zipf": 2, "empty_rows_cols": 3,
                                 "qp_diag": 4}[kind])
    m, n = 150, 260
    if kind == "zipf":
        d = lp_instance(m, n, seed=instance_seed(77), nnz=3000, rows="zipf")
        A = sp.csr_matrix((d["val"], d["col"], d["row_ptr"]), shape=(m, n))
    else:
        A = sp.random(m, n, density=0.03, random_state=rng, format="csr",
                      data_rvs=lambda k: rng.standard_normal(k))
        if kind == "empty_rows_cols":
            A = sp.lil_matrix(A)
            A[:7, :] = 0.0
            A[:, :11] = 0.0
            A = sp.csr_matrix(A)
            A.eliminate_zeros()
    qd = rng.uniform(0.1, 1.0, size=n) if kind == "qp_diag" else None
    for ruiz in (0, 10):
        Dr, Dc = O.scaling_factors(A, ruiz, True, qd)
        At = (sp.diags(Dr) @ A @ sp.diags(Dc)).toarray()
        nrm = np.linalg.norm(At, 2)
        assert nrm <= 1.0 + 1e-12, (ruiz, nrm)
        assert nrm >= 0.3  # the bound is not vacuous on these matrices
