"""Pins of the unrolled-differentiation oracle (oracle/unrolled.py).

* Along a fixed path the returned point is a piecewise-affine function of the
  data, so central differences of the path replayed with perturbed data equal
  the reverse sweep's gradients up to rounding (every parameter kind: c, the
  row bounds of equality and inequality rows, the variable bounds, D).
* At convergence on a non-degenerate strictly convex QP the unrolled gradient
  tends to the implicit-function gradient of the optimum (oracle.adjoint,
  itself pinned by differences of converged solves).
* One step from zero: x1 = proj(-tau c~), so dL/dc = -tau D_c^2 gx inside the box.
"""
import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import pdhg as O
from oracle import unrolled as U
from synth import instance_seed, qp_instance


def _mixed_rows_problem(seed=202):
    """The 50 x 25 QP with every other equality row made one-sided on the side
    its multiplier has at the optimum (y_i > 0: lc_i <= a_i x, y_i < 0:
    a_i x <= uc_i), so the optimum is unchanged and both kinds of row are
    active."""
    d = qp_instance(50, 25, seed=instance_seed(seed), a_density=0.04, f_cols=32,
                    f_density=0.04, min_row=2)
    p = O.problem_from_arrays(d)
    r = O.solve_qp(p, O.Options(eps_abs=1e-9, eps_rel=1e-9, iteration_limit=10**6))
    assert r.status == "optimal"
    lc, uc = p.lc.copy(), p.uc.copy()
    for i in range(0, p.m, 2):
        if r.y[i] > 0:
            uc[i] = np.inf
        else:
            lc[i] = -np.inf
    return O.Problem(p.A, p.c, lc, uc, p.l, p.u, p.Q), d


def _path_loss(p, res, sched, gx, gy):
    ps = O.scale_problem(p, res.Dr, res.Dc)
    xa, ya = U.replay(ps, sched)
    return float(gx @ (res.Dc * xa) + gy @ (res.Dr * ya))


def test_unrolled_gradient_matches_path_differences():
    p, _ = _mixed_rows_problem()
    opts = O.Options(eps_abs=1e-14, eps_rel=1e-14, iteration_limit=400, check_every=16)
    res, tape = U.taped_solve(p, opts)
    assert res.iterations == 400
    assert sum(1 for e in tape if e[0] == "restart") >= 2
    rng = np.random.default_rng(9)
    gx = rng.standard_normal(p.n)
    gy = rng.standard_normal(p.m)
    G = U.unrolled_gradient(p, res, tape, gx, gy)
    # the returned point is the taped path's end
    ps = O.scale_problem(p, res.Dr, res.Dc)
    xa, ya = U.replay(ps, U.schedule(tape))
    np.testing.assert_allclose(res.Dc * xa, res.x, rtol=0, atol=1e-12)
    sched = U.schedule(tape)
    h = 1e-7

    def fd(make):
        return (_path_loss(make(+h), res, sched, gx, gy)
                - _path_loss(make(-h), res, sched, gx, gy)) / (2 * h)

    def close(a, b):
        assert a == pytest.approx(b, rel=1e-5, abs=1e-6)

    def with_(**kw):
        base = dict(A=p.A, c=p.c, lc=p.lc, uc=p.uc, l=p.l, u=p.u, Q=p.Q)
        base.update(kw)
        return O.Problem(**base)

    # c, along coordinates and along one random direction
    for j in rng.choice(p.n, 6, replace=False):
        close(fd(lambda s, j=j: with_(c=p.c + s * np.eye(p.n)[j])), G["c"][j])
    dirc = rng.standard_normal(p.n)
    close(fd(lambda s: with_(c=p.c + s * dirc)), float(G["c"] @ dirc))
    # row bounds: equality rows move both bounds, inequality rows their finite one
    eq = np.flatnonzero(p.lc == p.uc)
    lo_only = np.flatnonzero(np.isfinite(p.lc) & ~np.isfinite(p.uc))
    hi_only = np.flatnonzero(~np.isfinite(p.lc) & np.isfinite(p.uc))
    assert len(eq) and len(lo_only) and len(hi_only)
    for i in eq[:5]:
        e = np.eye(p.m)[i]
        close(fd(lambda s, e=e: with_(lc=p.lc + s * e, uc=p.uc + s * e)),
              G["lc"][i] + G["uc"][i])
    for i in lo_only[:3]:
        e = np.eye(p.m)[i]
        assert G["lc"][i] != 0
        close(fd(lambda s, e=e: with_(lc=p.lc + s * e)), G["lc"][i])
    for i in hi_only[:3]:
        e = np.eye(p.m)[i]
        assert G["uc"][i] != 0
        close(fd(lambda s, e=e: with_(uc=p.uc + s * e)), G["uc"][i])
    # variable bounds: the ones the path touched have nonzero gradients
    for key in ("l", "u"):
        hit = np.flatnonzero(G[key] != 0)
        assert len(hit) > 0
        for j in hit[:4]:
            e = np.eye(p.n)[j]
            close(fd(lambda s, e=e, key=key: with_(**{key: getattr(p, key) + s * e})),
                  G[key][j])
    # D of Q = diag(D) + F F^T
    for j in rng.choice(p.n, 5, replace=False):
        def mk(s, j=j):
            D = p.Q.D.copy()
            D[j] += s
            return with_(Q=O.DiagLowRankQ(D, p.Q.F))
        close(fd(mk), G["D"][j])


def test_unrolled_gradient_tends_to_the_implicit_adjoint():
    p, d = _mixed_rows_problem()
    xt = d["x_target"]
    opts = O.Options(eps_abs=1e-11, eps_rel=1e-11, iteration_limit=10**6)
    res, tape = U.taped_solve(p, opts)
    assert res.status == "optimal"
    g = res.x - xt
    G = U.unrolled_gradient(p, res, tape, g)
    free, rows = AD.active_sets(p, res.x, res.y, 1e-7, 1e-7)
    dc, db, dD = AD.qp_adjoint(p, res.x, res.y, g, free, rows)
    scale = np.linalg.norm(dc)
    assert np.linalg.norm(G["c"] - dc) <= 1e-5 * scale
    assert np.linalg.norm(G["lc"] + G["uc"] - db) <= 1e-5 * np.linalg.norm(db)
    assert np.linalg.norm(G["D"] - dD) <= 1e-5 * np.linalg.norm(dD)


def test_one_step_closed_form():
    p, _ = _mixed_rows_problem()
    res, tape = U.taped_solve(p, O.Options(iteration_limit=1))
    (_, k, tau, sigma, *_), = tape
    assert k == 0
    gx = np.random.default_rng(2).standard_normal(p.n)
    G = U.unrolled_gradient(p, res, tape, gx)
    ps = O.scale_problem(p, res.Dr, res.Dc)
    v = -tau * ps.c
    inside = (v > ps.l) & (v < ps.u)
    np.testing.assert_allclose(G["c"][inside], -tau * res.Dc[inside] ** 2 * gx[inside],
                               rtol=1e-14, atol=0)
    assert np.all(G["c"][~inside] == 0)


def test_sparse_q_unrolled_gradient_matches_path_differences():
    """A general sparse Q: dL/dc and the gradient of Q's diagonal along the path."""
    import scipy.sparse as sp
    from synth import qp_sparse_q_instance
    d = qp_sparse_q_instance(50, 25, seed=instance_seed(204), a_density=0.04, b_density=0.04,
                             min_row=2)
    p = O.problem_from_arrays(d)
    res, tape = U.taped_solve(p, O.Options(eps_abs=1e-14, eps_rel=1e-14, iteration_limit=300,
                                           check_every=16))
    rng = np.random.default_rng(12)
    gx = rng.standard_normal(p.n)
    G = U.unrolled_gradient(p, res, tape, gx)
    sched = U.schedule(tape)
    gy = np.zeros(p.m)
    h = 1e-7

    def fd(make):
        return (_path_loss(make(+h), res, sched, gx, gy)
                - _path_loss(make(-h), res, sched, gx, gy)) / (2 * h)

    for j in rng.choice(p.n, 4, replace=False):
        e = np.eye(p.n)[j]
        assert fd(lambda s, e=e: O.Problem(p.A, p.c + s * e, p.lc, p.uc, p.l, p.u, p.Q)) == \
            pytest.approx(G["c"][j], rel=1e-5, abs=1e-6)
    for j in rng.choice(p.n, 4, replace=False):
        e = np.eye(p.n)[j]
        mk = lambda s, e=e: O.Problem(p.A, p.c, p.lc, p.uc, p.l, p.u,  # noqa: E731
                                      O.SparseQ(p.Q.Q + sp.diags(s * e)))
        assert fd(mk) == pytest.approx(G["D"][j], rel=1e-5, abs=1e-6)
