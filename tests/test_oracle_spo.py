"""Pins of the SPO+ oracle: zero at the true cost, convexity along a line, and
the subgradient against central differences of the loss computed with HiGHS
at a point where the inner LP has a unique, non-degenerate optimum."""
import numpy as np
import pytest
from scipy.optimize import linprog

from oracle import pdhg as O
from oracle import spo
from synth import instance_seed, lp_instance


def _highs(p, c):
    A = p.A.toarray()
    eq = p.lc == p.uc
    r = linprog(c, A_ub=-A[~eq], b_ub=-p.lc[~eq], A_eq=A[eq], b_eq=p.lc[eq],
                bounds=list(zip(p.l, p.u)), method="highs")
    assert r.status == 0
    return r.x, r.fun


def _case():
    d = lp_instance(20, 40, seed=instance_seed(404), density=0.3, variant="nondegenerate",
                    tight_frac=0.6)
    p = O.problem_from_arrays(d)
    x_star, z_star = _highs(p, p.c)
    return p, x_star, z_star


OPTS = O.Options(eps_abs=1e-10, eps_rel=1e-10, iteration_limit=10**6)


def test_zero_at_the_true_cost():
    p, x_star, z_star = _case()
    loss, g, _ = spo.spo_plus(p, p.c, x_star, z_star, OPTS)
    assert loss == pytest.approx(0.0, abs=1e-7)


def test_convex_along_a_line():
    p, x_star, z_star = _case()
    rng = np.random.default_rng(3)
    c0, c1 = p.c + rng.normal(0, 1, p.n), p.c + rng.normal(0, 1, p.n)
    l0 = spo.spo_plus(p, c0, x_star, z_star, OPTS)[0]
    l1 = spo.spo_plus(p, c1, x_star, z_star, OPTS)[0]
    lm = spo.spo_plus(p, 0.5 * (c0 + c1), x_star, z_star, OPTS)[0]
    assert lm <= 0.5 * (l0 + l1) + 1e-7
    assert l0 >= -1e-7 and l1 >= -1e-7


def test_subgradient_matches_central_differences():
    p, x_star, z_star = _case()
    rng = np.random.default_rng(5)
    c_hat = p.c + rng.normal(0, 0.5, p.n)
    loss, g, _ = spo.spo_plus(p, c_hat, x_star, z_star, OPTS)

    def highs_loss(ch):
        xt, vt = _highs(p, 2 * ch - p.c)
        return -vt + 2 * ch @ x_star - z_star

    assert loss == pytest.approx(highs_loss(c_hat), abs=1e-6)
    h = 1e-6
    for j in rng.choice(p.n, 8, replace=False):
        e = np.zeros(p.n)
        e[j] = h
        fd = (highs_loss(c_hat + e) - highs_loss(c_hat - e)) / (2 * h)
        assert fd == pytest.approx(g[j], abs=1e-5)


def test_grid_shortest_path_lp_value_is_the_dijkstra_distance():
    """The node-arc LP of the grid shortest path (Sec. 4, the Warcraft LP) solved
    by the oracle has the value of the shortest path found by Dijkstra's
    algorithm (networkx) on the same arc costs, and an integral solution."""
    import networkx as nx
    import scipy.sparse as sp
    from synth import grid_shortest_path_lp
    g = grid_shortest_path_lp(8, B=3, seed=instance_seed(31))
    A = sp.csr_matrix((g["val"], g["col"], g["row_ptr"]), shape=(g["m"], g["n"]))
    for b in range(g["B"]):
        p = O.Problem(A, g["C"][b], g["lc"], g["uc"], g["l"], g["u"])
        r = O.solve_lp(p, O.Options(eps_abs=1e-8, eps_rel=1e-8, iteration_limit=10**6))
        assert r.status == "optimal"
        G = nx.DiGraph()
        G.add_weighted_edges_from(zip(g["tails"].tolist(), g["heads"].tolist(),
                                      g["C"][b].tolist()))
        dist = nx.dijkstra_path_length(G, 0, g["m"] - 1)
        assert r.kkt["primal_obj"] == pytest.approx(dist, rel=1e-6)
        assert np.max(np.minimum(np.abs(r.x), np.abs(1 - r.x))) < 1e-4
