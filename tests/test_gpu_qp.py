"""GPU parity of the QP path (rAPDHG, Algorithm 2) against the FP64 oracle.
Q = diag(D) + F F^T with F sparse n x r, as in the differentiable-QP workload, and
a general sparse Q (mpax_qp_create)."""
import numpy as np
import pytest

from oracle import pdhg as O
from synth import instance_seed, qp_instance, qp_sparse_q_instance, random_state
from tests.gpu_util import create, lib, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


CASES = {
    # cfg3 shape at reduced size: A 0.1% density, F n x 32 at 1% density
    "qp_20k_10k": lambda: qp_instance(20000, 10000, seed=instance_seed(201), a_density=1e-3,
                                      f_cols=32, f_density=0.01),
    # the n = 50 finite-difference copy: densities raised so each row has >= 2 entries
    "qp_50_25": lambda: qp_instance(50, 25, seed=instance_seed(202), a_density=0.04,
                                    f_cols=32, f_density=0.04, min_row=2),
    # general sparse Q = B B^T + diag (about 5 entries per row at 20k)
    "qpq_20k_10k": lambda: qp_sparse_q_instance(20000, 10000, seed=instance_seed(203),
                                                a_density=1e-3, b_density=1e-4),
    "qpq_50_25": lambda: qp_sparse_q_instance(50, 25, seed=instance_seed(204), a_density=0.04,
                                              b_density=0.04, min_row=2),
}


def _oracle_steps(ps, st, k, tau, sigma, iters):
    x, y, xa, ya = st["x"].copy(), st["y"].copy(), st["xbar"].copy(), st["ybar"].copy()
    for t in range(iters):
        x, y, xa, ya, _ = O.apdhg_step_qp(ps, x, y, xa, ya, k + t, tau, sigma)
    return x, y, xa, ya


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec,k,iters,tol", [(0, 0, 1, 1e-12), (0, 5, 1, 1e-12),
                                              (0, 2, 30, 1e-10), (1, 3, 1, 1e-5)])
def test_apdhg_iterations_match_oracle(C, case, prec, k, iters, tol):
    d = CASES[case]()
    p = O.problem_from_arrays(d)
    ps = O.prepare(p, O.Options())[0]
    st = random_state(p.n, p.m, seed=instance_seed(300 + k))
    tau, sigma = 0.3, 0.5
    x, y, xa, ya = _oracle_steps(ps, st, k, tau, sigma, iters)
    h = create(C, d)
    try:
        C.mpax_prepare(h, C.mpax_options_default(precision=prec))
        C.mpax_set_iterate(h, st["x"], st["y"], st["xbar"], st["ybar"], k, tau, sigma)
        C.mpax_iterate(h, iters)
        gx, gy, gxa, gya = C.mpax_get_iterate(h, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    for got, ref in ((gx, x), (gy, y), (gxa, xa), (gya, ya)):
        assert rel_inf(got, ref) <= tol


@pytest.mark.parametrize("case", list(CASES))
def test_qp_norms_and_kkt_match_oracle(C, case):
    d = CASES[case]()
    p = O.problem_from_arrays(d)
    ps, Dr, Dc, nA, nQ, eta, omega = O.prepare(p, O.Options())
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, p.n)
    y = rng.standard_normal(p.m)
    ref = O.kkt(p, x, y)
    h = create(C, d)
    try:
        C.mpax_prepare(h, C.mpax_options_default())
        gDr, gDc, info = C.mpax_get_scaling(h, d["m"], d["n"])
        got = C.mpax_kkt(h, x, y)
    finally:
        C.mpax_destroy(h)
    assert rel_inf(gDr, Dr) <= 1e-12 and rel_inf(gDc, Dc) <= 1e-12
    assert info["norm_A"] == pytest.approx(nA, rel=1e-9)
    assert info["norm_Q"] == pytest.approx(nQ, rel=1e-9)
    assert info["omega"] == pytest.approx(omega, rel=1e-12)
    scale = 1 + abs(ref["primal_obj"]) + abs(ref["dual_obj"])
    for key in ("primal_res", "dual_res", "rel_kkt"):
        assert got[key] == pytest.approx(ref[key], rel=1e-12, abs=1e-15), key
    for key in ("primal_obj", "dual_obj", "gap"):
        assert abs(got[key] - ref[key]) <= 1e-12 * scale, key


@pytest.mark.parametrize("case,prec,eps", [("qp_50_25", 0, 1e-8), ("qp_20k_10k", 0, 1e-6),
                                           ("qp_20k_10k", 1, 1e-4), ("qpq_50_25", 0, 1e-8),
                                           ("qpq_20k_10k", 0, 1e-6), ("qpq_20k_10k", 1, 1e-4)])
def test_qp_solve_matches_oracle(C, case, prec, eps):
    d = CASES[case]()
    p = O.problem_from_arrays(d)
    ref = O.solve_qp(p, O.Options(eps_abs=eps, eps_rel=eps, iteration_limit=500000))
    assert ref.status == "optimal"
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(precision=prec, eps_abs=eps, eps_rel=eps,
                                               iteration_limit=500000))
        stats = C.mpax_get_stats(h)
        x, y = C.mpax_get_solution(h, d["m"], d["n"])
        lam = C.mpax_get_reduced_cost(h, d["n"])
    finally:
        C.mpax_destroy(h)
    assert stats["termination_name"] == "optimal"
    assert rel_inf(lam, p.qx(x) + p.c - p.A.T @ y) <= 1e-12
    chk = O.kkt(p, x, y, eps, eps)
    assert chk["converged"]
    # strictly convex: the solution is unique; distance bounded by the tolerance
    assert np.max(np.abs(x - ref.x)) <= 1e3 * eps
    assert chk["primal_obj"] == pytest.approx(ref.kkt["primal_obj"], rel=10 * eps, abs=10 * eps)
    if prec == 0:
        assert 0.5 * ref.iterations <= stats["iterations"] <= 2 * ref.iterations
