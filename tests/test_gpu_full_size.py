"""Parity at the bench's full size: the 500k x 1M LP with 10M Zipf-distributed
nonzeros, in the launch configuration bench.py times.  The oracle computes
everything here at full size (its own scaling, one iteration, the KKT
evaluation); the solve is checked through properties that hold at any size
(the oracle's FP64 KKT test of the returned point, the constructed optimum)."""
import numpy as np
import pytest

from oracle import pdhg as O
from synth import instance_seed, lp_instance, random_state
from tests.gpu_util import lib, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


@pytest.fixture(scope="module")
def bench_lp():
    d = lp_instance(500_000, 1_000_000, seed=instance_seed(2), nnz=10_000_000, rows="zipf")
    return d, O.problem_from_arrays(d)


def _create(C, d):
    import torch
    keys = ("row_ptr", "col", "val", "c", "lc", "uc", "l", "u")
    dev = {k: torch.from_numpy(np.ascontiguousarray(d[k])).cuda() for k in keys}
    return C.mpax_lp_create(d["m"], d["n"], *[dev[k] for k in keys]), dev


def test_mixed_solve_meets_the_tolerance_in_the_oracle_evaluation(C, bench_lp):
    d, p = bench_lp
    h, _ = _create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(precision=1))
        s = C.mpax_get_stats(h)
        x, y = C.mpax_get_solution(h, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    assert s["termination_name"] == "optimal"
    chk = O.kkt(p, x, y, 1e-4, 1e-4)
    assert chk["converged"], chk["rel_kkt"]
    # the construction's optimum: every feasible point has value c^T x0
    assert chk["primal_obj"] == pytest.approx(d["opt_value"], rel=1e-3, abs=1e-3)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_one_iteration_matches_the_oracle_at_full_size(C, bench_lp, prec, tol):
    d, p = bench_lp
    opts = O.Options()
    Dr, Dc = O.scaling_factors(p.A, opts.ruiz_iters, opts.pock_chambolle)
    ps = O.scale_problem(p, Dr, Dc)
    st = random_state(p.n, p.m, seed=instance_seed(2024))
    k, tau, sigma = 3, 0.35, 0.6
    xh, yh, _ = O.pdhg_step_lp(ps, st["x"], st["y"], tau, sigma)
    x1 = O.halpern(xh, st["x"], st["x_anchor"], k, 1.0)
    y1 = O.halpern(yh, st["y"], st["y_anchor"], k, 1.0)
    h, _ = _create(C, d)
    try:
        C.mpax_prepare(h, C.mpax_options_default(precision=prec))
        C.mpax_set_iterate(h, st["x"], st["y"], st["x_anchor"], st["y_anchor"], k, tau, sigma)
        C.mpax_iterate(h, 1)
        gx, gy, gxh, gyh = C.mpax_get_iterate(h, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    assert rel_inf(gxh, xh) <= tol
    assert rel_inf(gyh, yh) <= tol
    assert rel_inf(gx, x1) <= tol
    assert rel_inf(gy, y1) <= tol


def test_kkt_evaluation_matches_the_oracle_at_full_size(C, bench_lp):
    d, p = bench_lp
    rng = np.random.default_rng(9)
    x = np.clip(rng.uniform(0, 10, p.n), p.l, p.u)
    y = rng.standard_normal(p.m)
    ref = O.kkt(p, x, y)
    h, _ = _create(C, d)
    try:
        C.mpax_prepare(h, C.mpax_options_default(precision=0))
        got = C.mpax_kkt(h, x, y)
    finally:
        C.mpax_destroy(h)
    for key in ("primal_res", "dual_res", "rel_kkt"):
        assert got[key] == pytest.approx(ref[key], rel=1e-12, abs=1e-15), key
    scale = 1 + abs(ref["primal_obj"]) + abs(ref["dual_obj"])
    for key in ("primal_obj", "dual_obj", "gap"):
        assert abs(got[key] - ref[key]) <= 1e-12 * scale, key
