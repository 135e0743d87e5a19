"""GPU feasibility polishing (Sec. 3.3) against the oracle's polish_lp on the
same inputs: the returned pair meets both polishing tolerances in the oracle's
FP64 evaluation, tracks the oracle's polished pair, and the reported KKT values
are those of the returned pair."""
import numpy as np
import pytest

from oracle import pdhg as O
from synth import instance_seed, lp_instance
from tests.gpu_util import create, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


@pytest.mark.parametrize("seed,prec", [(404, 0), (405, 0), (404, 1)])
def test_polished_pair_meets_the_tolerances(C, seed, prec):
    d = lp_instance(200, 400, seed=instance_seed(seed), density=0.02, variant="nondegenerate")
    p = O.problem_from_arrays(d)
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(precision=prec, eps_abs=1e-3, eps_rel=1e-3,
                                               feasibility_polishing=1, eps_feas_polish=1e-6))
        s = C.mpax_get_stats(h)
        x, y = C.mpax_get_solution(h, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    assert s["termination_name"] == "optimal"
    assert s["polish_iterations"] > 0
    k = O.kkt(p, x, y)
    assert k["primal_res"] <= 1e-6 * (1 + k["b_norm"])
    assert k["dual_res"] <= 1e-6 * (1 + k["c_norm"])
    # the reported figures are those of the returned pair
    assert s["primal_res"] == pytest.approx(k["primal_res"], rel=1e-6, abs=1e-12)
    assert s["rel_kkt"] == pytest.approx(k["rel_kkt"], rel=1e-6, abs=1e-12)
    if prec == 0:
        # the oracle's polishing of the oracle's own point, the same written rules
        r = O.solve_lp(p, O.Options(eps_abs=1e-3, eps_rel=1e-3))
        xp, yp, rp, rd = O.polish_lp(p, r.x, r.y)
        assert abs(s["polish_iterations"] - (rp.iterations + rd.iterations)) <= 4 * 64
        np.testing.assert_allclose(x, xp, atol=1e-4 * (1 + np.abs(xp).max()))
