"""GPU infeasibility detection (LP) against the oracle's classification on the
same inputs, in FP64 and in mixed precision (where the FP32 run stalls and the
FP64 continuation certifies)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg as O
from synth import instance_seed, lp_instance
from tests.gpu_util import lib

pytestmark = pytest.mark.gpu
INF = np.inf


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


def _arrays(p):
    A = sp.csr_matrix(p.A)
    return dict(m=p.m, n=p.n, row_ptr=A.indptr.astype(np.int64), col=A.indices.astype(np.int32),
                val=A.data.astype(np.float64), c=p.c, lc=p.lc, uc=p.uc, l=p.l, u=p.u)


def _gpu_status(C, p, prec):
    d = _arrays(p)
    h = C.mpax_lp_create(d["m"], d["n"], d["row_ptr"], d["col"], d["val"], d["c"], d["lc"],
                         d["uc"], d["l"], d["u"])
    try:
        C.mpax_solve(h, C.mpax_options_default(precision=prec, iteration_limit=200000))
        return C.mpax_get_stats(h)
    finally:
        C.mpax_destroy(h)


def _p(A, c, lc, uc, l, u):
    return O.Problem(sp.csr_matrix(np.asarray(A, dtype=np.float64)), np.asarray(c, float),
                     np.asarray(lc, float), np.asarray(uc, float), np.asarray(l, float),
                     np.asarray(u, float))


def _contradicting(m, n, seed, **kw):
    d = lp_instance(m, n, seed=instance_seed(seed), **kw)
    p0 = O.problem_from_arrays(d)
    A = sp.vstack([p0.A, p0.A[0]]).tocsr()
    return O.Problem(A, p0.c, np.append(p0.lc, p0.uc[0] + 1.0), np.append(p0.uc, INF), p0.l, p0.u)


CASES = {
    "two_equalities": lambda: _p([[1, 1], [1, 1]], [1, 1], [1, 2], [1, 2], [0, 0], [10, 10]),
    "above_box": lambda: _p([[1, 1]], [1, -1], [3], [INF], [0, 0], [1, 1]),
    "unbounded_diag": lambda: _p([[1, -1]], [-1, 0], [0], [0], [0, 0], [INF, INF]),
    "unbounded_ineq": lambda: _p([[1, -1]], [-1, -1], [-1], [INF], [0, 0], [INF, INF]),
    "random_30x60": lambda: _contradicting(30, 60, 5, density=0.2),
    "zipf_20k_40k": lambda: _contradicting(20_000, 40_000, 9, nnz=400_000, rows="zipf"),
}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", list(CASES))
def test_classification_matches_oracle(C, case, prec):
    p = CASES[case]()
    ref = O.solve_lp(p, O.Options(iteration_limit=200000))
    assert ref.status in ("primal_infeasible", "dual_infeasible")
    s = _gpu_status(C, p, prec)
    assert s["termination_name"] == ref.status, (s["termination_name"], s["iterations"])
    if prec == 0:
        # the same written rules: the same check (up to a few checks of rounding drift)
        assert abs(s["iterations"] - ref.iterations) <= 4 * 64


def test_detection_can_be_turned_off(C):
    p = CASES["two_equalities"]()
    d = _arrays(p)
    h = C.mpax_lp_create(d["m"], d["n"], d["row_ptr"], d["col"], d["val"], d["c"], d["lc"],
                         d["uc"], d["l"], d["u"])
    try:
        C.mpax_solve(h, C.mpax_options_default(precision=0, iteration_limit=2048,
                                               eps_primal_infeasible=0.0, eps_dual_infeasible=0.0))
        s = C.mpax_get_stats(h)
    finally:
        C.mpax_destroy(h)
    assert s["termination_name"] == "iteration_limit"
