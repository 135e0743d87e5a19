"""The two kernels of the fused SpMV half-steps, and the autotuner that picks one.

spmv_fused (one warp per work item) and spmv_pipe (persistent warps owning
contiguous item ranges, matrix rows staged by TMA bulk copies) run the same
work items with the same products and the same order of every sum, so a solve
must return identical bits with either: checked here on whole solves (LP and QP,
FP64 and mixed precision), on matrices whose long rows are cut into many slices
that the pipelined kernel spreads over several warps.  The autotuner times both
on the problem's own matrices once per matrix signature and reuses its choice.
"""
import numpy as np
import pytest

from synth import instance_seed, lp_instance, qp_instance
from tests.gpu_util import create, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


def long_row_lp(seed):
    """LP whose rows of A hold up to 6,000 nonzeros (24 slices of 256) between
    many short ones, so a long row's slices land in several warps' ranges."""
    rng = np.random.default_rng(seed)
    m, n = 3000, 60000
    lens = rng.integers(1, 30, size=m)
    lens[rng.choice(m, size=40, replace=False)] = rng.integers(300, 6000, size=40)
    rows = [np.sort(rng.choice(n, size=k, replace=False)) for k in lens]
    rp = np.zeros(m + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lens)
    col = np.concatenate(rows).astype(np.int32)
    val = rng.standard_normal(int(rp[-1]))
    x0 = rng.uniform(0.0, 10.0, size=n)
    import scipy.sparse as sp
    ax = sp.csr_matrix((val, col, rp), shape=(m, n)) @ x0
    lc = np.where(np.arange(m) < m // 2, ax, ax - rng.uniform(0, 1, size=m))
    uc = np.where(np.arange(m) < m // 2, ax, np.inf)
    y0 = np.where(np.arange(m) < m // 2, rng.standard_normal(m), 0.0)
    c = sp.csr_matrix((val, col, rp), shape=(m, n)).T @ y0
    return dict(m=m, n=n, nnz=int(rp[-1]), row_ptr=rp, col=col, val=val, c=c, lc=lc, uc=uc,
                l=np.zeros(n), u=np.full(n, 10.0))


CASES = {
    "zipf_20k_40k": lambda: lp_instance(20000, 40000, seed=instance_seed(102), nnz=400000,
                                        rows="zipf"),
    "zipf_100k_200k": lambda: lp_instance(100000, 200000, seed=instance_seed(111), nnz=2000000,
                                          rows="zipf"),
    "long_rows": lambda: long_row_lp(112),
    "qp_4000": lambda: qp_instance(4000, 2000, seed=instance_seed(113), a_density=2e-3,
                                   min_row=2),
}


def solve(C, d, **kw):
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(**kw))
        st = C.mpax_get_stats(h)
        x, y = C.mpax_get_solution(h, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    return x, y, st


def same_bits(a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return a.shape == b.shape and np.array_equal(a.view(np.int64), b.view(np.int64))


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_kernels_return_identical_bits(C, case, precision):
    d = CASES[case]()
    kw = dict(precision=precision, eps_abs=1e-6, eps_rel=1e-6, iteration_limit=3000)
    x0, y0, s0 = solve(C, d, spmv_kernel=0, **kw)
    assert list(s0["spmv_kernel"]) == [0, 0] and s0["iterations"] > 64
    for kind in (1, 2):
        x1, y1, s1 = solve(C, d, spmv_kernel=kind, **kw)
        assert list(s1["spmv_kernel"]) == [kind, kind]
        assert s0["iterations"] == s1["iterations"] and s0["restarts"] == s1["restarts"], kind
        assert same_bits(x0, x1) and same_bits(y0, y1), kind
        assert s0["rel_kkt"] == s1["rel_kkt"], kind


def test_autotuner_times_once_and_reuses_its_choice(C):
    # a signature no other test uses, so the first prepare times both kernels
    d = lp_instance(30000, 60000, seed=instance_seed(114), nnz=700000, rows="zipf")
    kw = dict(precision=1, eps_abs=1e-4, eps_rel=1e-4)
    x_t, y_t, s_t = solve(C, d, spmv_kernel=-1, **kw)
    us = list(s_t["spmv_tune_us"])
    assert all(u > 0 for u in us), us
    kinds = list(s_t["spmv_kernel"])
    for q in range(2):  # the fastest kind was kept (another must beat kind 0 by 3%)
        score = [us[3 * q], 1.03 * us[3 * q + 1], 1.03 * us[3 * q + 2]]
        assert kinds[q] == int(np.argmin(score))
    x_c, y_c, s_c = solve(C, d, spmv_kernel=-1, **kw)  # same signature: cached
    assert list(s_c["spmv_tune_us"]) == [0.0] * 6
    assert list(s_c["spmv_kernel"]) == kinds
    x_f, y_f, s_f = solve(C, d, spmv_kernel=0, **kw)
    assert same_bits(x_t, x_f) and same_bits(y_t, y_f) and same_bits(x_c, x_f)
    assert s_t["iterations"] == s_f["iterations"]
