"""GPU parity of the LP path (r^2HPDHG, Algorithm 1) against the FP64 oracle.

Every comparison runs the CUDA library through its C ABI and the oracle on the
same seeded inputs.  Tolerances: one iteration from an identical state 1e-12
(FP64) and 1e-5 (mixed), normwise relative in the inf-norm; integer work
(transpose) bit-exact; converged solves to the stated relative KKT error."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg as O
from synth import csr_random, instance_seed, lp_instance, random_state
from tests.gpu_util import create, lib, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


def zipf_lp(m, n, nnz, seed, variant="literal"):
    return lp_instance(m, n, seed=instance_seed(seed), nnz=nnz, rows="zipf", variant=variant)


def mixed_bounds_lp(m, n, density, seed):
    """Random LP with every bound type (equality, one-sided, free rows; boxed,
    one-sided, free columns) and some empty rows."""
    rng = np.random.default_rng(seed)
    rp, col, val = csr_random(m, n, rng, density=density)
    kinds_r = rng.integers(0, 4, size=m)
    b = rng.standard_normal(m)
    lc = np.where(kinds_r == 0, b, np.where(kinds_r == 1, b - 1, -np.inf))
    uc = np.where(kinds_r == 0, b, np.where(kinds_r == 2, b + 1, np.inf))
    kinds_c = rng.integers(0, 4, size=n)
    l = np.where(kinds_c <= 1, -1.0, -np.inf)
    u = np.where((kinds_c == 0) | (kinds_c == 2), 2.0, np.inf)
    return dict(m=m, n=n, nnz=int(rp[-1]), row_ptr=rp, col=col, val=val,
                c=rng.standard_normal(n), lc=lc, uc=uc, l=l, u=u)


CASES = {
    "bernoulli_300x500": lambda: lp_instance(300, 500, seed=instance_seed(101), density=0.03),
    "zipf_20k_40k": lambda: zipf_lp(20000, 40000, 400000, 102),
    "mixed_bounds": lambda: mixed_bounds_lp(2000, 3000, 0.004, 103),
}


# ----------------------------------------------------------------------------- structure

def _dense_column_csr(m, n, seed):
    """Every row holds column 0 (an A^T row longer than the shared-memory sort)."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(m):
        extra = rng.choice(np.arange(1, n), size=rng.integers(0, 4), replace=False)
        rows.append(np.sort(np.concatenate([[0], extra])))
    rp = np.zeros(m + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    return rp, col, rng.standard_normal(int(rp[-1]))


@pytest.mark.parametrize("case", ["bernoulli_300x500", "zipf_20k_40k", "dense_column"])
def test_transpose_bit_exact(C, case):
    if case == "dense_column":
        rp, col, val = _dense_column_csr(6000, 50, 5)
        m, n = 6000, 50
        d = dict(m=m, n=n, row_ptr=rp, col=col, val=val, c=np.zeros(n), lc=np.full(m, -np.inf),
                 uc=np.full(m, np.inf), l=np.zeros(n), u=np.ones(n))
    else:
        d = CASES[case]()
    h = create(C, d)
    try:
        C.mpax_prepare(h, C.mpax_options_default())
        rpT, colT, valT = C.mpax_get_transpose(h, d["n"], int(d["row_ptr"][-1]))
    finally:
        C.mpax_destroy(h)
    At = sp.csr_matrix((d["val"], d["col"], d["row_ptr"]), shape=(d["m"], d["n"])).T.tocsr()
    At.sort_indices()
    np.testing.assert_array_equal(rpT, At.indptr)
    np.testing.assert_array_equal(colT, At.indices)
    np.testing.assert_array_equal(valT, At.data)


# ----------------------------------------------------------------------------- preprocessing

@pytest.mark.parametrize("case", list(CASES))
def test_scaling_and_norm_match_oracle(C, case):
    d = CASES[case]()
    p = O.problem_from_arrays(d)
    opts = O.Options()
    Dr, Dc = O.scaling_factors(p.A, opts.ruiz_iters, opts.pock_chambolle)
    ps = O.scale_problem(p, Dr, Dc)
    nA, _ = O.power_norm_A(ps.A, opts.power_max_iter, opts.power_tol)
    omega0 = O.initial_primal_weight(ps.c, O.bound_vector(ps.lc, ps.uc))
    h = create(C, d)
    try:
        C.mpax_prepare(h, C.mpax_options_default())
        gDr, gDc, info = C.mpax_get_scaling(h, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    assert rel_inf(gDr, Dr) <= 1e-12
    assert rel_inf(gDc, Dc) <= 1e-12
    assert info["norm_A"] == pytest.approx(nA, rel=1e-9)
    assert info["eta"] == pytest.approx(0.998 / nA, rel=1e-9)
    assert info["omega"] == pytest.approx(omega0, rel=1e-12)


# ----------------------------------------------------------------------------- one iteration

def _oracle_iterations(ps, st, k, tau, sigma, gamma, iters):
    x, y = st["x"].copy(), st["y"].copy()
    xa, ya = st["x_anchor"], st["y_anchor"]
    xh = yh = None
    for t in range(iters):
        xh, yh, _ = O.pdhg_step_lp(ps, x, y, tau, sigma)
        x, y = O.halpern(xh, x, xa, k + t, gamma), O.halpern(yh, y, ya, k + t, gamma)
    return x, y, xh, yh


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec,k,gamma,iters,tol", [
    (0, 0, 1.0, 1, 1e-12), (0, 7, 1.0, 1, 1e-12), (0, 3, 0.5, 1, 1e-12),
    (0, 0, 1.0, 40, 1e-10), (1, 5, 1.0, 1, 1e-5), (1, 2, 0.5, 1, 1e-5)])
def test_iterations_match_oracle(C, case, prec, k, gamma, iters, tol):
    d = CASES[case]()
    p = O.problem_from_arrays(d)
    opts = O.Options(reflection_gamma=gamma)
    Dr, Dc = O.scaling_factors(p.A, opts.ruiz_iters, opts.pock_chambolle)
    ps = O.scale_problem(p, Dr, Dc)
    st = random_state(p.n, p.m, seed=instance_seed(k + 1000))
    tau, sigma = 0.35, 0.6
    x, y, xh, yh = _oracle_iterations(ps, st, k, tau, sigma, gamma, iters)
    h = create(C, d)
    try:
        C.mpax_prepare(h, C.mpax_options_default(precision=prec, reflection_gamma=gamma))
        C.mpax_set_iterate(h, st["x"], st["y"], st["x_anchor"], st["y_anchor"], k, tau, sigma)
        C.mpax_iterate(h, iters)
        gx, gy, gxh, gyh = C.mpax_get_iterate(h, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    assert rel_inf(gxh, xh) <= tol
    assert rel_inf(gyh, yh) <= tol
    assert rel_inf(gx, x) <= tol
    assert rel_inf(gy, y) <= tol


# ----------------------------------------------------------------------------- KKT

@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_kkt_matches_oracle(C, case, prec, tol):
    d = CASES[case]()
    p = O.problem_from_arrays(d)
    rng = np.random.default_rng(3)
    x = np.clip(rng.standard_normal(p.n) * 3, p.l, p.u)
    y = rng.standard_normal(p.m)
    ref = O.kkt(p, x, y)
    h = create(C, d)
    try:
        C.mpax_prepare(h, C.mpax_options_default(precision=prec))
        got = C.mpax_kkt(h, x, y)
    finally:
        C.mpax_destroy(h)
    scale = 1 + abs(ref["primal_obj"]) + abs(ref["dual_obj"])
    for key in ("primal_res", "dual_res", "rel_kkt"):
        assert got[key] == pytest.approx(ref[key], rel=tol, abs=tol * 1e-3), key
    for key in ("primal_obj", "dual_obj", "gap"):
        assert abs(got[key] - ref[key]) <= tol * scale, key


# ----------------------------------------------------------------------------- solves

@pytest.mark.parametrize("variant", ["literal", "nondegenerate"])
def test_solve_200x400_fp64_to_1e8(C, variant):
    d = lp_instance(200, 400, seed=instance_seed(1), density=0.02, variant=variant)
    p = O.problem_from_arrays(d)
    ref = O.solve_lp(p, O.Options(eps_abs=1e-8, eps_rel=1e-8, iteration_limit=400000))
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(eps_abs=1e-8, eps_rel=1e-8,
                                               iteration_limit=400000))
        stats = C.mpax_get_stats(h)
        x, y = C.mpax_get_solution(h, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    assert stats["termination_name"] == "optimal"
    assert stats["rel_kkt"] <= 1e-8
    chk = O.kkt(p, x, y, 1e-8, 1e-8)
    assert chk["rel_kkt"] <= 1.0001e-8
    assert chk["rel_kkt"] == pytest.approx(stats["rel_kkt"], rel=1e-6, abs=1e-13)
    assert chk["primal_obj"] == pytest.approx(d["opt_value"], rel=1e-7)
    # same written rules: the iteration counts agree up to rounding-level decisions
    assert 0.5 * ref.iterations <= stats["iterations"] <= 2 * ref.iterations


def test_solve_zipf_mixed_to_1e4(C):
    d = zipf_lp(20000, 40000, 400000, 104, variant="nondegenerate")
    p = O.problem_from_arrays(d)
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(precision=1, iteration_limit=200000))
        stats = C.mpax_get_stats(h)
        x, y = C.mpax_get_solution(h, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    assert stats["termination_name"] == "optimal"
    chk = O.kkt(p, x, y)
    assert chk["converged"] and chk["rel_kkt"] <= 1e-4
    assert chk["primal_obj"] == pytest.approx(d["opt_value"], rel=1e-3)


def test_device_and_host_inputs_agree(C):
    d = CASES["zipf_20k_40k"]()
    res = []
    for device in (False, True):
        h = create(C, d, device=device)
        try:
            C.mpax_solve(h, C.mpax_options_default(iteration_limit=640))
            res.append((C.mpax_get_stats(h), C.mpax_get_solution(h, d["m"], d["n"])))
        finally:
            C.mpax_destroy(h)
    (s0, (x0, y0)), (s1, (x1, y1)) = res
    assert s0["iterations"] == s1["iterations"] == 640
    np.testing.assert_array_equal(x0, x1)  # deterministic: fixed-order reductions only
    np.testing.assert_array_equal(y0, y1)


# ----------------------------------------------------------------------------- edge cases

def test_no_rows_box_lp(C):
    n = 1000
    rng = np.random.default_rng(1)
    c = rng.standard_normal(n)
    d = dict(m=0, n=n, row_ptr=np.zeros(1, dtype=np.int64), col=np.zeros(0, dtype=np.int32),
             val=np.zeros(0), c=c, lc=np.zeros(0), uc=np.zeros(0), l=np.zeros(n),
             u=np.full(n, 3.0))
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(eps_abs=1e-9, eps_rel=1e-9, iteration_limit=10**6))
        x, _ = C.mpax_get_solution(h, 0, n)
        stats = C.mpax_get_stats(h)
    finally:
        C.mpax_destroy(h)
    assert stats["termination_name"] == "optimal"
    np.testing.assert_allclose(x, np.where(c > 0, 0.0, 3.0), atol=1e-6)


def test_iteration_limit_and_empty_rows(C):
    d = lp_instance(500, 800, seed=instance_seed(5), density=0.002)  # many empty rows
    assert np.sum(np.diff(d["row_ptr"]) == 0) > 50
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(iteration_limit=1))
        s1 = C.mpax_get_stats(h)
        C.mpax_solve(h, C.mpax_options_default(iteration_limit=100, check_every=64))
        s2 = C.mpax_get_stats(h)
    finally:
        C.mpax_destroy(h)
    assert s1["termination_name"] == "iteration_limit" and s1["iterations"] == 1
    assert s2["termination_name"] == "iteration_limit" and s2["iterations"] == 100
    assert s2["kkt_checks"] == 2


def test_long_rows_many_slices(C):
    """A few rows far longer than one slice next to empty and short rows."""
    m, n = 64, 30000
    rng = np.random.default_rng(8)
    lengths = np.zeros(m, dtype=np.int64)
    lengths[::7] = rng.integers(2000, 12000, size=len(lengths[::7]))
    lengths[3::7] = rng.integers(1, 40, size=len(lengths[3::7]))
    rp = np.zeros(m + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lengths)
    col = np.concatenate([np.sort(rng.choice(n, size=L, replace=False)) for L in lengths
                          if L > 0]).astype(np.int32)
    val = rng.standard_normal(int(rp[-1]))
    x0 = rng.uniform(0, 1, n)
    A = sp.csr_matrix((val, col, rp), shape=(m, n))
    b = A @ x0
    d = dict(m=m, n=n, row_ptr=rp, col=col, val=val, c=A.T @ rng.standard_normal(m), lc=b,
             uc=b, l=np.zeros(n), u=np.ones(n))
    p = O.problem_from_arrays(d)
    ps = O.scale_problem(p, *O.scaling_factors(p.A))
    st = random_state(n, m, seed=9)
    x, y, xh, yh = _oracle_iterations(ps, st, 2, 0.4, 0.3, 1.0, 3)
    h = create(C, d)
    try:
        C.mpax_prepare(h, C.mpax_options_default())
        C.mpax_set_iterate(h, st["x"], st["y"], st["x_anchor"], st["y_anchor"], 2, 0.4, 0.3)
        C.mpax_iterate(h, 3)
        gx, gy, gxh, gyh = C.mpax_get_iterate(h, m, n)
    finally:
        C.mpax_destroy(h)
    for a, b_ in ((gx, x), (gy, y), (gxh, xh), (gyh, yh)):
        assert rel_inf(a, b_) <= 1e-12


def test_invalid_inputs_are_rejected(C):
    d = lp_instance(30, 40, seed=instance_seed(6), density=0.2)
    bad = dict(d)
    col = d["col"].copy()
    r = int(np.argmax(np.diff(d["row_ptr"]) >= 2))
    b = int(d["row_ptr"][r])
    col[b], col[b + 1] = col[b + 1], col[b]
    bad["col"] = col
    with pytest.raises(C.MpaxError) as ei:
        create(C, bad)
    assert ei.value.status == 1 and "increasing" in str(ei.value)
    for key, val in (("l", np.full(40, 11.0)), ("c", np.full(40, np.nan))):
        bad = dict(d)
        bad[key] = val
        with pytest.raises(C.MpaxError):
            create(C, bad)
    h = create(C, d)
    try:
        with pytest.raises(C.MpaxError) as ei:
            C.mpax_get_solution(h, d["m"], d["n"])
        assert ei.value.status == 4
        with pytest.raises(C.MpaxError):
            C.mpax_solve(h, C.mpax_options_default(check_every=0))
    finally:
        C.mpax_destroy(h)


def test_time_limit(C):
    d = lp_instance(200, 400, seed=instance_seed(1), density=0.02, variant="nondegenerate")
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(eps_abs=1e-12, eps_rel=1e-12, time_limit=0.0))
        stats = C.mpax_get_stats(h)
    finally:
        C.mpax_destroy(h)
    assert stats["termination_name"] in ("time_limit", "optimal")
    assert stats["iterations"] <= 192


def test_mixed_with_fp64_continuation_reaches_1e8(C):
    """Below the FP32 floor the mixed solve stalls and finishes in FP64 from its
    FP32 point (the final polishing step of the precision pattern)."""
    d = lp_instance(200, 400, seed=instance_seed(1), density=0.02, variant="nondegenerate")
    p = O.problem_from_arrays(d)
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(precision=1, eps_abs=1e-8, eps_rel=1e-8,
                                               iteration_limit=400000))
        stats = C.mpax_get_stats(h)
        x, y = C.mpax_get_solution(h, d["m"], d["n"])
        C.mpax_solve(h, C.mpax_options_default(precision=1, eps_abs=1e-8, eps_rel=1e-8,
                                               iteration_limit=30000, fp64_continuation=0))
        plain = C.mpax_get_stats(h)
    finally:
        C.mpax_destroy(h)
    assert stats["termination_name"] == "optimal"
    assert 0 < stats["fp64_iterations"] < stats["iterations"]
    chk = O.kkt(p, x, y, 1e-8, 1e-8)
    assert chk["converged"]
    assert chk["primal_obj"] == pytest.approx(d["opt_value"], rel=1e-7)
    # FP32 alone does not get there
    assert plain["termination_name"] == "iteration_limit" and plain["rel_kkt"] > 1e-8


def test_certified_norm_bound_without_power_iteration(C):
    """power_max_iter = 0 takes ||A~||_2 := 1 (the Pock-Chambolle bound): the FP64
    solve follows the oracle's run with the same rule."""
    d = lp_instance(200, 400, seed=instance_seed(77), density=0.02, variant="nondegenerate")
    p = O.problem_from_arrays(d)
    ref = O.solve_lp(p, O.Options(eps_abs=1e-8, eps_rel=1e-8, power_max_iter=0))
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(precision=0, eps_abs=1e-8, eps_rel=1e-8,
                                               power_max_iter=0))
        s = C.mpax_get_stats(h)
        x, y = C.mpax_get_solution(h, d["m"], d["n"])
        with pytest.raises(Exception):
            C.mpax_solve(h, C.mpax_options_default(power_max_iter=0, pock_chambolle=0))
    finally:
        C.mpax_destroy(h)
    assert s["norm_A"] == 1.0
    assert s["termination_name"] == "optimal"
    assert abs(s["iterations"] - ref.iterations) <= 2 * 64
    assert O.kkt(p, x, y, 1e-8, 1e-8)["converged"]


def test_f32_create_and_reduced_costs(C):
    """mpax_lp_create_f32 on FP32-representable data solves exactly the problem of
    the FP64 create (bitwise equal results), and the reduced costs are
    c - A^T y at the returned point (oracle arithmetic)."""
    d = lp_instance(200, 400, seed=instance_seed(11), density=0.02, variant="nondegenerate")
    f = {k: np.asarray(d[k], dtype=np.float32) for k in ("val", "c", "lc", "uc", "l", "u")}
    d64 = dict(d, **{k: v.astype(np.float64) for k, v in f.items()})
    opts = C.mpax_options_default(eps_abs=1e-6, eps_rel=1e-6, iteration_limit=100000)
    h1 = create(C, d64)
    h2 = C.mpax_lp_create_f32(d["m"], d["n"], d["row_ptr"], d["col"], f["val"], f["c"], f["lc"],
                              f["uc"], f["l"], f["u"])
    try:
        C.mpax_solve(h1, opts)
        C.mpax_solve(h2, opts)
        x1, y1 = C.mpax_get_solution(h1, d["m"], d["n"])
        x2, y2 = C.mpax_get_solution(h2, d["m"], d["n"])
        lam = C.mpax_get_reduced_cost(h1, d["n"])
    finally:
        C.mpax_destroy(h1)
        C.mpax_destroy(h2)
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2)
    p = O.problem_from_arrays(d64)
    aty = p.A.T @ y1
    ref = p.c - aty
    # lam is a difference of O(1) terms: rounding is relative to them
    assert np.max(np.abs(lam - ref)) <= 1e-13 * (np.max(np.abs(p.c)) + np.max(np.abs(aty)))
    assert np.max(np.abs(ref)) > 0.05


# ----------------------------------------------------------------------------- restarts

@pytest.mark.parametrize("case,eps", [("lp_200x400", 1e-8), ("zipf_20k_40k", 1e-6)])
def test_restart_log_matches_oracle(C, case, eps):
    """Restart rule and primal-weight update (Sec. 3's adaptive restarts and
    primal-weight updates, in the written reading): in FP64 the GPU restarts at
    the same iterations as the oracle and its primal weight after every restart
    equals the oracle's."""
    if case == "lp_200x400":
        d = lp_instance(200, 400, seed=instance_seed(1), density=0.02, variant="nondegenerate")
    else:
        d = zipf_lp(20000, 40000, 400000, 102, variant="nondegenerate")
    p = O.problem_from_arrays(d)
    ref = O.solve_lp(p, O.Options(eps_abs=eps, eps_rel=eps, iteration_limit=400000))
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(eps_abs=eps, eps_rel=eps, iteration_limit=400000))
        stats = C.mpax_get_stats(h)
        it, om, cnt = C.mpax_get_restart_history(h)
    finally:
        C.mpax_destroy(h)
    assert ref.status == "optimal" and stats["termination_name"] == "optimal"
    assert cnt == stats["restarts"] == ref.restarts == len(ref.restart_log)
    k = min(cnt, 256)
    assert list(it) == [t for t, _ in ref.restart_log[:k]]
    # the weights agree to rounding accumulated over the solve (1.2e-9 after the
    # 22 restarts of 275k iterations of the 200 x 400 LP)
    np.testing.assert_allclose(om, [w for _, w in ref.restart_log[:k]], rtol=1e-7, atol=0)
    assert stats["iterations"] == ref.iterations
