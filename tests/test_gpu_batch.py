"""GPU parity of the ragged batch path (one persistent launch over many LPs)
against the FP64 oracle run on each instance separately."""
import numpy as np
import pytest

from oracle import pdhg as O
from synth import ragged_lp_batch
from tests.gpu_util import lib, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


def _create(C, d, device=False):
    keys = ("m_off", "n_off", "row_ptr", "col", "val", "c", "lc", "uc", "l", "u")
    arrs = [d[k] for k in keys]
    if device:
        import torch
        arrs = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
    return C.mpax_lp_batch_create(d["B"], *arrs)


def _fp32_kkt_bound(p, x, y, chk):
    """First-order bound on |rel_kkt(FP32 row sums) - rel_kkt(exact)| at (x, y).

    A row sum of L terms computed in FP32 from FP32-rounded scaled values has
    error at most (L + 1) u sum_j |a_j v_j|, u = 2^-24 (standard recursive-summation
    bound plus the rounding of each stored value).  The projections in r_p and r_d
    are 1-Lipschitz, the dual objective's bound terms move by |bound| |d lambda_j|,
    the primal objective is formed in FP64 and does not move, and max() is
    1-Lipschitz in each argument."""
    u = 2.0 ** -24
    A = abs(p.A)
    Lr = np.diff(p.A.indptr) + 1.0
    Lc = np.bincount(p.A.indices, minlength=p.n) + 1.0
    e_ax = u * Lr * (A @ np.abs(x))
    e_aty = u * Lc * (A.T @ np.abs(y))
    bmag = np.where(np.isfinite(p.l), np.abs(p.l), 0.0)
    bmag = np.maximum(bmag, np.where(np.isfinite(p.u), np.abs(p.u), 0.0))
    dp = np.linalg.norm(e_ax) / (1.0 + chk["b_norm"])
    dd = np.linalg.norm(e_aty) / (1.0 + chk["c_norm"])
    dg = float(bmag @ e_aty) / (1.0 + abs(chk["primal_obj"]) + abs(chk["dual_obj"]))
    return max(dp, dd, dg)


@pytest.mark.parametrize("prec,eps,pmax", [(0, 1e-6, 1000), (1, 1e-4, 1000), (0, 1e-6, 0),
                                           (1, 1e-4, 0)])
def test_batch_matches_oracle_per_instance(C, prec, eps, pmax):
    d = ragged_lp_batch(24, seed=5150, m_lo=20, m_hi=300, density=0.05)
    h = _create(C, d, device=(prec == 1))
    try:
        C.mpax_batch_solve(h, C.mpax_options_default(precision=prec, eps_abs=eps, eps_rel=eps,
                                                     iteration_limit=500000,
                                                     power_max_iter=pmax))
        summary, per = C.mpax_batch_get_stats(h, d["B"])
        x, y = C.mpax_batch_get_solution(h, int(d["m_off"][-1]), int(d["n_off"][-1]))
    finally:
        C.mpax_batch_destroy(h)
    assert summary["n_optimal"] == d["B"]
    assert summary["kernel_launches"] >= 1
    for b, inst in enumerate(d["instances"]):
        p = O.problem_from_arrays(inst)
        xs = x[d["n_off"][b]:d["n_off"][b + 1]]
        ys = y[d["m_off"][b]:d["m_off"][b + 1]]
        chk = O.kkt(p, xs, ys, eps, eps)
        assert chk["converged"], (b, chk["rel_kkt"])
        if prec:
            # the mixed path forms A x^ and A^T y^ of its own check from FP32 scaled
            # values with FP32 row sums; its relative KKT error may differ from the
            # FP64 evaluation by at most the first-order rounding bound of those sums
            bound = _fp32_kkt_bound(p, xs, ys, chk)
            assert abs(chk["rel_kkt"] - per["rel_kkt"][b]) <= 2.0 * bound + 1e-12, (b, bound)
        else:
            assert chk["rel_kkt"] == pytest.approx(per["rel_kkt"][b], rel=1e-8, abs=1e-12)
        assert chk["primal_obj"] == pytest.approx(inst["opt_value"], rel=30 * eps, abs=30 * eps)
        if prec == 0 and b < 8:
            ref = O.solve_lp(p, O.Options(eps_abs=eps, eps_rel=eps, iteration_limit=500000,
                                          power_max_iter=pmax))
            # the same written rules give the same trajectory up to rounding
            assert abs(per["iterations"][b] - ref.iterations) <= 2 * 64


def test_batch_iteration_limit_and_stats(C):
    d = ragged_lp_batch(16, seed=77, m_lo=10, m_hi=60, density=0.1)
    h = _create(C, d)
    try:
        C.mpax_batch_solve(h, C.mpax_options_default(iteration_limit=100, eps_abs=1e-14,
                                                     eps_rel=1e-14))
        summary, per = C.mpax_batch_get_stats(h, d["B"])
    finally:
        C.mpax_batch_destroy(h)
    assert np.all(per["status"] == 4) and np.all(per["iterations"] == 100)
    assert summary["iterations_total"] == 1600 and summary["n_optimal"] == 0
    assert np.all(per["seconds"] > 0)
    assert summary["instance_seconds_p50"] <= summary["instance_seconds_p99"]


def test_batch_rejects_bad_columns(C):
    d = ragged_lp_batch(3, seed=9, m_lo=10, m_hi=20, density=0.2)
    bad = dict(d)
    col = d["col"].copy()
    col[0] = d["n_off"][1] + 5  # beyond instance 0's columns
    bad["col"] = col
    with pytest.raises(C.MpaxError) as ei:
        _create(C, bad)
    assert ei.value.status == 1


def test_batch_mixed_continues_stalled_instances_in_fp64(C):
    """64 instances of the bench recipe (m ~ U{50..2000}, 1% density).  With a
    one-check stall window many FP32 runs count as stalled and are continued in
    FP64 from their FP32 points; every instance must still meet 1e-4 in the
    oracle's evaluation.  Without continuation no instance is handed over."""
    d = ragged_lp_batch(64)
    out = {}
    for cont in (1, 0):
        h = _create(C, d, device=True)
        try:
            C.mpax_batch_solve(h, C.mpax_options_default(precision=1, fp64_continuation=cont,
                                                         stall_checks=1, iteration_limit=20000))
            summary, per = C.mpax_batch_get_stats(h, d["B"])
            x, y = C.mpax_batch_get_solution(h, int(d["m_off"][-1]), int(d["n_off"][-1]))
        finally:
            C.mpax_batch_destroy(h)
        out[cont] = (summary, per, x, y)
    summary, per, x, y = out[1]
    assert summary["n_optimal"] == d["B"]
    assert summary["fp64_instances"] >= 1
    for b, inst in enumerate(d["instances"]):
        p = O.problem_from_arrays(inst)
        chk = O.kkt(p, x[d["n_off"][b]:d["n_off"][b + 1]], y[d["m_off"][b]:d["m_off"][b + 1]])
        assert chk["converged"], (b, chk["rel_kkt"])
    assert out[0][0]["fp64_instances"] == 0


def _mixed_bounds_instance(m, n, density, rng):
    """Feasible, bounded LP with every bound type: equality, >=, <= and free rows
    (some rows empty); boxed, lower-only, upper-only and free columns.  x0 lies
    inside the column bounds, the row bounds hold at x0, and c = A_eq^T y0, so
    c^T x = y0^T b_eq on the whole feasible set."""
    from synth import csr_random
    rp, col, val = csr_random(m, n, rng, density=density)
    kc = rng.integers(0, 4, size=n)
    l = np.where((kc == 0) | (kc == 1), -1.0, -np.inf)
    u = np.where((kc == 0) | (kc == 2), 2.0, np.inf)
    x0 = rng.uniform(-0.5, 1.5, size=n)
    ax = np.bincount(np.repeat(np.arange(m), np.diff(rp)), weights=val * x0[col], minlength=m)
    kr = rng.integers(0, 4, size=m)
    lc = np.where(kr == 0, ax, np.where(kr == 1, ax - rng.uniform(0, 1, m), -np.inf))
    uc = np.where(kr == 0, ax, np.where(kr == 2, ax + rng.uniform(0, 1, m), np.inf))
    y0 = np.where(kr == 0, rng.standard_normal(m), 0.0)
    c = np.bincount(col, weights=val * y0[np.repeat(np.arange(m), np.diff(rp))], minlength=n)
    return dict(m=m, n=n, nnz=int(rp[-1]), row_ptr=rp, col=col, val=val, c=c, lc=lc, uc=uc,
                l=l, u=u, opt_value=float(c @ x0))


def test_batch_with_every_bound_type(C):
    rng = np.random.default_rng(2027)
    insts = [_mixed_bounds_instance(int(rng.integers(30, 200)), int(rng.integers(40, 300)),
                                    0.05, rng) for _ in range(12)]
    B = len(insts)
    m_off = np.concatenate([[0], np.cumsum([d["m"] for d in insts])]).astype(np.int64)
    n_off = np.concatenate([[0], np.cumsum([d["n"] for d in insts])]).astype(np.int64)
    nz_off = np.concatenate([[0], np.cumsum([d["nnz"] for d in insts])])
    d = dict(B=B, m_off=m_off, n_off=n_off,
             row_ptr=np.concatenate([[0]] + [x["row_ptr"][1:] + nz_off[i]
                                             for i, x in enumerate(insts)]).astype(np.int64),
             **{k: np.concatenate([x[k] for x in insts]) for k in ("col", "val", "c", "lc",
                                                                  "uc", "l", "u")})
    for prec, eps in ((0, 1e-6), (1, 1e-4)):
        h = _create(C, d, device=(prec == 1))
        try:
            C.mpax_batch_solve(h, C.mpax_options_default(precision=prec, eps_abs=eps,
                                                         eps_rel=eps, iteration_limit=200000))
            summary, per = C.mpax_batch_get_stats(h, B)
            x, y = C.mpax_batch_get_solution(h, int(m_off[-1]), int(n_off[-1]))
        finally:
            C.mpax_batch_destroy(h)
        assert summary["n_optimal"] == B
        for b, inst in enumerate(insts):
            p = O.problem_from_arrays(inst)
            chk = O.kkt(p, x[n_off[b]:n_off[b + 1]], y[m_off[b]:m_off[b + 1]], eps, eps)
            assert chk["converged"], (prec, b, chk["rel_kkt"])
            assert chk["primal_obj"] == pytest.approx(inst["opt_value"], rel=30 * eps,
                                                      abs=30 * eps)


def _pack(insts):
    """Pack instance dictionaries like synth.ragged_lp_batch."""
    B = len(insts)
    m_off = np.zeros(B + 1, dtype=np.int64)
    n_off = np.zeros(B + 1, dtype=np.int64)
    nnz_off = np.zeros(B + 1, dtype=np.int64)
    np.cumsum([d["m"] for d in insts], out=m_off[1:])
    np.cumsum([d["n"] for d in insts], out=n_off[1:])
    np.cumsum([d["nnz"] for d in insts], out=nnz_off[1:])
    row_ptr = np.concatenate([[0]] + [d["row_ptr"][1:] + nnz_off[i] for i, d in enumerate(insts)])
    cat = lambda k: np.concatenate([d[k] for d in insts])  # noqa: E731
    return dict(B=B, m_off=m_off, n_off=n_off, row_ptr=row_ptr.astype(np.int64),
                col=cat("col"), val=cat("val"), c=cat("c"), lc=cat("lc"), uc=cat("uc"),
                l=cat("l"), u=cat("u"), instances=insts)


def _iterate_batch():
    from synth import instance_seed, lp_instance
    ms = [20, 64, 150, 333, 700, 2000]
    return _pack([lp_instance(m, 2 * m, seed=instance_seed(7000 + i), density=0.01 if m > 500
                              else 0.05, variant="nondegenerate") for i, m in enumerate(ms)])


@pytest.mark.parametrize("prec,k,tol,pmax", [(0, 192, 1e-12, 0), (0, 192, 1e-12, 1000),
                                              (1, 64, 1e-5, 0)],
                         ids=["fp64_192_bound", "fp64_192_power", "mixed_64_bound"])
def test_batch_iterates_match_oracle(C, prec, k, tol, pmax):
    """Iterate-level parity of the persistent batch kernel (eqs. 3-4, Algorithm 1
    per instance): k iterations from zero, with the checks, restarts and
    primal-weight updates they include, give the oracle's (x^, y^) of the last
    check element by element (normwise relative in the inf-norm), with the same
    number of restarts, for instances from m = 20 to m = 2000.  In mixed
    precision the step sizes come from the certified bound ||A~||_2 <= 1: an FP32
    power iteration may stop one round earlier or later than the FP64 one, which
    moves its estimate (and so tau, sigma) by up to power_tol."""
    d = _iterate_batch()
    h = _create(C, d)
    try:
        C.mpax_batch_solve(h, C.mpax_options_default(precision=prec, iteration_limit=k,
                                                     eps_abs=1e-14, eps_rel=1e-14,
                                                     power_max_iter=pmax))
        summary, per = C.mpax_batch_get_stats(h, d["B"])
        x, y = C.mpax_batch_get_solution(h, int(d["m_off"][-1]), int(d["n_off"][-1]))
    finally:
        C.mpax_batch_destroy(h)
    assert np.all(per["iterations"] == k)
    restarts = 0
    for b, inst in enumerate(d["instances"]):
        p = O.problem_from_arrays(inst)
        ref = O.solve_lp(p, O.Options(eps_abs=1e-14, eps_rel=1e-14, iteration_limit=k,
                                      power_max_iter=pmax, eps_primal_infeasible=0.0,
                                      eps_dual_infeasible=0.0))
        xs = x[d["n_off"][b]:d["n_off"][b + 1]]
        ys = y[d["m_off"][b]:d["m_off"][b + 1]]
        assert ref.iterations == k
        assert rel_inf(xs, ref.x) <= tol, (b, rel_inf(xs, ref.x))
        assert rel_inf(ys, ref.y) <= tol, (b, rel_inf(ys, ref.y))
        restarts += ref.restarts
    assert summary["restarts_total"] == restarts


def _oversized_batch():
    from synth import instance_seed, lp_instance
    small = [lp_instance(m, 2 * m, seed=instance_seed(7100 + i), density=0.05,
                         variant="nondegenerate") for i, m in enumerate([40, 120, 300])]
    # m + n = 36,000: shared memory in FP32 (<= 51,200), global memory in FP64 (> 25,600)
    mid = lp_instance(12000, 24000, seed=instance_seed(7110), density=3e-4,
                      variant="nondegenerate")
    # m + n = 60,000: global memory in both precisions
    big = lp_instance(20000, 40000, seed=instance_seed(7111), density=1.5e-4,
                      variant="nondegenerate")
    return _pack(small[:2] + [mid] + small[2:] + [big])


def _check_batch(d, x, y, per, eps):
    for b, inst in enumerate(d["instances"]):
        p = O.problem_from_arrays(inst)
        xs = x[d["n_off"][b]:d["n_off"][b + 1]]
        ys = y[d["m_off"][b]:d["m_off"][b + 1]]
        chk = O.kkt(p, xs, ys, eps, eps)
        assert per["status"][b] == 1 and chk["converged"], (b, chk["rel_kkt"])
        assert chk["primal_obj"] == pytest.approx(inst["opt_value"], rel=30 * eps, abs=30 * eps)


def test_batch_instances_beyond_shared_memory_fp64(C):
    """Instances whose vectors exceed a CTA's shared memory run from global
    memory (m + n = 36,000 and 60,000 in FP64), beside shared-memory ones in the
    same launch; with such an instance in the launch no row pointers are staged."""
    d = _oversized_batch()
    eps = 1e-6
    h = _create(C, d)
    try:
        C.mpax_batch_solve(h, C.mpax_options_default(precision=0, eps_abs=eps, eps_rel=eps,
                                                     iteration_limit=200000))
        summary, per = C.mpax_batch_get_stats(h, d["B"])
        x, y = C.mpax_batch_get_solution(h, int(d["m_off"][-1]), int(d["n_off"][-1]))
    finally:
        C.mpax_batch_destroy(h)
    assert summary["n_optimal"] == d["B"]
    _check_batch(d, x, y, per, eps)


def test_batch_fp64_continuation_of_an_instance_beyond_shared_memory(C):
    """A mixed solve below the FP32 floor stalls; its FP64 continuation launch
    takes instances whose FP64 vectors no longer fit in shared memory (the
    m + n = 36,000 one fits in FP32 but not in FP64), and every instance meets
    the tolerance in the oracle's evaluation."""
    d = _oversized_batch()
    eps = 1e-7
    h = _create(C, d)
    try:
        C.mpax_batch_solve(h, C.mpax_options_default(precision=1, eps_abs=eps, eps_rel=eps,
                                                     iteration_limit=400000))
        summary, per = C.mpax_batch_get_stats(h, d["B"])
        x, y = C.mpax_batch_get_solution(h, int(d["m_off"][-1]), int(d["n_off"][-1]))
    finally:
        C.mpax_batch_destroy(h)
    assert summary["fp64_instances"] >= 1
    assert summary["n_optimal"] == d["B"]
    _check_batch(d, x, y, per, eps)


@pytest.mark.parametrize("many", [False, True], ids=["one_per_sm", "many_per_sm"])
@pytest.mark.parametrize("prec", [0, 1])
def test_batch_whole_instance_staging_gives_identical_bits(C, prec, many):
    """batch_stage = 1 copies every instance that fits (both matrices, data and
    iterates) into shared memory before it iterates when each instance has an
    SM (6 instances here); the arithmetic and its order are those of the
    in-place path, so a fixed number of iterations (checks, restarts and
    primal-weight updates included) gives the same bits.  With 200 instances
    (more than the SMs) nothing is staged whole and the option changes nothing."""
    if many:
        d = ragged_lp_batch(200, seed=5151, m_lo=20, m_hi=300, density=0.05)
    else:
        d = _iterate_batch()
    out = []
    for stage in (1, 0):
        h = _create(C, d)
        try:
            C.mpax_batch_solve(h, C.mpax_options_default(precision=prec, iteration_limit=320,
                                                         eps_abs=1e-14, eps_rel=1e-14,
                                                         batch_stage=stage))
            summary, per = C.mpax_batch_get_stats(h, d["B"])
            x, y = C.mpax_batch_get_solution(h, int(d["m_off"][-1]), int(d["n_off"][-1]))
        finally:
            C.mpax_batch_destroy(h)
        out.append((x, y, per["iterations"], summary["restarts_total"]))
    (x1, y1, i1, r1), (x0, y0, i0, r0) = out
    assert np.array_equal(i1, i0) and r1 == r0
    assert np.array_equal(x1, x0)
    assert np.array_equal(y1, y0)


def test_batch_stage_option_is_validated(C):
    d = ragged_lp_batch(2, seed=5152, m_lo=20, m_hi=40, density=0.05)
    h = _create(C, d)
    try:
        with pytest.raises(C.MpaxError):
            C.mpax_batch_solve(h, C.mpax_options_default(batch_stage=2))
    finally:
        C.mpax_batch_destroy(h)
