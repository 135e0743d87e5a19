"""GPU unrolled differentiation of a QP solve (mpax_qp_unrolled_grad) against the
oracle's reverse sweep along the same path (oracle/unrolled.py, pinned by path
differences), and at convergence against the implicit adjoint."""
import numpy as np
import pytest

from oracle import pdhg as O
from oracle import unrolled as U
from synth import instance_seed, qp_instance
from tests.gpu_util import create, lib, rel_inf
from tests.test_oracle_unrolled import _mixed_rows_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


def _case(name):
    if name == "small":
        # equality, lower- and upper-bounded rows, all active
        p, d = _mixed_rows_problem()
        return dict(d, lc=p.lc, uc=p.uc), 400, 16
    if name == "sparse_q":
        from synth import qp_sparse_q_instance
        return qp_sparse_q_instance(2000, 1000, seed=instance_seed(205), a_density=5e-3,
                                    b_density=1e-3), 320, 32
    # 4000 variables: several SpMV tiles, long and short rows, a ragged tail
    d = qp_instance(4000, 2000, seed=instance_seed(201), a_density=5e-3, f_cols=32,
                    f_density=0.01)
    return d, 640, 64


@pytest.mark.parametrize("name", ["small", "4k", "sparse_q"])
def test_unrolled_gradient_matches_oracle(C, name):
    d, iters, every = _case(name)
    p = O.problem_from_arrays(d)
    res, tape = U.taped_solve(p, O.Options(eps_abs=1e-14, eps_rel=1e-14, iteration_limit=iters,
                                           check_every=every))
    rng = np.random.default_rng(17)
    gx = rng.standard_normal(d["n"])
    gy = rng.standard_normal(d["m"])
    ref = U.unrolled_gradient(p, res, tape, gx, gy)
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(eps_abs=1e-14, eps_rel=1e-14,
                                               iteration_limit=iters, check_every=every,
                                               record_tape=1))
        st = C.mpax_get_stats(h)
        x0, y0 = C.mpax_get_solution(h, d["m"], d["n"])
        G = C.mpax_qp_unrolled_grad(h, gx, d["m"], d["n"], gy)
        x1, y1 = C.mpax_get_solution(h, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    # the same path: length, restarts and end point
    assert st["iterations"] == res.iterations == iters
    assert st["restarts"] == res.restarts
    assert rel_inf(x0, res.x) <= 1e-9
    # the backward pass leaves the returned point as it was
    assert np.array_equal(x0, x1) and np.array_equal(y0, y1)
    for k in ("c", "lc", "uc", "l", "u", "D"):
        assert rel_inf(G[k], ref[k]) <= 1e-8, (k, rel_inf(G[k], ref[k]))
    assert np.max(np.abs(ref["c"])) > 0 and np.max(np.abs(ref["D"])) > 0


def test_unrolled_gradient_tends_to_the_implicit_adjoint(C):
    d = qp_instance(4000, 2000, seed=instance_seed(201), a_density=5e-3, f_cols=32,
                    f_density=0.01)
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(eps_abs=1e-9, eps_rel=1e-9,
                                               iteration_limit=10**6, record_tape=1))
        assert C.mpax_get_stats(h)["termination"] == C.MPAX_TERM_OPTIMAL
        x, _ = C.mpax_get_solution(h, d["m"], d["n"])
        g = x - d["x_target"]
        G = C.mpax_qp_unrolled_grad(h, g, d["m"], d["n"])
        dc, db, dD, info = C.mpax_qp_adjoint(h, g, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    assert info["rel_residual"] <= 1e-8
    assert np.linalg.norm(G["c"] - dc) <= 1e-3 * np.linalg.norm(dc)
    assert np.linalg.norm(G["lc"] + G["uc"] - db) <= 1e-3 * np.linalg.norm(db)
    assert np.linalg.norm(G["D"] - dD) <= 1e-3 * np.linalg.norm(dD)


def test_unrolled_gradient_needs_a_taped_fp64_solve(C):
    d, _, _ = _case("small")
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(iteration_limit=128))
        with pytest.raises(C.MpaxError) as ei:
            C.mpax_qp_unrolled_grad(h, np.ones(d["n"]), d["m"], d["n"])
        assert ei.value.status == C.MPAX_ERR_NOT_SOLVED
        with pytest.raises(C.MpaxError) as ei:
            C.mpax_solve(h, C.mpax_options_default(precision=C.MPAX_PREC_MIXED, record_tape=1))
        assert ei.value.status == C.MPAX_ERR_UNSUPPORTED
        # a taped solve, then an untaped one: the tape is gone
        C.mpax_solve(h, C.mpax_options_default(iteration_limit=128, record_tape=1))
        C.mpax_qp_unrolled_grad(h, np.ones(d["n"]), d["m"], d["n"])
        C.mpax_solve(h, C.mpax_options_default(iteration_limit=128))
        with pytest.raises(C.MpaxError):
            C.mpax_qp_unrolled_grad(h, np.ones(d["n"]), d["m"], d["n"])
    finally:
        C.mpax_destroy(h)


def test_unrolled_layer_matches_the_adjoint_layer(C):
    """QPUnrolledLayer and QPLayer on a converged solve: the same gradients in
    (c, b, D) to the solve's accuracy."""
    import torch
    from paper_2412_09734_gb300.autograd import QPLayer, QPUnrolledLayer
    d = qp_instance(50, 25, seed=instance_seed(202), a_density=0.04, f_cols=32,
                    f_density=0.04, min_row=2)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    data = dict(m=d["m"], n=d["n"], row_ptr=dev(d["row_ptr"]), col=dev(d["col"]),
                val=dev(d["val"]), l=dev(d["l"]), u=dev(d["u"]), f_row_ptr=dev(d["f_row_ptr"]),
                f_col=dev(d["f_col"]), f_val=dev(d["f_val"]), r=d["f_cols"])
    opts = dict(eps_abs=1e-11, eps_rel=1e-11, iteration_limit=10**6)
    xt = dev(d["x_target"])
    grads = []
    for layer in (QPLayer, QPUnrolledLayer):
        c = dev(d["c"]).requires_grad_(True)
        b = dev(d["lc"]).requires_grad_(True)
        D = dev(d["D"]).requires_grad_(True)
        x = layer.apply(c, b, D, data, opts)
        (0.5 * torch.sum((x - xt) ** 2)).backward()
        grads.append([t.grad.cpu().numpy() for t in (c, b, D)])
    for ga, gu in zip(*grads):
        assert np.linalg.norm(gu - ga) <= 1e-4 * np.linalg.norm(ga)


@pytest.mark.parametrize("form", ["diag_lowrank", "sparse_q"])
def test_box_qp_without_rows(C, form):
    """m = 0, Q diagonal: x* = clamp(-c / D, l, u) (closed form), and at
    convergence the unrolled gradient of g . x is -g / D on the free coordinates
    and 0 on the clamped ones."""
    n = 3000
    rng = np.random.default_rng(21)
    D = rng.uniform(0.1, 1.0, n)
    c = 2.0 * rng.standard_normal(n)
    l, u = -np.ones(n), np.ones(n)
    empty = dict(m=0, n=n, row_ptr=np.zeros(1, dtype=np.int64), col=np.zeros(0, dtype=np.int32),
                 val=np.zeros(0), c=c, lc=np.zeros(0), uc=np.zeros(0), l=l, u=u)
    if form == "diag_lowrank":
        d = dict(empty, D=D, f_cols=1, f_row_ptr=np.zeros(n + 1, dtype=np.int64),
                 f_col=np.zeros(0, dtype=np.int32), f_val=np.zeros(0))
    else:
        d = dict(empty, q_row_ptr=np.arange(n + 1, dtype=np.int64),
                 q_col=np.arange(n, dtype=np.int32), q_val=D)
    g = rng.standard_normal(n)
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(eps_abs=1e-10, eps_rel=1e-10,
                                               iteration_limit=10**6, record_tape=1))
        assert C.mpax_get_stats(h)["termination"] == C.MPAX_TERM_OPTIMAL
        x, _ = C.mpax_get_solution(h, 0, n)
        G = C.mpax_qp_unrolled_grad(h, g, 0, n)
    finally:
        C.mpax_destroy(h)
    xs = np.clip(-c / D, l, u)
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-7)
    free = np.abs(xs) < 1 - 1e-3
    np.testing.assert_allclose(G["c"][free], -g[free] / D[free], rtol=1e-6, atol=1e-9)
    assert np.max(np.abs(G["c"][~free])) <= 1e-9
