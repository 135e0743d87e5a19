"""GPU differentiation layer against the oracle's adjoint (which is itself pinned
by central finite differences in tests/test_oracle_adjoint.py), plus the
torch.autograd wrappers against finite differences of GPU solves."""
import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import pdhg as O
from synth import instance_seed, lp_instance, qp_instance
from tests.gpu_util import create, lib, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


def _lp_case():
    return lp_instance(20, 40, seed=instance_seed(404), density=0.3, variant="nondegenerate",
                       tight_frac=0.6)


def _qp_small():
    return qp_instance(50, 25, seed=instance_seed(202), a_density=0.04, f_cols=32,
                       f_density=0.04, min_row=2)


def test_lp_value_gradient_matches_oracle(C):
    d = _lp_case()
    p = O.problem_from_arrays(d)
    ref = O.solve_lp(p, O.Options(eps_abs=1e-11, eps_rel=1e-11, iteration_limit=10**6))
    gr = AD.lp_value_gradient(p, ref.x, ref.y)
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(eps_abs=1e-11, eps_rel=1e-11,
                                               iteration_limit=10**6))
        g = C.mpax_lp_value_grad(h, d["m"], d["n"])
    finally:
        C.mpax_destroy(h)
    for k in ("c", "lc", "uc", "l", "u"):
        assert np.max(np.abs(g[k] - gr[k])) <= 1e-6 * (1 + np.max(np.abs(gr[k]))), k


@pytest.mark.parametrize("case,eps,tol", [("small", 1e-11, 1e-5), ("4k", 1e-8, 1e-3),
                                          ("sparse_q", 1e-11, 1e-5)])
def test_qp_adjoint_matches_oracle(C, case, eps, tol):
    if case == "small":
        d = _qp_small()
    elif case == "sparse_q":
        from synth import qp_sparse_q_instance
        d = qp_sparse_q_instance(50, 25, seed=instance_seed(204), a_density=0.04,
                                 b_density=0.04, min_row=2)
    else:
        d = qp_instance(4000, 2000, seed=instance_seed(201), a_density=5e-3, f_cols=32,
                        f_density=0.01)
    p = O.problem_from_arrays(d)
    ref = O.solve_qp(p, O.Options(eps_abs=eps, eps_rel=eps, iteration_limit=10**6))
    assert ref.status == "optimal"
    free, rows = AD.active_sets(p, ref.x, ref.y, 1e-7, 1e-7)
    rdc, rdb, rdD = AD.qp_adjoint(p, ref.x, ref.y, ref.x - d["x_target"], free, rows)
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(eps_abs=eps, eps_rel=eps, iteration_limit=10**6))
        x, y = C.mpax_get_solution(h, d["m"], d["n"])
        dc, db, dD, info = C.mpax_qp_adjoint(h, x - d["x_target"], d["m"], d["n"], tol=1e-12,
                                             max_iter=20000)
    finally:
        C.mpax_destroy(h)
    assert info["rel_residual"] <= 1e-10
    # the adjoint at the oracle's own optimum: the two solves' points differ by
    # the solve tolerance, which bounds this comparison
    assert rel_inf(dc, rdc) <= tol
    assert rel_inf(db, rdb) <= tol
    assert rel_inf(dD, rdD) <= tol
    # the same linear system: the oracle's direct solve at the GPU's point (same
    # active-set rule); MINRES to a 1e-12 residual must agree to 1e-6
    free_g, rows_g = AD.active_sets(p, x, y, 1e-7, 1e-7)
    gdc, gdb, gdD = AD.qp_adjoint(p, x, y, x - d["x_target"], free_g, rows_g)
    assert rel_inf(dc, gdc) <= 1e-6
    assert rel_inf(db, gdb) <= 1e-6
    assert rel_inf(dD, gdD) <= 1e-6


def test_qp_adjoint_step_limit_zero_gradient_and_determinism(C):
    """The MINRES steps run in captured graphs of three steps with the host
    reading the state every few dozen steps: a step limit that is not a
    multiple of three must still stop exactly there, the MINRES residual must
    not grow with the step count, a zero loss gradient takes no step and gives
    zero, and two runs give identical bits (fixed-order reductions)."""
    d = qp_instance(4000, 2000, seed=instance_seed(201), a_density=5e-3, f_cols=32,
                    f_density=0.01)
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(eps_abs=1e-8, eps_rel=1e-8,
                                               iteration_limit=10**6))
        x, _ = C.mpax_get_solution(h, d["m"], d["n"])
        g = x - d["x_target"]
        prev = np.inf
        for k in (1, 2, 4, 7, 8):
            _, _, _, info = C.mpax_qp_adjoint(h, g, d["m"], d["n"], tol=1e-14, max_iter=k)
            assert info["iterations"] == k
            assert info["rel_residual"] <= prev * (1 + 1e-12)
            prev = info["rel_residual"]
        a = C.mpax_qp_adjoint(h, g, d["m"], d["n"], tol=1e-10, max_iter=20000)
        b = C.mpax_qp_adjoint(h, g, d["m"], d["n"], tol=1e-10, max_iter=20000)
        assert a[3] == b[3] and a[3]["iterations"] < 20000
        assert a[3]["rel_residual"] <= 1e-10
        for u, v in zip(a[:3], b[:3]):
            assert np.array_equal(u, v)
        z = C.mpax_qp_adjoint(h, np.zeros(d["n"]), d["m"], d["n"])
        assert z[3]["iterations"] == 0 and z[3]["rel_residual"] == 0.0
        for u in z[:3]:
            assert not np.any(u)
    finally:
        C.mpax_destroy(h)


def test_qp_layer_autograd_matches_finite_differences(C):
    import torch
    from paper_2412_09734_gb300.autograd import QPLayer
    d = _qp_small()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    data = dict(m=d["m"], n=d["n"], row_ptr=dev(d["row_ptr"]), col=dev(d["col"]),
                val=dev(d["val"]), l=dev(d["l"]), u=dev(d["u"]), f_row_ptr=dev(d["f_row_ptr"]),
                f_col=dev(d["f_col"]), f_val=dev(d["f_val"]), r=d["f_cols"])
    opts = dict(eps_abs=1e-11, eps_rel=1e-11, iteration_limit=10**6)
    xt = dev(d["x_target"])
    c = dev(d["c"]).requires_grad_(True)
    b = dev(d["lc"]).requires_grad_(True)
    D = dev(d["D"]).requires_grad_(True)
    x = QPLayer.apply(c, b, D, data, opts)
    loss = 0.5 * torch.sum((x - xt) ** 2)
    loss.backward()

    def L(c_, b_, D_):
        with torch.no_grad():
            xx = QPLayer.apply(c_, b_, D_, data, opts)
            return float(0.5 * torch.sum((xx - xt) ** 2))

    h = 1e-6
    with torch.no_grad():
        for j in (0, 7, 19, 33):
            e = torch.zeros_like(c)
            e[j] = h
            fd = (L(c + e, b, D) - L(c - e, b, D)) / (2 * h)
            assert fd == pytest.approx(float(c.grad[j]), rel=1e-4, abs=1e-6)
        for i in (1, 12):
            e = torch.zeros_like(b)
            e[i] = h
            fd = (L(c, b + e, D) - L(c, b - e, D)) / (2 * h)
            assert fd == pytest.approx(float(b.grad[i]), rel=1e-4, abs=1e-6)


def test_lp_value_layer_autograd(C):
    import torch
    from paper_2412_09734_gb300.autograd import LPValue
    d = _lp_case()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    data = dict(m=d["m"], n=d["n"], row_ptr=dev(d["row_ptr"]), col=dev(d["col"]),
                val=dev(d["val"]), l=dev(d["l"]), u=dev(d["u"]))
    c = dev(d["c"]).requires_grad_(True)
    v = LPValue.apply(c, dev(d["lc"]), dev(d["uc"]), data,
                      dict(eps_abs=1e-11, eps_rel=1e-11, iteration_limit=10**6))
    v.backward()
    assert float(v) == pytest.approx(d["opt_value"], rel=1e-8)
    np.testing.assert_allclose(c.grad.cpu().numpy(), d["x0"], atol=1e-6)


def test_qp_adjoint_solves_its_system_at_full_size(C):
    """The 200k-variable QP of the bench (n = 200,000, m = 100,000, Q = D + F F^T
    with F 200,000 x 32): a direct solve of the adjoint system is out of reach there
    (F F^T alone holds ~1.3e8 nonzeros), so the returned adjoint is checked against
    the system itself, assembled on the host from the problem data.  With F, R the
    active sets of the oracle's rule at the returned point (Sec. 3.4, the same
    thresholds as the library), w = -dc_F and v = db_R must satisfy
        Q_FF w + A_RF^T v = g_F,   A_RF w = 0
    to the solve's tolerance, dc and db must vanish outside F and R, and
    dD = -w x on F."""
    import scipy.sparse as sp
    d = qp_instance(200_000, 100_000, seed=instance_seed(3), a_density=1e-4, f_cols=32,
                    f_density=0.01)
    m, n = d["m"], d["n"]
    h = create(C, d)
    try:
        C.mpax_solve(h, C.mpax_options_default(precision=C.MPAX_PREC_MIXED))
        x, y = C.mpax_get_solution(h, m, n)
        g = x - d["x_target"]
        dc, db, dD, info = C.mpax_qp_adjoint(h, g, m, n, tol=1e-10, max_iter=20000)
    finally:
        C.mpax_destroy(h)
    assert info["rel_residual"] <= 1e-10
    p = O.problem_from_arrays(d)
    free, rows = AD.active_sets(p, x, y, 1e-7, 1e-7)
    assert not np.any(dc[~free]) and not np.any(db[~rows]) and not np.any(dD[~free])
    A = sp.csr_matrix((d["val"], d["col"], d["row_ptr"]), shape=(m, n))
    F = sp.csr_matrix((d["f_val"], d["f_col"], d["f_row_ptr"]), shape=(n, d["f_cols"]))
    Fi, Ri = np.flatnonzero(free), np.flatnonzero(rows)
    w, v = -dc[Fi], db[Ri]
    ARF = A[Ri][:, Fi]
    FF = F[Fi]
    top = d["D"][Fi] * w + FF @ (FF.T @ w) + ARF.T @ v - g[Fi]
    bot = ARF @ w
    scale = np.linalg.norm(g[Fi])
    assert np.linalg.norm(np.concatenate([top, bot])) <= 1e-6 * scale
    np.testing.assert_array_equal(dD[Fi], -w * x[Fi])
