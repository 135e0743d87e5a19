"""The seeded input generators keep the recipe they state: deterministic per seed,
valid CSR (sorted distinct in-range columns), Zipf totals exact, feasible by
construction with the stated optimum, and Q symmetric positive definite."""
import numpy as np
import pytest
import scipy.sparse as sp

from synth import (instance_seed, knapsack_lp, lp_instance, qp_instance, qp_sparse_q_instance,
                   ragged_lp_batch, shared_dense_lp_batch)
from synth.generators import zipf_row_lengths


def _check_csr(row_ptr, col, m, n):
    assert row_ptr[0] == 0 and len(row_ptr) == m + 1
    assert np.all(np.diff(row_ptr) >= 0) and row_ptr[-1] == len(col)
    assert np.all((col >= 0) & (col < n))
    for i in range(m):
        r = col[row_ptr[i]:row_ptr[i + 1]]
        assert np.all(np.diff(r) > 0)  # sorted and distinct


def test_instances_are_deterministic_per_seed():
    a = lp_instance(300, 600, seed=instance_seed(3), density=0.02)
    b = lp_instance(300, 600, seed=instance_seed(3), density=0.02)
    c = lp_instance(300, 600, seed=instance_seed(4), density=0.02)
    for k in ("row_ptr", "col", "val", "c", "lc", "uc"):
        np.testing.assert_array_equal(a[k], b[k])
    assert not np.array_equal(a["c"], c["c"])


def test_zipf_row_lengths_hit_the_total_exactly():
    rng = np.random.default_rng(1)
    L = zipf_row_lengths(5000, 100_000, rng, max_len=10_000, n_cols=20_000)
    assert L.sum() == 100_000
    assert L.min() >= 1 and L.max() <= 10_000


@pytest.mark.parametrize("variant", ["literal", "nondegenerate"])
def test_lp_instance_is_feasible_with_the_stated_optimum(variant):
    d = lp_instance(400, 800, seed=instance_seed(12), density=0.02, variant=variant)
    _check_csr(d["row_ptr"], d["col"], d["m"], d["n"])
    A = sp.csr_matrix((d["val"], d["col"], d["row_ptr"]), shape=(d["m"], d["n"]))
    x0 = d["x0"]
    ax = A @ x0
    assert np.all(x0 >= d["l"]) and np.all(x0 <= d["u"])
    assert np.all(ax >= d["lc"] - 1e-9) and np.all(ax <= d["uc"] + 1e-9)
    assert d["opt_value"] == pytest.approx(float(d["c"] @ x0), rel=1e-12)


def test_zipf_lp_keeps_its_nonzero_count():
    d = lp_instance(2000, 4000, seed=instance_seed(2), nnz=40_000, rows="zipf")
    assert d["nnz"] == 40_000
    _check_csr(d["row_ptr"], d["col"], d["m"], d["n"])


def test_qp_instances():
    d = qp_instance(300, 150, seed=instance_seed(5), a_density=0.02, f_cols=8, f_density=0.1)
    _check_csr(d["row_ptr"], d["col"], d["m"], d["n"])
    _check_csr(d["f_row_ptr"], d["f_col"], d["n"], d["f_cols"])
    assert np.all((d["D"] >= 0.1) & (d["D"] <= 1.0))
    q = qp_sparse_q_instance(300, 150, seed=instance_seed(6), a_density=0.02, b_density=0.01)
    _check_csr(q["q_row_ptr"], q["q_col"], q["n"], q["n"])
    Q = sp.csr_matrix((q["q_val"], q["q_col"], q["q_row_ptr"]), shape=(300, 300)).toarray()
    assert np.max(np.abs(Q - Q.T)) <= 1e-12 * np.max(np.abs(Q))
    assert np.linalg.eigvalsh(0.5 * (Q + Q.T))[0] >= 0.1 - 1e-9  # B B^T + diag(>= 0.1)


def test_batch_generators():
    b = ragged_lp_batch(6, seed=instance_seed(7), m_lo=20, m_hi=60)
    assert b["m_off"][-1] == len(b["lc"]) and b["n_off"][-1] == len(b["c"])
    assert b["nnz_off"][-1] == len(b["col"]) == b["row_ptr"][-1]
    for k in range(6):
        nk = b["n_off"][k + 1] - b["n_off"][k]
        cols = b["col"][b["nnz_off"][k]:b["nnz_off"][k + 1]]
        assert np.all((cols >= 0) & (cols < nk))  # local column indices
    s = shared_dense_lp_batch(32, 64, 3, seed=instance_seed(8))
    assert s["A"].shape == (32, 64) and s["A"].dtype == np.float32
    assert s["C"].shape == (3, 64)
    k = knapsack_lp(10, 200, seed=instance_seed(9))
    np.testing.assert_allclose(k["uc"], 0.25 * k["A"].astype(np.float64).sum(axis=1), rtol=1e-6)
    assert np.all(k["c"] <= 0)  # the value maximisation min -v^T x


def test_grid_shortest_path_lp_is_a_node_arc_incidence():
    from synth import grid_shortest_path_lp
    g = grid_shortest_path_lp(6, B=2, seed=instance_seed(10))
    _check_csr(g["row_ptr"], g["col"], g["m"], g["n"])
    A = sp.csr_matrix((g["val"], g["col"], g["row_ptr"]), shape=(g["m"], g["n"])).toarray()
    # every arc leaves its tail (+1) and enters its head (-1)
    assert np.all(A[g["tails"], np.arange(g["n"])] == 1)
    assert np.all(A[g["heads"], np.arange(g["n"])] == -1)
    assert np.all(np.abs(A).sum(axis=0) == 2)
    # 8-neighbour arcs on a 6 x 6 grid: 4 k (k - 1) + 4 (k - 1)^2 directed arcs
    assert g["n"] == 4 * 6 * 5 + 4 * 25
    assert g["lc"][0] == 1 and g["lc"][-1] == -1 and g["lc"].sum() == 0
    assert np.array_equal(g["C"], g["W"][:, g["heads"]])


def test_ragged_instances_are_those_of_the_batch():
    """A few instances of a ragged batch, built alone, equal the slices of the
    packed batch, and each is the recipe's instance: lp_instance(m_k, 2 m_k) with
    instance_seed(k) (the bench's oracle sample of the 4096-instance batch relies
    on this)."""
    from synth import ragged_lp_instances
    seed = instance_seed(11)
    b = ragged_lp_batch(12, seed=seed, m_lo=20, m_hi=80)
    picked = ragged_lp_instances(12, [0, 5, 11], seed=seed, m_lo=20, m_hi=80)
    for got, k in zip(picked, (0, 5, 11)):
        m0, m1 = b["m_off"][k], b["m_off"][k + 1]
        n0, n1 = b["n_off"][k], b["n_off"][k + 1]
        z0, z1 = b["nnz_off"][k], b["nnz_off"][k + 1]
        assert got["m"] == m1 - m0 and got["n"] == n1 - n0 == 2 * got["m"]
        np.testing.assert_array_equal(got["row_ptr"], b["row_ptr"][m0:m1 + 1] - z0)
        np.testing.assert_array_equal(got["col"], b["col"][z0:z1])
        np.testing.assert_array_equal(got["val"], b["val"][z0:z1])
        for key, (o0, o1) in (("c", (n0, n1)), ("l", (n0, n1)), ("u", (n0, n1)),
                              ("lc", (m0, m1)), ("uc", (m0, m1))):
            np.testing.assert_array_equal(got[key], b[key][o0:o1])
        ref = lp_instance(int(got["m"]), int(got["n"]), seed=instance_seed(k, seed),
                          density=0.01, lo=0.0, hi=10.0)
        for key in ("row_ptr", "col", "val", "c", "lc", "uc", "l", "u"):
            np.testing.assert_array_equal(got[key], ref[key])
