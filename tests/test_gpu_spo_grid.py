"""SPO+ over a sparse feasible set through the ragged batch: the grid shortest-path
LP of the paper's Warcraft experiment (Sec. 4, the node-arc LP), B cost vectors
solved as B instances of one launch.  Values against Dijkstra's algorithm; losses
and subgradients against the oracle's SPO+ on the same costs."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg as O
from oracle import spo
from synth import grid_shortest_path_lp, instance_seed
from tests.gpu_util import lib

pytestmark = pytest.mark.gpu

OPTS = dict(eps_abs=1e-7, eps_rel=1e-7, iteration_limit=10**6)


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


def _dijkstra(g, cost):
    import networkx as nx
    G = nx.DiGraph()
    G.add_weighted_edges_from(zip(g["tails"].tolist(), g["heads"].tolist(), cost.tolist()))
    return nx.dijkstra_path_length(G, 0, g["m"] - 1)


def test_sparse_lp_values_are_shortest_path_lengths(C):
    import torch
    from paper_2412_09734_gb300.autograd import SparseFeasibleSet, SparseLPValues
    g = grid_shortest_path_lp(8, B=6, seed=instance_seed(41))
    fs = SparseFeasibleSet(g, g["B"])
    Cm = torch.from_numpy(g["C"]).cuda().requires_grad_(True)
    v = SparseLPValues.apply(Cm, fs, OPTS)
    v.sum().backward()
    X = Cm.grad.cpu().numpy()
    A = sp.csr_matrix((g["val"], g["col"], g["row_ptr"]), shape=(g["m"], g["n"]))
    for b in range(g["B"]):
        dist = _dijkstra(g, g["C"][b])
        assert float(v[b]) == pytest.approx(dist, rel=1e-5)
        # the gradient row is the optimal flow: conservation, in the box, value dist
        assert np.max(np.abs(A @ X[b] - g["lc"])) <= 1e-5
        assert X[b].min() >= -1e-6 and X[b].max() <= 1 + 1e-6
        assert float(g["C"][b] @ X[b]) == pytest.approx(dist, rel=1e-5)


def test_sparse_spo_plus_matches_oracle(C):
    import torch
    from paper_2412_09734_gb300.autograd import (SparseFeasibleSet, SparseLPValues,
                                                 SPOPlusLossSparse)
    g = grid_shortest_path_lp(8, B=4, seed=instance_seed(42))
    fs = SparseFeasibleSet(g, g["B"])
    rng = np.random.default_rng(5)
    Ct = torch.from_numpy(g["C"]).cuda()
    with torch.no_grad():
        zt = SparseLPValues.apply(Ct, fs, OPTS)
    # the true optimal flows (GPU), for the GPU loss
    Ctg = Ct.clone().requires_grad_(True)
    SparseLPValues.apply(Ctg, fs, OPTS).sum().backward()
    Xt = Ctg.grad.detach()
    Ch_np = g["C"] + rng.normal(0, 0.3, g["C"].shape)
    Ch = torch.from_numpy(Ch_np).cuda().requires_grad_(True)
    loss = SPOPlusLossSparse.apply(Ch, Ct, Xt, zt, fs, OPTS)
    loss.sum().backward()
    G = Ch.grad.cpu().numpy()
    Lg = loss.detach().cpu().numpy()
    A = sp.csr_matrix((g["val"], g["col"], g["row_ptr"]), shape=(g["m"], g["n"]))
    oo = O.Options(eps_abs=1e-8, eps_rel=1e-8, iteration_limit=10**6)
    for b in range(g["B"]):
        p = O.Problem(A, g["C"][b].copy(), g["lc"], g["uc"], g["l"], g["u"])
        ref = O.solve_lp(p, oo)  # the oracle's own true optimum
        lo, _, _ = spo.spo_plus(p, Ch_np[b], ref.x, ref.kkt["primal_obj"], oo)
        assert Lg[b] == pytest.approx(lo, rel=1e-3, abs=1e-3)
        for _ in range(3):
            delta = rng.normal(0, 0.1, g["n"])
            l2 = spo.spo_plus(p, Ch_np[b] + delta, ref.x, ref.kkt["primal_obj"], oo)[0]
            assert l2 >= lo + G[b] @ delta - 1e-3 * (1 + abs(lo))


def test_spo_plus_layers_stay_on_the_device(C, monkeypatch):
    """SPO+ forward and backward with CUDA tensors move no tensor to the host: the
    costs 2 c^ - c, the solve, the losses and the subgradients are formed in the
    library on device pointers, and every tensor-to-host conversion is disabled
    while the layers run."""
    import torch
    from paper_2412_09734_gb300.autograd import (SparseFeasibleSet, SparseLPValues,
                                                 SPOPlusLossSparse)
    g = grid_shortest_path_lp(6, B=3, seed=instance_seed(43))
    fs = SparseFeasibleSet(g, g["B"])
    Ct = torch.from_numpy(g["C"]).cuda()
    Ch = (Ct + 0.2 * torch.randn_like(Ct)).requires_grad_(True)

    def no_host(*a, **k):
        raise AssertionError("a tensor was copied to the host")

    with monkeypatch.context() as mp:
        for name in ("cpu", "numpy", "item", "tolist"):
            mp.setattr(torch.Tensor, name, no_host)
        Ctg = Ct.clone().requires_grad_(True)
        zt = SparseLPValues.apply(Ctg, fs, OPTS)
        zt.sum().backward()
        Xt = Ctg.grad.detach()
        loss = SPOPlusLossSparse.apply(Ch, Ct, Xt, zt.detach(), fs, OPTS)
        loss.sum().backward()
        assert loss.is_cuda and Ch.grad.is_cuda and Xt.is_cuda
    # the loss of the true costs is zero (x~ = x* when c^ = c)
    with torch.no_grad():
        l0 = SPOPlusLossSparse.apply(Ct, Ct, Xt, zt.detach(), fs, OPTS)
    assert float(l0.abs().max()) <= 1e-5 * (1 + float(zt.abs().max()))


def test_replicated_batch_equals_packed_copies(C):
    """B copies built on the device (mpax_lp_batch_create_replicated) are the
    block-diagonal batch that B host-packed copies give: identical solves in FP64."""
    g = grid_shortest_path_lp(6, B=3, seed=instance_seed(44))
    B, m, n = g["B"], g["m"], g["n"]
    nnz = int(g["row_ptr"][-1])
    rp = np.concatenate([[0], (g["row_ptr"][1:][None, :] + nnz * np.arange(B)[:, None]).ravel()])
    tile = lambda a: np.tile(a, B)  # noqa: E731
    opts = C.mpax_options_default(eps_abs=1e-8, eps_rel=1e-8, iteration_limit=10**6)
    res = []
    hp = C.mpax_lp_batch_create(B, np.arange(B + 1) * m, np.arange(B + 1) * n, rp,
                                tile(g["col"]), tile(g["val"]), g["C"].ravel(), tile(g["lc"]),
                                tile(g["uc"]), tile(g["l"]), tile(g["u"]))
    hr = C.mpax_lp_batch_create_replicated(B, m, n, g["row_ptr"], g["col"], g["val"], g["lc"],
                                           g["uc"], g["l"], g["u"])
    try:
        C.mpax_batch_set_costs(hr, g["C"].ravel())
        for h in (hp, hr):
            C.mpax_batch_solve(h, opts)
            res.append(C.mpax_batch_get_solution(h, B * m, B * n)
                       + (C.mpax_batch_get_objective(h, B),))
    finally:
        C.mpax_batch_destroy(hp)
        C.mpax_batch_destroy(hr)
    for a, b in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, b)
