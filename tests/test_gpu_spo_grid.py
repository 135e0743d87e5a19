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
    from paper_2412_09734_gb300.autograd import SparseLPValues
    g = grid_shortest_path_lp(8, B=6, seed=instance_seed(41))
    Cm = torch.from_numpy(g["C"]).cuda().requires_grad_(True)
    v = SparseLPValues.apply(Cm, g, OPTS)
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
    from paper_2412_09734_gb300.autograd import SparseLPValues, SPOPlusLossSparse
    g = grid_shortest_path_lp(8, B=4, seed=instance_seed(42))
    rng = np.random.default_rng(5)
    Ct = torch.from_numpy(g["C"]).cuda()
    with torch.no_grad():
        zt = SparseLPValues.apply(Ct, g, OPTS)
    # the true optimal flows (GPU), for the GPU loss
    Ctg = Ct.clone().requires_grad_(True)
    SparseLPValues.apply(Ctg, g, OPTS).sum().backward()
    Xt = Ctg.grad.detach()
    Ch_np = g["C"] + rng.normal(0, 0.3, g["C"].shape)
    Ch = torch.from_numpy(Ch_np).cuda().requires_grad_(True)
    loss = SPOPlusLossSparse.apply(Ch, Ct, Xt, zt, g, OPTS)
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
