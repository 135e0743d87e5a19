"""Seeded synthetic LP/QP instances shaped like the paper's workloads.

This module builds problem *data* only (matrices, bound vectors, warm-start
states).  It contains no step of the PDHG method: it is the one module that both
the CUDA path's tests and the oracle's tests import.
"""
from .generators import (  # noqa: F401
    MASTER_SEED,
    instance_seed,
    csr_random,
    lp_instance,
    qp_instance,
    qp_sparse_q_instance,
    ragged_lp_batch,
    ragged_lp_instances,
    shared_dense_lp_batch,
    knapsack_lp,
    grid_shortest_path_lp,
    random_state,
)
