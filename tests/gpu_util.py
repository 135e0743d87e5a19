"""Shared helpers for the GPU tests (library handle from a generator dict)."""
import numpy as np


def lib():
    from paper_2412_09734_gb300 import build
    build.build()
    from paper_2412_09734_gb300 import mpax
    return mpax


def create(C, d, device=False):
    """Library handle for a synth LP/QP dictionary; device=True passes CUDA tensors."""
    conv = (lambda a: a)
    if device:
        import torch
        conv = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda())
    args = [conv(d[k]) for k in ("row_ptr", "col", "val", "c", "lc", "uc", "l", "u")]
    if "q_row_ptr" in d:
        return C.mpax_qp_create(d["m"], d["n"], *args, conv(d["q_row_ptr"]), conv(d["q_col"]),
                                conv(d["q_val"]))
    if "D" in d:
        return C.mpax_qp_create_diag_lowrank(d["m"], d["n"], *args, conv(d["D"]), d["f_cols"],
                                             conv(d["f_row_ptr"]), conv(d["f_col"]),
                                             conv(d["f_val"]))
    return C.mpax_lp_create(d["m"], d["n"], *args)


def rel_inf(a, b):
    """max |a - b| / max(max |b|, tiny): normwise relative error in the inf-norm."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
