"""Convenience wrapper: one library handle per problem, freed with the object."""
from __future__ import annotations

import numpy as np

from . import mpax as C


class Problem:
    """An LP, or a QP with Q = diag(D) + F F^T (D=, F=) or with a general sparse
    symmetric Q (Q=(q_row_ptr, q_col, q_val), both triangles), owned by the CUDA
    library.

    Arrays may be numpy (host) or CUDA torch tensors (device); they are copied
    into library-owned device memory at construction.
    """

    def __init__(self, m, n, row_ptr, col, val, c, lc, uc, l, u, *, D=None, F=None, Q=None,
                 stream=None):
        self.m, self.n = int(m), int(n)
        self.is_qp = D is not None or Q is not None
        if Q is not None:
            q_row_ptr, q_col, q_val = Q
            self.h = C.mpax_qp_create(self.m, self.n, row_ptr, col, val, c, lc, uc, l, u,
                                      q_row_ptr, q_col, q_val, stream=stream)
        elif self.is_qp:
            f_row_ptr, f_col, f_val, r = F
            self.h = C.mpax_qp_create_diag_lowrank(self.m, self.n, row_ptr, col, val, c, lc, uc,
                                                   l, u, D, int(r), f_row_ptr, f_col, f_val,
                                                   stream=stream)
        else:
            self.h = C.mpax_lp_create(self.m, self.n, row_ptr, col, val, c, lc, uc, l, u,
                                      stream=stream)

    @classmethod
    def from_dict(cls, d, device=None):
        """Build from a dictionary with keys m, n, row_ptr, col, val, c, lc, uc,
        l, u (and D, f_row_ptr, f_col, f_val, f_cols, or q_row_ptr, q_col, q_val
        for a QP)."""
        conv = (lambda a: a) if device is None else (lambda a: _to_device(a, device))
        kw = {}
        if "D" in d:
            kw["D"] = conv(d["D"])
            kw["F"] = (conv(d["f_row_ptr"]), conv(d["f_col"]), conv(d["f_val"]), d["f_cols"])
        elif "q_row_ptr" in d:
            kw["Q"] = (conv(d["q_row_ptr"]), conv(d["q_col"]), conv(d["q_val"]))
        return cls(d["m"], d["n"], conv(d["row_ptr"]), conv(d["col"]), conv(d["val"]),
                   conv(d["c"]), conv(d["lc"]), conv(d["uc"]), conv(d["l"]), conv(d["u"]), **kw)

    def solve(self, x0=None, y0=None, **options):
        opts = C.mpax_options_default(**options)
        C.mpax_solve(self.h, opts, x0, y0)
        return C.mpax_get_stats(self.h)

    def solution(self, device=None):
        return C.mpax_get_solution(self.h, self.m, self.n, device)

    def stats(self):
        return C.mpax_get_stats(self.h)

    def reduced_cost(self, device=None):
        """lam = Q x + c - A^T y at the returned point."""
        return C.mpax_get_reduced_cost(self.h, self.n, device)

    def close(self):
        if getattr(self, "h", None):
            C.mpax_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass


def _to_device(a, device):
    import torch
    if isinstance(a, torch.Tensor):
        return a.to(device)
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)
