"""mpax_lp_kkt_noalloc: the relative KKT evaluation for callers that cannot
allocate device memory.  It must give what mpax_kkt (the handle-based entry
point, whose scratch the library allocates) gives, on two calls in a row that
share the library's static scratch array.

This file is collected last on purpose: a run that stops at the first failure
has already run every other test when it gets here."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

from synth import instance_seed, lp_instance
from tests.gpu_util import create, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


def _device_problem(d):
    import torch
    A = sp.csr_matrix((d["val"], d["col"], d["row_ptr"]), shape=(d["m"], d["n"]))
    At = A.T.tocsr()
    At.sort_indices()
    arrs = dict(row_ptr=d["row_ptr"].astype(np.int64), col=d["col"].astype(np.int32),
                val=d["val"], row_ptr_t=At.indptr.astype(np.int64),
                col_t=At.indices.astype(np.int32), val_t=At.data, c=d["c"], lc=d["lc"],
                uc=d["uc"], l=d["l"], u=d["u"])
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in arrs.items()}


def _noalloc(C, d, dev, x, y):
    import torch
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = C._lib.mpax_lp_kkt_noalloc(
        d["m"], d["n"], int(d["row_ptr"][-1]), dev["row_ptr"].data_ptr(),
        dev["col"].data_ptr(), dev["val"].data_ptr(), dev["row_ptr_t"].data_ptr(),
        dev["col_t"].data_ptr(), dev["val_t"].data_ptr(), dev["c"].data_ptr(),
        dev["lc"].data_ptr(), dev["uc"].data_ptr(), dev["l"].data_ptr(), dev["u"].data_ptr(),
        x.data_ptr(), y.data_ptr(), out.data_ptr(), ctypes.c_void_p(stream))
    assert st == 0, C.mpax_last_error()
    torch.cuda.synchronize()
    keys = ("primal_res", "dual_res", "primal_obj", "dual_obj", "gap", "rel_kkt")
    return dict(zip(keys, out.cpu().numpy().tolist()))


def test_noalloc_kkt_matches_handle_kkt_twice(C):
    import torch
    d = lp_instance(20000, 40000, seed=instance_seed(102), nnz=400000, rows="zipf")
    dev = _device_problem(d)
    h = create(C, d)
    try:
        C.mpax_prepare(h, C.mpax_options_default())
        for seed in (1, 2):  # two calls in a row share the static scratch
            rng = np.random.default_rng(seed)
            x = np.clip(rng.standard_normal(d["n"]) * 4, d["l"], d["u"])
            # y sign-consistent with the row bounds (<= 0 where lc = -inf, >= 0
            # where uc = +inf), the points the solver returns
            y = rng.standard_normal(d["m"]) * seed
            y = np.where(np.isinf(d["uc"]), np.abs(y), y)
            y = np.where(np.isinf(d["lc"]), -np.abs(y), y)
            ref = C.mpax_kkt(h, x, y)
            got = _noalloc(C, d, dev, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
            scale = 1 + abs(ref["primal_obj"]) + abs(ref["dual_obj"])
            for key in ("primal_res", "dual_res", "rel_kkt"):
                assert got[key] == pytest.approx(ref[key], rel=1e-12, abs=1e-15), key
            for key in ("primal_obj", "dual_obj", "gap"):
                assert abs(got[key] - ref[key]) <= 1e-12 * scale, key
    finally:
        C.mpax_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_scratch(C):
    out = ctypes.c_void_p(1)
    st = C._lib.mpax_lp_kkt_noalloc(1 << 25, 4, 0, out, None, None, out, None, None, out, out,
                                    out, out, out, out, out, out, None)
    assert st == 7 and "16777216" in C.mpax_last_error()
