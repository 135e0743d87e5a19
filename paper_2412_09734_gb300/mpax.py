"""Thin ctypes binding of libmpax_gb300.so (include/mpax.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Functions keep the C names.  Array arguments may be numpy arrays
(host memory, kind=MPAX_MEM_HOST) or CUDA torch tensors (device memory,
kind=MPAX_MEM_DEVICE); the kind is inferred from the first array argument.
A missing library raises at import of this module: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpax_gb300.so")

MPAX_OK = 0
MPAX_MEM_HOST = 0
MPAX_MEM_DEVICE = 1
MPAX_PREC_FP64 = 0
MPAX_PREC_MIXED = 1
MPAX_ERR_INVALID_ARGUMENT = 1
MPAX_ERR_NOT_SOLVED = 4
MPAX_ERR_UNSUPPORTED = 7
MPAX_TERM_OPTIMAL = 1
TERMINATION = {0: "unsolved", 1: "optimal", 2: "primal_infeasible", 3: "dual_infeasible",
               4: "iteration_limit", 5: "time_limit", 6: "numerical_error"}

EXPORTED = ["mpax_version", "mpax_last_error", "mpax_status_string", "mpax_options_default",
            "mpax_lp_create", "mpax_lp_create_f32", "mpax_qp_create_diag_lowrank",
            "mpax_qp_create", "mpax_get_reduced_cost", "mpax_solve",
            "mpax_get_solution",
            "mpax_get_stats", "mpax_destroy", "mpax_prepare", "mpax_get_scaling",
            "mpax_get_transpose", "mpax_set_iterate", "mpax_iterate", "mpax_get_iterate",
            "mpax_kkt", "mpax_lp_value_grad", "mpax_qp_adjoint", "mpax_qp_unrolled_grad",
            "mpax_lp_batch_create", "mpax_batch_solve", "mpax_batch_get_solution",
            "mpax_batch_get_stats", "mpax_batch_destroy", "mpax_lp_shared_create", "mpax_shared_solve",
            "mpax_shared_get_solution", "mpax_shared_get_stats", "mpax_shared_destroy",
            "mpax_lp_kkt_noalloc", "mpax_get_restart_history",
            "mpax_lp_batch_create_replicated", "mpax_batch_set_costs",
            "mpax_batch_get_objective", "mpax_batch_spo_plus", "mpax_shared_set_costs",
            "mpax_shared_get_objective", "mpax_shared_spo_plus", "mpax_dense_bf16x3"]


class MpaxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mpax status {status}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [
        ("verbose", ctypes.c_int32), ("display_frequency", ctypes.c_int32),
        ("warm_start", ctypes.c_int32), ("feasibility_polishing", ctypes.c_int32),
        ("eps_abs", ctypes.c_double), ("eps_rel", ctypes.c_double),
        ("eps_primal_infeasible", ctypes.c_double), ("eps_dual_infeasible", ctypes.c_double),
        ("eps_feas_polish", ctypes.c_double), ("iteration_limit", ctypes.c_int64),
        ("time_limit", ctypes.c_double),
        ("precision", ctypes.c_int32), ("check_every", ctypes.c_int32),
        ("ruiz_iters", ctypes.c_int32), ("pock_chambolle", ctypes.c_int32),
        ("reflection_gamma", ctypes.c_double), ("restart_sufficient", ctypes.c_double),
        ("restart_necessary", ctypes.c_double), ("restart_artificial", ctypes.c_double),
        ("primal_weight_smoothing", ctypes.c_double), ("step_safety", ctypes.c_double),
        ("power_max_iter", ctypes.c_int32), ("power_tol", ctypes.c_double),
        ("use_graphs", ctypes.c_int32), ("profile_kernels", ctypes.c_int32),
        ("fp64_continuation", ctypes.c_int32), ("stall_checks", ctypes.c_int32),
        ("record_tape", ctypes.c_int32), ("spmv_kernel", ctypes.c_int32),
        ("batch_stage", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("termination", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("iterations", ctypes.c_int64), ("restarts", ctypes.c_int64),
        ("kkt_checks", ctypes.c_int64),
        ("primal_obj", ctypes.c_double), ("dual_obj", ctypes.c_double), ("gap", ctypes.c_double),
        ("primal_res", ctypes.c_double), ("dual_res", ctypes.c_double),
        ("rel_kkt", ctypes.c_double),
        ("omega", ctypes.c_double), ("eta", ctypes.c_double), ("norm_A", ctypes.c_double),
        ("norm_Q", ctypes.c_double),
        ("prepare_seconds", ctypes.c_double), ("solve_seconds", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64),
        ("profile_ms", ctypes.c_double * 4), ("profile_launches", ctypes.c_int64 * 4),
        ("fp64_iterations", ctypes.c_int64), ("polish_iterations", ctypes.c_int64),
        ("backward_launches", ctypes.c_int64),
        ("spmv_kernel", ctypes.c_int32 * 2), ("spmv_tune_us", ctypes.c_double * 6),
        ("profile_ms_aux", ctypes.c_double), ("profile_launches_aux", ctypes.c_int64),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        d["termination_name"] = TERMINATION.get(self.termination, "?")
        return d


class BatchStats(ctypes.Structure):
    _fields_ = [
        ("B", ctypes.c_int32), ("n_optimal", ctypes.c_int32),
        ("iterations_total", ctypes.c_int64), ("iterations_max", ctypes.c_int64),
        ("restarts_total", ctypes.c_int64), ("rel_kkt_max", ctypes.c_double),
        ("instance_seconds_p50", ctypes.c_double), ("instance_seconds_p99", ctypes.c_double),
        ("instance_seconds_max", ctypes.c_double), ("solve_seconds", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64), ("fp64_instances", ctypes.c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is not built; run `python -m paper_2412_09734_gb300.build` "
        "(or __graft_entry__.build()) first")

_lib = ctypes.CDLL(LIB_PATH)
_P = ctypes.c_void_p
_I32, _I64, _D, _INT = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_int
_sig = {
    "mpax_version": ([], ctypes.c_char_p),
    "mpax_last_error": ([], ctypes.c_char_p),
    "mpax_status_string": ([_INT], ctypes.c_char_p),
    "mpax_options_default": ([ctypes.POINTER(Options)], None),
    "mpax_lp_create": ([_I32, _I32, _I64] + [_P] * 8 + [_INT, _P, ctypes.POINTER(_P)], _INT),
    "mpax_qp_create_diag_lowrank": ([_I32, _I32, _I64] + [_P] * 9 + [_I32, _I64, _P, _P, _P,
                                                                       _INT, _P,
                                                                       ctypes.POINTER(_P)],
                                    _INT),
    "mpax_lp_create_f32": ([_I32, _I32, _I64] + [_P] * 8 + [_INT, _P, ctypes.POINTER(_P)],
                           _INT),
    "mpax_get_reduced_cost": ([_P, _P, _INT], _INT),
    "mpax_qp_create": ([_I32, _I32, _I64] + [_P] * 8 + [_I64, _P, _P, _P, _INT, _P,
                                                          ctypes.POINTER(_P)], _INT),
    "mpax_solve": ([_P, ctypes.POINTER(Options), _P, _P, _INT], _INT),
    "mpax_get_solution": ([_P, _P, _P, _INT], _INT),
    "mpax_get_stats": ([_P, ctypes.POINTER(Stats)], _INT),
    "mpax_get_restart_history": ([_P, ctypes.c_int32, _P, _P, _P], _INT),
    "mpax_destroy": ([_P], None),
    "mpax_prepare": ([_P, ctypes.POINTER(Options)], _INT),
    "mpax_get_scaling": ([_P, _P, _P, _P, _INT], _INT),
    "mpax_get_transpose": ([_P, _P, _P, _P, _INT], _INT),
    "mpax_set_iterate": ([_P, _P, _P, _P, _P, _I64, _D, _D, _INT], _INT),
    "mpax_iterate": ([_P, _I64], _INT),
    "mpax_get_iterate": ([_P, _P, _P, _P, _P, _INT], _INT),
    "mpax_kkt": ([_P, _P, _P, _INT, _P], _INT),
    "mpax_lp_kkt_noalloc": ([_I32, _I32, _I64] + [_P] * 15, _INT),
    "mpax_lp_value_grad": ([_P, _P, _P, _P, _P, _P, _INT], _INT),
    "mpax_qp_adjoint": ([_P, _P, _P, _P, _P, _D, _I32, _INT, _P], _INT),
    "mpax_qp_unrolled_grad": ([_P] * 9 + [_INT], _INT),
    "mpax_lp_batch_create": ([_I32] + [_P] * 10 + [_INT, _P, ctypes.POINTER(_P)], _INT),
    "mpax_batch_solve": ([_P, ctypes.POINTER(Options)], _INT),
    "mpax_batch_get_solution": ([_P, _P, _P, _INT], _INT),
    "mpax_batch_get_stats": ([_P, ctypes.POINTER(BatchStats), _P, _P, _P, _P, _P], _INT),
    "mpax_batch_destroy": ([_P], None),
    "mpax_lp_shared_create": ([_I32, _I32, _I32] + [_P] * 6 + [_INT, _P, ctypes.POINTER(_P)],
                              _INT),
    "mpax_shared_solve": ([_P, ctypes.POINTER(Options), _I32], _INT),
    "mpax_shared_get_solution": ([_P, _P, _P, _INT], _INT),
    "mpax_shared_get_stats": ([_P, ctypes.POINTER(BatchStats)] + [_P] * 6, _INT),
    "mpax_shared_destroy": ([_P], None),
    "mpax_lp_batch_create_replicated": ([_I32, _I32, _I32, _I64] + [_P] * 7 +
                                        [_INT, _P, ctypes.POINTER(_P)], _INT),
    "mpax_batch_set_costs": ([_P, _P, _INT], _INT),
    "mpax_batch_get_objective": ([_P, _P, _INT], _INT),
    "mpax_batch_spo_plus": ([_P, ctypes.POINTER(Options)] + [_P] * 6 + [_INT], _INT),
    "mpax_shared_set_costs": ([_P, _P, _INT], _INT),
    "mpax_shared_get_objective": ([_P, _P, _INT], _INT),
    "mpax_shared_spo_plus": ([_P, ctypes.POINTER(Options), _I32] + [_P] * 6 + [_INT], _INT),
    "mpax_dense_bf16x3": ([_I32, _I32, _I32, _I32, _I32, _P, _P, _P, _INT, _P], _INT),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def _check(status):
    if status != MPAX_OK:
        raise MpaxError(status, _lib.mpax_last_error().decode())


# ---------------------------------------------------------------------------
# marshalling
# ---------------------------------------------------------------------------

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _kind_of(*arrays):
    for a in arrays:
        if a is None:
            continue
        if _is_torch(a):
            return MPAX_MEM_DEVICE if a.is_cuda else MPAX_MEM_HOST
        return MPAX_MEM_HOST
    return MPAX_MEM_HOST


class _Keep:
    """Holds converted arrays alive for the duration of a call."""

    def __init__(self, kind):
        self.kind = kind
        self.refs = []

    def ptr(self, a, dtype):
        if a is None:
            return None
        if _is_torch(a):
            import torch
            tdt = {np.float64: torch.float64, np.float32: torch.float32, np.int64: torch.int64,
                   np.int32: torch.int32}[dtype]
            if self.kind == MPAX_MEM_DEVICE and not a.is_cuda:
                raise ValueError("mixed host/device arguments")
            if self.kind == MPAX_MEM_HOST and a.is_cuda:
                raise ValueError("mixed host/device arguments")
            t = a.to(tdt).contiguous()
            self.refs.append(t)
            return t.data_ptr() if t.numel() else None
        if self.kind == MPAX_MEM_DEVICE:
            raise ValueError("mixed host/device arguments")
        arr = np.ascontiguousarray(a, dtype=dtype)
        self.refs.append(arr)
        return arr.ctypes.data if arr.size else None


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover
        pass
    return None


# ---------------------------------------------------------------------------
# C names
# ---------------------------------------------------------------------------

def mpax_version():
    return _lib.mpax_version().decode()


def mpax_last_error():
    return _lib.mpax_last_error().decode()


def mpax_options_default(**overrides):
    o = Options()
    _lib.mpax_options_default(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def mpax_lp_create(m, n, row_ptr, col_idx, val, c, lc, uc, l, u, stream=None):
    kind = _kind_of(row_ptr, val)
    k = _Keep(kind)
    nnz = int(len(val)) if not _is_torch(val) else int(val.numel())
    h = _P()
    _check(_lib.mpax_lp_create(m, n, nnz, k.ptr(row_ptr, np.int64), k.ptr(col_idx, np.int32),
                               k.ptr(val, np.float64), k.ptr(c, np.float64),
                               k.ptr(lc, np.float64), k.ptr(uc, np.float64),
                               k.ptr(l, np.float64), k.ptr(u, np.float64), kind,
                               _stream(stream), ctypes.byref(h)))
    return h


def mpax_qp_create_diag_lowrank(m, n, row_ptr, col_idx, val, c, lc, uc, l, u, D, r,
                                f_row_ptr, f_col_idx, f_val, stream=None):
    kind = _kind_of(row_ptr, val)
    k = _Keep(kind)
    nnz = int(len(val)) if not _is_torch(val) else int(val.numel())
    f_nnz = int(len(f_val)) if not _is_torch(f_val) else int(f_val.numel())
    h = _P()
    _check(_lib.mpax_qp_create_diag_lowrank(
        m, n, nnz, k.ptr(row_ptr, np.int64), k.ptr(col_idx, np.int32), k.ptr(val, np.float64),
        k.ptr(c, np.float64), k.ptr(lc, np.float64), k.ptr(uc, np.float64),
        k.ptr(l, np.float64), k.ptr(u, np.float64), k.ptr(D, np.float64), r, f_nnz,
        k.ptr(f_row_ptr, np.int64), k.ptr(f_col_idx, np.int32), k.ptr(f_val, np.float64),
        kind, _stream(stream), ctypes.byref(h)))
    return h


def mpax_lp_create_f32(m, n, row_ptr, col_idx, val, c, lc, uc, l, u, stream=None):
    """mpax_lp_create with FP32 values and vectors (widened to FP64 on entry)."""
    kind = _kind_of(row_ptr, val)
    k = _Keep(kind)
    nnz = int(len(val)) if not _is_torch(val) else int(val.numel())
    h = _P()
    _check(_lib.mpax_lp_create_f32(
        m, n, nnz, k.ptr(row_ptr, np.int64), k.ptr(col_idx, np.int32), k.ptr(val, np.float32),
        k.ptr(c, np.float32), k.ptr(lc, np.float32), k.ptr(uc, np.float32),
        k.ptr(l, np.float32), k.ptr(u, np.float32), kind, _stream(stream), ctypes.byref(h)))
    return h


def mpax_get_reduced_cost(h, n, device=None):
    """lam = Q x + c - A^T y at the returned point (unscaled)."""
    lam, kind = _out(n, device)
    _check(_lib.mpax_get_reduced_cost(h, _ptr_out(lam), kind))
    return lam


def mpax_qp_create(m, n, row_ptr, col_idx, val, c, lc, uc, l, u, q_row_ptr, q_col_idx, q_val,
                   stream=None):
    """QP with a general sparse symmetric PSD Q (CSR, both triangles stored)."""
    kind = _kind_of(row_ptr, val)
    k = _Keep(kind)
    nnz = int(len(val)) if not _is_torch(val) else int(val.numel())
    q_nnz = int(len(q_val)) if not _is_torch(q_val) else int(q_val.numel())
    h = _P()
    _check(_lib.mpax_qp_create(
        m, n, nnz, k.ptr(row_ptr, np.int64), k.ptr(col_idx, np.int32), k.ptr(val, np.float64),
        k.ptr(c, np.float64), k.ptr(lc, np.float64), k.ptr(uc, np.float64),
        k.ptr(l, np.float64), k.ptr(u, np.float64), q_nnz, k.ptr(q_row_ptr, np.int64),
        k.ptr(q_col_idx, np.int32), k.ptr(q_val, np.float64), kind, _stream(stream),
        ctypes.byref(h)))
    return h


def mpax_solve(h, opts, x0=None, y0=None):
    kind = _kind_of(x0, y0)
    k = _Keep(kind)
    _check(_lib.mpax_solve(h, ctypes.byref(opts), k.ptr(x0, np.float64),
                           k.ptr(y0, np.float64), kind))


def mpax_prepare(h, opts):
    _check(_lib.mpax_prepare(h, ctypes.byref(opts)))


def _out(n, like):
    if like is not None and _is_torch(like) and like.is_cuda:
        import torch
        return torch.empty(n, dtype=torch.float64, device=like.device), MPAX_MEM_DEVICE
    return np.empty(n, dtype=np.float64), MPAX_MEM_HOST


def _ptr_out(a):
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr() if a.numel() else None
    return a.ctypes.data if a.size else None


def mpax_get_solution(h, m, n, device=None):
    """Returns (x, y) as numpy arrays, or CUDA tensors when `device` is a CUDA
    tensor used as a template."""
    x, kind = _out(n, device)
    y, _ = _out(m, device)
    _check(_lib.mpax_get_solution(h, _ptr_out(x), _ptr_out(y), kind))
    return x, y


def mpax_get_stats(h):
    s = Stats()
    _check(_lib.mpax_get_stats(h, ctypes.byref(s)))
    return s.as_dict()


def mpax_get_restart_history(h, cap=256):
    """(iterations at each restart, primal weight after it) of the last run."""
    it = np.zeros(cap, dtype=np.int64)
    om = np.zeros(cap, dtype=np.float64)
    cnt = ctypes.c_int32(0)
    _check(_lib.mpax_get_restart_history(h, cap, it.ctypes.data_as(ctypes.c_void_p),
                                         om.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)))
    k = min(cnt.value, cap)
    return it[:k].copy(), om[:k].copy(), cnt.value


def mpax_destroy(h):
    if h:
        _lib.mpax_destroy(h)


def mpax_get_scaling(h, m, n):
    Dr = np.empty(m)
    Dc = np.empty(n)
    info = np.empty(4)
    _check(_lib.mpax_get_scaling(h, _ptr_out(Dr), _ptr_out(Dc), info.ctypes.data,
                                 MPAX_MEM_HOST))
    return Dr, Dc, dict(norm_A=info[0], norm_Q=info[1], eta=info[2], omega=info[3])


def mpax_get_transpose(h, n, nnz):
    rp = np.empty(n + 1, dtype=np.int64)
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz)
    _check(_lib.mpax_get_transpose(h, rp.ctypes.data, _ptr_out(col), _ptr_out(val),
                                   MPAX_MEM_HOST))
    return rp, col, val


def mpax_set_iterate(h, x, y, x_aux, y_aux, k, tau, sigma):
    kind = _kind_of(x, y)
    kp = _Keep(kind)
    _check(_lib.mpax_set_iterate(h, kp.ptr(x, np.float64), kp.ptr(y, np.float64),
                                 kp.ptr(x_aux, np.float64), kp.ptr(y_aux, np.float64), int(k),
                                 float(tau), float(sigma), kind))


def mpax_iterate(h, iters):
    _check(_lib.mpax_iterate(h, int(iters)))


def mpax_get_iterate(h, m, n):
    x, y, xh, yh = np.empty(n), np.empty(m), np.empty(n), np.empty(m)
    _check(_lib.mpax_get_iterate(h, _ptr_out(x), _ptr_out(y), _ptr_out(xh), _ptr_out(yh),
                                 MPAX_MEM_HOST))
    return x, y, xh, yh


def mpax_kkt(h, x, y):
    kind = _kind_of(x, y)
    kp = _Keep(kind)
    out = np.empty(6)
    if kind == MPAX_MEM_DEVICE:
        import torch
        dout = torch.empty(6, dtype=torch.float64, device=x.device)
        _check(_lib.mpax_kkt(h, kp.ptr(x, np.float64), kp.ptr(y, np.float64), kind,
                             dout.data_ptr()))
        out = dout.cpu().numpy()
    else:
        _check(_lib.mpax_kkt(h, kp.ptr(x, np.float64), kp.ptr(y, np.float64), kind,
                             out.ctypes.data))
    keys = ("primal_res", "dual_res", "primal_obj", "dual_obj", "gap", "rel_kkt")
    return dict(zip(keys, out.tolist()))


# ---------------------------------------------------------------------------
# ragged batch
# ---------------------------------------------------------------------------

def mpax_lp_batch_create(B, m_off, n_off, row_ptr, col_idx, val, c, lc, uc, l, u, stream=None):
    kind = _kind_of(row_ptr, val)
    k = _Keep(kind)
    h = _P()
    # offsets are read on the host side of the call in either memory kind
    _check(_lib.mpax_lp_batch_create(
        int(B), k.ptr(m_off, np.int64), k.ptr(n_off, np.int64), k.ptr(row_ptr, np.int64),
        k.ptr(col_idx, np.int32), k.ptr(val, np.float64), k.ptr(c, np.float64),
        k.ptr(lc, np.float64), k.ptr(uc, np.float64), k.ptr(l, np.float64),
        k.ptr(u, np.float64), kind, _stream(stream), ctypes.byref(h)))
    return h


def mpax_batch_solve(h, opts):
    _check(_lib.mpax_batch_solve(h, ctypes.byref(opts)))


def _out_buf(shape, device):
    """An FP64 output buffer: a CUDA tensor on `device`'s device when `device` is a
    CUDA tensor, else a numpy array; with its pointer and memory kind."""
    if device is not None and _is_torch(device) and device.is_cuda:
        import torch
        t = torch.empty(shape, dtype=torch.float64, device=device.device)
        return t, (t.data_ptr() if t.numel() else None), MPAX_MEM_DEVICE
    a = np.empty(shape)
    return a, (a.ctypes.data if a.size else None), MPAX_MEM_HOST


def mpax_batch_get_solution(h, m_total, n_total, device=None):
    x, px, kind = _out_buf(n_total, device)
    y, py, _ = _out_buf(m_total, device)
    _check(_lib.mpax_batch_get_solution(h, px, py, kind))
    return x, y


def mpax_lp_batch_create_replicated(B, m, n, row_ptr, col_idx, val, lc, uc, l, u, stream=None):
    kind = _kind_of(row_ptr, val)
    k = _Keep(kind)
    nnz = int(len(val)) if not _is_torch(val) else int(val.numel())
    h = _P()
    _check(_lib.mpax_lp_batch_create_replicated(
        int(B), int(m), int(n), nnz, k.ptr(row_ptr, np.int64), k.ptr(col_idx, np.int32),
        k.ptr(val, np.float64), k.ptr(lc, np.float64), k.ptr(uc, np.float64),
        k.ptr(l, np.float64), k.ptr(u, np.float64), kind, _stream(stream), ctypes.byref(h)))
    return h


def mpax_batch_set_costs(h, c):
    kind = _kind_of(c)
    k = _Keep(kind)
    _check(_lib.mpax_batch_set_costs(h, k.ptr(c, np.float64), kind))


def mpax_batch_get_objective(h, B, device=None):
    v, pv, kind = _out_buf(B, device)
    _check(_lib.mpax_batch_get_objective(h, pv, kind))
    return v


def mpax_batch_spo_plus(h, opts, c_hat, c_true, x_true, z_true):
    """(loss (B,), grad (like c_hat)) of SPO+; CUDA tensors in give CUDA tensors out."""
    kind = _kind_of(c_hat)
    k = _Keep(kind)
    B = int(len(z_true)) if not _is_torch(z_true) else int(z_true.numel())
    total = int(np.prod(c_hat.shape))
    loss, pl, _ = _out_buf(B, c_hat if kind == MPAX_MEM_DEVICE else None)
    grad, pg, _ = _out_buf(tuple(c_hat.shape), c_hat if kind == MPAX_MEM_DEVICE else None)
    assert total == (grad.numel() if _is_torch(grad) else grad.size)
    _check(_lib.mpax_batch_spo_plus(h, ctypes.byref(opts), k.ptr(c_hat, np.float64),
                                    k.ptr(c_true, np.float64), k.ptr(x_true, np.float64),
                                    k.ptr(z_true, np.float64), pl, pg, kind))
    return loss, grad


def mpax_batch_get_stats(h, B):
    s = BatchStats()
    st = np.empty(B, dtype=np.int32)
    it = np.empty(B, dtype=np.int64)
    kk = np.empty(B)
    po = np.empty(B)
    sec = np.empty(B)
    _check(_lib.mpax_batch_get_stats(h, ctypes.byref(s), st.ctypes.data, it.ctypes.data,
                                     kk.ctypes.data, po.ctypes.data, sec.ctypes.data))
    return s.as_dict(), dict(status=st, iterations=it, rel_kkt=kk, primal_obj=po, seconds=sec)


def mpax_batch_destroy(h):
    if h:
        _lib.mpax_batch_destroy(h)


# ---------------------------------------------------------------------------
# differentiation
# ---------------------------------------------------------------------------

def mpax_lp_value_grad(h, m, n, device=None):
    """Returns dict(c, lc, uc, l, u) of optimal-value gradients."""
    outs = {k: _out(sz, device)[0] for k, sz in (("c", n), ("lc", m), ("uc", m), ("l", n),
                                                 ("u", n))}
    kind = MPAX_MEM_DEVICE if (device is not None and _is_torch(device) and device.is_cuda) \
        else MPAX_MEM_HOST
    _check(_lib.mpax_lp_value_grad(h, _ptr_out(outs["c"]), _ptr_out(outs["lc"]),
                                   _ptr_out(outs["uc"]), _ptr_out(outs["l"]),
                                   _ptr_out(outs["u"]), kind))
    return outs


def mpax_qp_adjoint(h, g, m, n, tol=1e-10, max_iter=10000):
    """Returns (dc, db, dD, info) for the loss gradient g = dL/dx*."""
    kind = _kind_of(g)
    kp = _Keep(kind)
    gp = kp.ptr(g, np.float64)
    dc, _ = _out(n, g if kind == MPAX_MEM_DEVICE else None)
    db, _ = _out(m, g if kind == MPAX_MEM_DEVICE else None)
    dD, _ = _out(n, g if kind == MPAX_MEM_DEVICE else None)
    info = np.zeros(2)
    _check(_lib.mpax_qp_adjoint(h, gp, _ptr_out(dc), _ptr_out(db), _ptr_out(dD), float(tol),
                                int(max_iter), kind, info.ctypes.data))
    return dc, db, dD, dict(iterations=int(info[0]), rel_residual=float(info[1]))


def mpax_qp_unrolled_grad(h, gx, m, n, gy=None):
    """Gradients of L = gx . x + gy . y along the path of the last solve, which
    ran with record_tape = 1: dict(c, lc, uc, l, u, D); CUDA tensors when gx is
    one, else numpy arrays."""
    kind = _kind_of(gx)
    kp = _Keep(kind)
    gxp = kp.ptr(gx, np.float64)
    gyp = kp.ptr(gy, np.float64) if gy is not None else None
    tmpl = gx if kind == MPAX_MEM_DEVICE else None
    outs = {k: _out(sz, tmpl)[0] for k, sz in (("c", n), ("lc", m), ("uc", m), ("l", n),
                                               ("u", n), ("D", n))}
    _check(_lib.mpax_qp_unrolled_grad(h, gxp, gyp, _ptr_out(outs["c"]), _ptr_out(outs["lc"]),
                                      _ptr_out(outs["uc"]), _ptr_out(outs["l"]),
                                      _ptr_out(outs["u"]), _ptr_out(outs["D"]), kind))
    return outs


# ---------------------------------------------------------------------------
# shared dense matrix batch
# ---------------------------------------------------------------------------

def mpax_lp_shared_create(m, n, B, A, C, lc, uc, l, u, stream=None):
    kind = _kind_of(A, C)
    k = _Keep(kind)
    if _is_torch(A):
        import torch
        Ap = A.to(torch.float32).contiguous()
        k.refs.append(Ap)
        a_ptr = Ap.data_ptr()
    else:
        Ap = np.ascontiguousarray(A, dtype=np.float32)
        k.refs.append(Ap)
        a_ptr = Ap.ctypes.data
    h = _P()
    _check(_lib.mpax_lp_shared_create(int(m), int(n), int(B), a_ptr, k.ptr(C, np.float64),
                                      k.ptr(lc, np.float64), k.ptr(uc, np.float64),
                                      k.ptr(l, np.float64), k.ptr(u, np.float64), kind,
                                      _stream(stream), ctypes.byref(h)))
    return h


def mpax_shared_solve(h, opts, fp32_products=False):
    _check(_lib.mpax_shared_solve(h, ctypes.byref(opts), 1 if fp32_products else 0))


def mpax_shared_set_costs(h, C):
    kind = _kind_of(C)
    k = _Keep(kind)
    _check(_lib.mpax_shared_set_costs(h, k.ptr(C, np.float64), kind))


def mpax_shared_get_objective(h, B, device=None):
    v, pv, kind = _out_buf(B, device)
    _check(_lib.mpax_shared_get_objective(h, pv, kind))
    return v


def mpax_shared_spo_plus(h, opts, C_hat, C_true, X_true, z_true, fp32_products=False):
    """(loss (B,), grad (B, n)) of SPO+ over the shared set; CUDA in, CUDA out."""
    kind = _kind_of(C_hat)
    k = _Keep(kind)
    B = int(C_hat.shape[0])
    loss, pl, _ = _out_buf(B, C_hat if kind == MPAX_MEM_DEVICE else None)
    grad, pg, _ = _out_buf(tuple(C_hat.shape), C_hat if kind == MPAX_MEM_DEVICE else None)
    _check(_lib.mpax_shared_spo_plus(h, ctypes.byref(opts), 1 if fp32_products else 0,
                                     k.ptr(C_hat, np.float64), k.ptr(C_true, np.float64),
                                     k.ptr(X_true, np.float64), k.ptr(z_true, np.float64),
                                     pl, pg, kind))
    return loss, grad


def mpax_shared_get_solution(h, m, n, B, device=None):
    """Returns (X, Y) as (B, n) and (B, m) FP64 arrays; CUDA tensors when `device`
    is a CUDA tensor used as a template."""
    if device is not None and _is_torch(device) and device.is_cuda:
        import torch
        X = torch.empty((B, n), dtype=torch.float64, device=device.device)
        Y = torch.empty((B, m), dtype=torch.float64, device=device.device)
        _check(_lib.mpax_shared_get_solution(h, X.data_ptr(), Y.data_ptr(), MPAX_MEM_DEVICE))
        return X, Y
    X = np.empty((B, n))
    Y = np.empty((B, m))
    _check(_lib.mpax_shared_get_solution(h, X.ctypes.data, Y.ctypes.data, MPAX_MEM_HOST))
    return X, Y


def mpax_shared_get_stats(h, B):
    s = BatchStats()
    st = np.empty(B, dtype=np.int32)
    it = np.empty(B, dtype=np.int64)
    kk = np.empty(B)
    po = np.empty(B)
    sec = np.empty(B)
    gi = np.zeros(9)
    _check(_lib.mpax_shared_get_stats(h, ctypes.byref(s), st.ctypes.data, it.ctypes.data,
                                      kk.ctypes.data, po.ctypes.data, sec.ctypes.data,
                                      gi.ctypes.data))
    d = s.as_dict()
    d.update(gemms=int(gi[0]), gemm_flops=float(gi[1]), norm_A=float(gi[2]),
             product_tile_k=(int(gi[3]), int(gi[4])),
             product_ms=(float(gi[5]), float(gi[6])), prepare_s=float(gi[7]),
             power_rounds=int(gi[8]))
    return d, dict(status=st, iterations=it, rel_kkt=kk, primal_obj=po, seconds=sec)


def mpax_shared_destroy(h):
    if h:
        _lib.mpax_shared_destroy(h)


# ---------------------------------------------------------------------------
# dense products of the shared-matrix batch
# ---------------------------------------------------------------------------

def mpax_dense_bf16x3(A, V, a_mn_major=False, tile_k=0, stream=None):
    """D (N x M) = rows of A_op V^T on the tensor cores (BF16x3); A is [M][K]
    (or [K][M] with a_mn_major), V is [N][K]; tile_k 0 / 32 / 64 picks the
    kernel's K block.  CUDA tensors in, CUDA tensor out."""
    kind = _kind_of(A, V)
    if a_mn_major:
        K, M = int(A.shape[0]), int(A.shape[1])
    else:
        M, K = int(A.shape[0]), int(A.shape[1])
    N = int(V.shape[0])
    k = _Keep(kind)
    pa, pv = k.ptr(A, np.float32), k.ptr(V, np.float32)
    if kind == MPAX_MEM_DEVICE:
        import torch
        D = torch.empty((N, M), dtype=torch.float32, device=A.device)
        pd = D.data_ptr()
    else:
        D = np.empty((N, M), dtype=np.float32)
        pd = D.ctypes.data
    _check(_lib.mpax_dense_bf16x3(M, N, K, 1 if a_mn_major else 0, int(tile_k), pa, pv, pd,
                                  kind, _stream(stream)))
    return D
