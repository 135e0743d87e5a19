"""torch.autograd layers over the C ABI (marshalling only; the solve and the
adjoint run in the library's kernels).

QPLayer: x* = argmin 1/2 x^T (diag(D) + F F^T) x + c^T x  s.t.  A x = b, l <= x <= u,
         differentiable in (c, b, D) through the implicit adjoint on the active set.
QPUnrolledLayer: the same solution map differentiated through the solver's
         iterations (the paper's QP gradients): the solve records its path and the
         backward runs the path in reverse.
LPValue: v = min c^T x  s.t.  lc <= A x <= uc, l <= x <= u, differentiable in
         (c, lc, uc) through the envelope theorem (dv/dc = x*, ...).
SharedLPValues: v_k = min c_k^T x  s.t.  lc <= A x <= uc, l <= x <= u for the B rows
         c_k of C with one dense A shared by the batch (a SharedFeasibleSet, on the
         device once); dv_k/dc_k = x_k*.
SPOPlusLoss: the SPO+ surrogate loss of predicted costs c^_k against true costs c_k
         over the same shared feasible set, with subgradient 2 (x*(c_k) - x~_k),
         x~_k = argmin (2 c^_k - c_k)^T x: one library call per forward forms the
         costs, solves the batch and returns the losses and subgradients.
SparseLPValues, SPOPlusLossSparse: the same two layers over one SPARSE feasible set
         (a SparseFeasibleSet: B copies of the set in one ragged batch, built on the
         device once; for example the grid shortest-path LP of the paper's Warcraft
         experiment).
Every layer passes CUDA tensors to the library and gets CUDA tensors back.
"""
from __future__ import annotations

import torch

from . import mpax as C


def _f64(t):
    return t.detach().to(torch.float64).contiguous()


class _Handle:
    """Owns a solved library handle for the backward pass and frees it when
    dropped: after backward, or with the graph (or the context, under no_grad)
    when no backward comes."""

    def __init__(self, h):
        self.h = h

    def close(self):
        h, self.h = self.h, None
        if h:
            C.mpax_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass


def _keep_if_needed(ctx, h):
    """The solved handle wrapped for the backward pass when one of (c, b, D)
    needs a gradient; otherwise freed at once and None."""
    if any(ctx.needs_input_grad[:3]):
        return _Handle(h)
    C.mpax_destroy(h)
    return None


def _require_handle(ctx):
    """The solve behind this node is freed by its first backward (its device
    memory is the size of the problem); a second backward through the same graph
    (retain_graph=True) has nothing left to differentiate."""
    if ctx.h is None or ctx.h.h is None:
        raise RuntimeError("the QP solve of this node was freed by an earlier backward; "
                           "run the forward again to differentiate it again")


class QPLayer(torch.autograd.Function):
    """forward(c, b, D, data, options) -> x*.

    `data` holds the fixed parts as CUDA tensors: m, n, row_ptr, col, val, l, u,
    f_row_ptr, f_col, f_val, r.  `options` are mpax_options fields."""

    @staticmethod
    def forward(ctx, c, b, D, data, options):
        d = data
        h = C.mpax_qp_create_diag_lowrank(
            d["m"], d["n"], d["row_ptr"], d["col"], d["val"], _f64(c), _f64(b), _f64(b),
            d["l"], d["u"], _f64(D), d["r"], d["f_row_ptr"], d["f_col"], d["f_val"])
        try:
            C.mpax_solve(h, C.mpax_options_default(**(options or {})))
            x, _ = C.mpax_get_solution(h, d["m"], d["n"], device=c)
        except Exception:
            C.mpax_destroy(h)
            raise
        ctx.m, ctx.n = d["m"], d["n"]
        ctx.h = _keep_if_needed(ctx, h)
        return x.to(c.dtype)

    @staticmethod
    def backward(ctx, gx):
        _require_handle(ctx)
        try:
            dc, db, dD, _ = C.mpax_qp_adjoint(ctx.h.h, _f64(gx), ctx.m, ctx.n)
        finally:
            ctx.h.close()
        return dc.to(gx.dtype), db.to(gx.dtype), dD.to(gx.dtype), None, None


class QPUnrolledLayer(torch.autograd.Function):
    """forward(c, b, D, data, options) -> x*, as QPLayer, in FP64 with the path
    recorded (record_tape); backward: gradients of the returned point along that
    path (restarts, step sizes and stopping point held fixed), which tend to
    QPLayer's as the solve converges.  Costs about two forward solves."""

    @staticmethod
    def forward(ctx, c, b, D, data, options):
        d = data
        opts = dict(options or {})
        opts.update(record_tape=1, precision=C.MPAX_PREC_FP64)
        h = C.mpax_qp_create_diag_lowrank(
            d["m"], d["n"], d["row_ptr"], d["col"], d["val"], _f64(c), _f64(b), _f64(b),
            d["l"], d["u"], _f64(D), d["r"], d["f_row_ptr"], d["f_col"], d["f_val"])
        try:
            C.mpax_solve(h, C.mpax_options_default(**opts))
            x, _ = C.mpax_get_solution(h, d["m"], d["n"], device=c)
        except Exception:
            C.mpax_destroy(h)
            raise
        ctx.m, ctx.n = d["m"], d["n"]
        ctx.h = _keep_if_needed(ctx, h)
        return x.to(c.dtype)

    @staticmethod
    def backward(ctx, gx):
        _require_handle(ctx)
        try:
            g = C.mpax_qp_unrolled_grad(ctx.h.h, _f64(gx), ctx.m, ctx.n)
        finally:
            ctx.h.close()
        db = g["lc"] + g["uc"]
        return g["c"].to(gx.dtype), db.to(gx.dtype), g["D"].to(gx.dtype), None, None


class LPValue(torch.autograd.Function):
    """forward(c, lc, uc, data, options) -> optimal value (0-dim tensor).

    `data` holds m, n, row_ptr, col, val, l, u as CUDA tensors."""

    @staticmethod
    def forward(ctx, c, lc, uc, data, options):
        d = data
        h = C.mpax_lp_create(d["m"], d["n"], d["row_ptr"], d["col"], d["val"], _f64(c),
                             _f64(lc), _f64(uc), d["l"], d["u"])
        try:
            C.mpax_solve(h, C.mpax_options_default(**(options or {})))
            stats = C.mpax_get_stats(h)
            g = C.mpax_lp_value_grad(h, d["m"], d["n"], device=c)
        finally:
            C.mpax_destroy(h)
        ctx.save_for_backward(g["c"], g["lc"], g["uc"])
        return torch.tensor(stats["primal_obj"], dtype=c.dtype, device=c.device)

    @staticmethod
    def backward(ctx, gv):
        dc, dlc, duc = ctx.saved_tensors
        return (gv * dc).to(gv.dtype), (gv * dlc).to(gv.dtype), (gv * duc).to(gv.dtype), None, None


class SharedFeasibleSet:
    """{x : lc <= A x <= uc, l <= x <= u} with one dense A (m x n, FP32), held by
    the library as a shared-matrix batch of B instances (A copied to the device
    once), for layers that solve B cost vectors over it at every forward."""

    def __init__(self, A, lc, uc, l, u, B):
        self.m, self.n = int(A.shape[0]), int(A.shape[1])
        self.B = int(B)
        zero = torch.zeros((self.B, self.n), dtype=torch.float64,
                           device=A.device if torch.is_tensor(A) else "cpu")
        self.h = C.mpax_lp_shared_create(self.m, self.n, self.B, A.detach() if torch.is_tensor(A)
                                         else A, zero, _f64(lc), _f64(uc), _f64(l), _f64(u))

    def close(self):
        h, self.h = self.h, None
        if h:
            C.mpax_shared_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass


class SparseFeasibleSet:
    """{x : lc <= A x <= uc, l <= x <= u} with a sparse A, held by the library as
    B copies in one ragged batch built on the device once (for example the grid
    shortest-path LP of the paper's Warcraft experiment), for layers that solve B
    cost vectors over it at every forward.  `data` holds m, n, row_ptr, col, val,
    lc, uc, l, u (numpy arrays or CUDA tensors)."""

    def __init__(self, data, B):
        d = data
        self.m, self.n, self.B = int(d["m"]), int(d["n"]), int(B)
        self.h = C.mpax_lp_batch_create_replicated(self.B, self.m, self.n, d["row_ptr"],
                                                   d["col"], d["val"], d["lc"], d["uc"],
                                                   d["l"], d["u"])

    def close(self):
        h, self.h = self.h, None
        if h:
            C.mpax_batch_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass


class SharedLPValues(torch.autograd.Function):
    """forward(C, fs, options, fp32_products) -> (B,) optimal values v_k = min c_k^T x
    over the SharedFeasibleSet fs; C is (B, n).  dv_k/dc_k = x_k*."""

    @staticmethod
    def forward(ctx, Cm, fs, options, fp32_products=False):
        C.mpax_shared_set_costs(fs.h, _f64(Cm))
        C.mpax_shared_solve(fs.h, C.mpax_options_default(**(options or {})), fp32_products)
        X, _ = C.mpax_shared_get_solution(fs.h, fs.m, fs.n, fs.B, device=Cm)
        v = C.mpax_shared_get_objective(fs.h, fs.B, device=Cm)
        ctx.save_for_backward(X)
        return v.to(Cm.dtype)

    @staticmethod
    def backward(ctx, gv):
        (X,) = ctx.saved_tensors
        return (gv[:, None] * X).to(gv.dtype), None, None, None


class SPOPlusLoss(torch.autograd.Function):
    """forward(C_hat, C_true, X_true, Z_true, fs, options, fp32_products) -> (B,)
    SPO+ losses  l_k = -min (2 c^_k - c_k)^T x + 2 c^_k^T x*_k - z*_k  over the
    SharedFeasibleSet fs, with subgradient 2 (x*_k - x~_k): one batched solve and
    the loss formed in the library.  X_true (B, n) and Z_true (B,) are the optima
    of the true costs (for example from SharedLPValues); only C_hat is
    differentiable."""

    @staticmethod
    def forward(ctx, C_hat, C_true, X_true, Z_true, fs, options, fp32_products=False):
        loss, grad = C.mpax_shared_spo_plus(fs.h, C.mpax_options_default(**(options or {})),
                                            _f64(C_hat), _f64(C_true), _f64(X_true),
                                            _f64(Z_true), fp32_products)
        ctx.save_for_backward(grad)
        return loss.to(C_hat.dtype)

    @staticmethod
    def backward(ctx, gl):
        (G,) = ctx.saved_tensors
        return ((gl[:, None] * G).to(gl.dtype),) + (None,) * 6


class SparseLPValues(torch.autograd.Function):
    """forward(C, fs, options) -> (B,) optimal values v_k = min c_k^T x over the
    SparseFeasibleSet fs (one ragged-batch solve); dv_k/dc_k = x_k*."""

    @staticmethod
    def forward(ctx, Cm, fs, options):
        C.mpax_batch_set_costs(fs.h, _f64(Cm))
        C.mpax_batch_solve(fs.h, C.mpax_options_default(**(options or {})))
        x, _ = C.mpax_batch_get_solution(fs.h, fs.B * fs.m, fs.B * fs.n, device=Cm)
        v = C.mpax_batch_get_objective(fs.h, fs.B, device=Cm)
        ctx.save_for_backward(x.view(fs.B, fs.n))
        return v.to(Cm.dtype)

    @staticmethod
    def backward(ctx, gv):
        (X,) = ctx.saved_tensors
        return (gv[:, None] * X).to(gv.dtype), None, None


class SPOPlusLossSparse(torch.autograd.Function):
    """forward(C_hat, C_true, X_true, Z_true, fs, options) -> (B,) SPO+ losses over
    the SparseFeasibleSet fs, one ragged-batch solve with the loss and its
    subgradient 2 (x*_k - x~_k) formed in the library.  Only C_hat is
    differentiable."""

    @staticmethod
    def forward(ctx, C_hat, C_true, X_true, Z_true, fs, options):
        loss, grad = C.mpax_batch_spo_plus(fs.h, C.mpax_options_default(**(options or {})),
                                           _f64(C_hat), _f64(C_true), _f64(X_true),
                                           _f64(Z_true))
        ctx.save_for_backward(grad)
        return loss.to(C_hat.dtype)

    @staticmethod
    def backward(ctx, gl):
        (G,) = ctx.saved_tensors
        return ((gl[:, None] * G).to(gl.dtype),) + (None,) * 5
