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
         c_k of C with one dense A shared by the batch; dv_k/dc_k = x_k*.
SPOPlusLoss: the SPO+ surrogate loss of predicted costs c^_k against true costs c_k
         over the same shared feasible set, with subgradient 2 (x*(c_k) - x~_k),
         x~_k = argmin (2 c^_k - c_k)^T x: one batched solve per forward.
SparseLPValues, SPOPlusLossSparse: the same two layers over one SPARSE feasible set
         (for example the grid shortest-path LP of the paper's Warcraft experiment):
         the B cost rows are solved as B instances of one ragged-batch launch.
"""
from __future__ import annotations

import numpy as np
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


class SharedLPValues(torch.autograd.Function):
    """forward(C, A, lc, uc, l, u, options, fp32_products) -> (B,) optimal values.

    C is (B, n); A is a dense (m, n) FP32 CUDA tensor shared by the batch.  Only C
    is differentiable: dv_k/dc_k = x_k*."""

    @staticmethod
    def forward(ctx, Cm, A, lc, uc, l, u, options, fp32_products=False):
        B, n = Cm.shape
        m = A.shape[0]
        h = C.mpax_lp_shared_create(m, n, B, A.detach(), _f64(Cm), _f64(lc), _f64(uc),
                                    _f64(l), _f64(u))
        try:
            C.mpax_shared_solve(h, C.mpax_options_default(**(options or {})), fp32_products)
            _, per = C.mpax_shared_get_stats(h, B)
            X, _ = C.mpax_shared_get_solution(h, m, n, B, device=Cm)
        finally:
            C.mpax_shared_destroy(h)
        ctx.save_for_backward(X)
        return torch.as_tensor(per["primal_obj"], dtype=Cm.dtype, device=Cm.device)

    @staticmethod
    def backward(ctx, gv):
        (X,) = ctx.saved_tensors
        return (gv[:, None] * X).to(gv.dtype), None, None, None, None, None, None, None


class SPOPlusLoss(torch.autograd.Function):
    """forward(C_hat, C_true, X_true, Z_true, A, lc, uc, l, u, options, fp32_products)
    -> (B,) losses  l_k = -min (2 c^_k - c_k)^T x + 2 c^_k^T x*_k - z*_k.

    X_true (B, n) and Z_true (B,) are the optima of the true costs (for example
    from SharedLPValues); only C_hat is differentiable."""

    @staticmethod
    def forward(ctx, C_hat, C_true, X_true, Z_true, A, lc, uc, l, u, options,
                fp32_products=False):
        B, n = C_hat.shape
        m = A.shape[0]
        Q = (2.0 * C_hat.detach() - C_true.detach()).to(torch.float64).contiguous()
        h = C.mpax_lp_shared_create(m, n, B, A.detach(), Q, _f64(lc), _f64(uc), _f64(l),
                                    _f64(u))
        try:
            C.mpax_shared_solve(h, C.mpax_options_default(**(options or {})), fp32_products)
            _, per = C.mpax_shared_get_stats(h, B)
            Xt, _ = C.mpax_shared_get_solution(h, m, n, B, device=C_hat)
        finally:
            C.mpax_shared_destroy(h)
        Xs = X_true.detach().to(torch.float64)
        v = torch.as_tensor(per["primal_obj"], dtype=torch.float64, device=C_hat.device)
        loss = -v + 2.0 * (C_hat.detach().to(torch.float64) * Xs).sum(1) - Z_true.to(torch.float64)
        ctx.save_for_backward(Xs - Xt)
        return loss.to(C_hat.dtype)

    @staticmethod
    def backward(ctx, gl):
        (D,) = ctx.saved_tensors
        return ((2.0 * gl.to(torch.float64)[:, None] * D).to(gl.dtype),) + (None,) * 10


# ---- one sparse feasible set, B cost vectors: the ragged batch ----------------

def _batch_solve(data, Cm, options):
    """Solve min c_k^T x over the sparse set `data` (numpy m, n, row_ptr, col,
    val, lc, uc, l, u) for the B rows c_k of Cm as one ragged batch (B copies of
    the CSR with local columns).  Returns (X (B, n) like Cm, values (B,) FP64)."""
    B = int(Cm.shape[0])
    m, n = int(data["m"]), int(data["n"])
    rp = np.asarray(data["row_ptr"], dtype=np.int64)
    nnz = int(rp[-1])
    m_off = np.arange(B + 1, dtype=np.int64) * m
    n_off = np.arange(B + 1, dtype=np.int64) * n
    row_ptr = np.concatenate([[0], (rp[1:][None, :] + nnz * np.arange(B)[:, None]).ravel()])
    tile = lambda a, t: np.tile(np.asarray(a, dtype=t), B)  # noqa: E731
    c = Cm.detach().to(torch.float64).cpu().numpy().reshape(-1)
    h = C.mpax_lp_batch_create(B, m_off, n_off, row_ptr, tile(data["col"], np.int32),
                               tile(data["val"], np.float64), c, tile(data["lc"], np.float64),
                               tile(data["uc"], np.float64), tile(data["l"], np.float64),
                               tile(data["u"], np.float64))
    try:
        C.mpax_batch_solve(h, C.mpax_options_default(**(options or {})))
        x, _ = C.mpax_batch_get_solution(h, B * m, B * n)
        _, per = C.mpax_batch_get_stats(h, B)
    finally:
        C.mpax_batch_destroy(h)
    X = torch.from_numpy(x.reshape(B, n)).to(device=Cm.device)
    v = torch.from_numpy(per["primal_obj"].copy()).to(device=Cm.device)
    return X, v


class SparseLPValues(torch.autograd.Function):
    """forward(C, data, options) -> (B,) optimal values v_k = min c_k^T x over the
    sparse set `data` (see _batch_solve); dv_k/dc_k = x_k*."""

    @staticmethod
    def forward(ctx, Cm, data, options):
        X, v = _batch_solve(data, Cm, options)
        ctx.save_for_backward(X)
        return v.to(Cm.dtype)

    @staticmethod
    def backward(ctx, gv):
        (X,) = ctx.saved_tensors
        return (gv[:, None] * X).to(gv.dtype), None, None


class SPOPlusLossSparse(torch.autograd.Function):
    """forward(C_hat, C_true, X_true, Z_true, data, options) -> (B,) SPO+ losses
    -min (2 c^_k - c_k)^T x + 2 c^_k^T x*_k - z*_k over the sparse set `data`,
    one ragged-batch solve; subgradient 2 (x*_k - x~_k).  Only C_hat is
    differentiable."""

    @staticmethod
    def forward(ctx, C_hat, C_true, X_true, Z_true, data, options):
        Q = 2.0 * C_hat.detach().to(torch.float64) - C_true.detach().to(torch.float64)
        Xt, v = _batch_solve(data, Q, options)
        Xs = X_true.detach().to(torch.float64)
        loss = -v + 2.0 * (C_hat.detach().to(torch.float64) * Xs).sum(1) - Z_true.to(torch.float64)
        ctx.save_for_backward(Xs - Xt)
        return loss.to(C_hat.dtype)

    @staticmethod
    def backward(ctx, gl):
        (D,) = ctx.saved_tensors
        return ((2.0 * gl.to(torch.float64)[:, None] * D).to(gl.dtype),) + (None,) * 5
