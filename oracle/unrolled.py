"""Oracle for differentiation by unrolling the QP iteration (Sec. 3.4: the
paper obtains a QP solution's gradients by differentiating through the steps
of Algorithm 2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

What is differentiated.  A solve of oracle.pdhg.solve_qp is a finite sequence
of rAPDHG steps (eqs. 5-6 with beta_k = theta_k = 2/(k+2)) and restarts.  One
step from (x, y, xa, ya) -- xa, ya the running averages -- with inner counter
k and step sizes tau, sigma (scaled data, Q~ = diag(D~) + F~ F~^T):

    b    = 2 / (k + 2)
    x_md = xa + b (x - xa)
    vx   = x - tau (Q~ x_md + c~ - A~^T y)
    x+   = proj_[l~,u~](vx)
    s    = A~ (2 x+ - x)
    vy   = y / sigma - s
    y+   = sigma (vy - proj_[-uc~,-lc~](vy))
    xa+  = xa + b (x+ - xa),    ya+ = ya + b (y+ - ya)

and a restart sets x <- xa, y <- ya.  The solve returns x = D_c xa_T,
y = D_r ya_T.  Starting from x = y = 0, that point is a function of
(c, lc, uc, l, u, D) along the path the solve took.

Readings (the paper states none of them):

  * Held fixed along the path: every decision of the solve (at which checks it
    restarted, where it stopped), every scalar it computed from its iterates
    (the primal weight, hence tau and sigma), the norm estimates and the
    scaling factors D_r, D_c.  The limit point of the iteration depends on
    none of them, so the derivative's limit is unchanged by holding them.
  * proj_[lo,hi](v) = min(max(v, lo), hi) has derivative 1 in v when
    lo < v < hi and 0 otherwise; otherwise it returns lo (v <= lo) or hi
    (v >= hi, v > lo) and has derivative 1 in that bound.  (A derivative is
    needed only away from these ties; the choice at a tie is a convention.)
  * The start point is zero and depends on no parameter.

Reverse sweep.  With adjoints (gx, gy, gxa, gya) of (x+, y+, xa+, ya+), one
step backwards is, in the order the forward step is undone:

    dual:    ty  = gy + b gya;  w = ty where vy was clamped, else 0 (y+ = 0
             identically where vy is inside);  y+ = y - sigma s - sigma bound
             there, so  gy <- w,  g_bound += -sigma w,  gs = -sigma w
    reflect: gxr = A~^T gs;  tx = gx + b gxa + 2 gxr;  gx <- -gxr
    primal:  ux = tx where vx is inside, else 0; g_l~ / g_u~ += tx at l / u;
             gx += ux;  gq = -tau ux;  g_c~ += gq;  gy += -A~ gq;
             g_D~ += gq * x_md;  gxmd = Q~ gq;  gx += b gxmd
    average: gxa <- (1 - b)(gxa + gxmd),  gya <- (1 - b) gya

(g_bound on the dual side is -sigma w: bound -uc~ when vy <= -uc~, so
g_uc~ += sigma w; else -lc~, so g_lc~ += sigma w).  A restart is undone by
gxa += gx, gx = 0, gya += gy, gy = 0.  Finally the scaled gradients are taken
back to the data: c~ = D_c c, l~ = l / D_c, u~ = u / D_c, lc~ = D_r lc,
uc~ = D_r uc, D~ = D_c^2 D.  An equality row (lc = uc = b) has
dL/db = dL/dlc + dL/duc.
"""
from __future__ import annotations

import numpy as np

from .pdhg import Options, Problem, clamp, scale_problem, solve_qp


def _codes(v, lo, hi):
    """0 where lo < v < hi; 1 where proj returns lo; 2 where it returns hi."""
    inside = (v > lo) & (v < hi)
    at_lo = ~(v > lo)
    return np.where(inside, 0, np.where(at_lo, 1, 2))


def taped_solve(p: Problem, opts: Options = Options()):
    """solve_qp with the record of its path.  Returns (Result, tape)."""
    tape = []
    res = solve_qp(p, opts, tape=tape)
    return res, tape


def schedule(tape):
    """The decisions and scalars of a path: ("step", k, tau, sigma) and ("restart",)."""
    return [e[:4] if e[0] == "step" else e for e in tape]


def replay(ps: Problem, sched, x0=None, y0=None):
    """Runs the scaled problem ps along a fixed schedule from (x0, y0) (zeros by
    default) and returns the final averages (xa, ya).  It is the function whose
    derivative unrolled_gradient computes, for finite-difference checks."""
    x = np.zeros(ps.n) if x0 is None else x0.copy()
    y = np.zeros(ps.m) if y0 is None else y0.copy()
    xa, ya = x.copy(), y.copy()
    for e in sched:
        if e[0] == "restart":
            x, y = xa.copy(), ya.copy()
            continue
        _, k, tau, sigma = e
        b = 2.0 / (k + 2)
        x_md = xa + b * (x - xa)
        vx = x - tau * (ps.qx(x_md) + ps.c - ps.A.T @ y)
        xn = clamp(vx, ps.l, ps.u)
        s = ps.A @ (2.0 * xn - x)
        vy = y / sigma - s
        yn = sigma * (vy - clamp(vy, -ps.uc, -ps.lc))
        xa = xa + b * (xn - xa)
        ya = ya + b * (yn - ya)
        x, y = xn, yn
    return xa, ya


def unrolled_gradient(p: Problem, res, tape, gx, gy=None):
    """Gradients of L = gx . x + gy . y at the returned point (x, y) of a taped
    solve, along its path: dict(c, lc, uc, l, u, D) (D: the diagonal of
    diag(D) + F F^T, or of a general sparse Q), all for the unscaled data."""
    Dr, Dc = res.Dr, res.Dc
    ps = scale_problem(p, Dr, Dc)
    n, m = p.n, p.m
    A = ps.A
    g_xa = Dc * np.asarray(gx, dtype=np.float64)
    g_ya = np.zeros(m) if gy is None else Dr * np.asarray(gy, dtype=np.float64)
    g_x = np.zeros(n)
    g_y = np.zeros(m)
    G = {k: np.zeros(n) for k in ("c", "l", "u", "D")}
    G.update({k: np.zeros(m) for k in ("lc", "uc")})
    for e in reversed(tape):
        if e[0] == "restart":
            g_xa = g_xa + g_x
            g_x = np.zeros(n)
            g_ya = g_ya + g_y
            g_y = np.zeros(m)
            continue
        _, k, tau, sigma, x, y, xa, ya = e
        # the forward step from its recorded start, for the codes and x_md
        b = 2.0 / (k + 2)
        x_md = xa + b * (x - xa)
        vx = x - tau * (ps.qx(x_md) + ps.c - A.T @ y)
        xn = clamp(vx, ps.l, ps.u)
        vy = y / sigma - A @ (2.0 * xn - x)
        cx = _codes(vx, ps.l, ps.u)
        cy = _codes(vy, -ps.uc, -ps.lc)
        # dual
        ty = g_y + b * g_ya
        w = np.where(cy == 0, 0.0, ty)
        G["uc"] += np.where(cy == 1, sigma * w, 0.0)
        G["lc"] += np.where(cy == 2, sigma * w, 0.0)
        gxr = A.T @ (-sigma * w)
        new_gy = w
        # reflection 2 x+ - x
        tx = g_x + b * g_xa + 2.0 * gxr
        new_gx = -gxr
        # primal
        ux = np.where(cx == 0, tx, 0.0)
        G["l"] += np.where(cx == 1, tx, 0.0)
        G["u"] += np.where(cx == 2, tx, 0.0)
        new_gx = new_gx + ux
        gq = -tau * ux
        G["c"] += gq
        new_gy = new_gy - A @ gq
        G["D"] += gq * x_md
        gxmd = ps.qx(gq)
        new_gx = new_gx + b * gxmd
        # averages
        g_xa = (1.0 - b) * (g_xa + gxmd)
        g_ya = (1.0 - b) * g_ya
        g_x, g_y = new_gx, new_gy
    out = dict(c=Dc * G["c"], l=G["l"] / Dc, u=G["u"] / Dc, lc=Dr * G["lc"], uc=Dr * G["uc"])
    if p.Q is not None:  # D of diag(D) + F F^T, or the diagonal of a general Q
        out["D"] = Dc * Dc * G["D"]
    return out


def solve_and_differentiate(p: Problem, gx, gy=None, opts: Options = Options()):
    """Taped solve plus its unrolled gradients: (Result, gradients dict)."""
    res, tape = taped_solve(p, opts)
    return res, unrolled_gradient(p, res, tape, gx, gy)


__all__ = ["taped_solve", "schedule", "replay", "unrolled_gradient",
           "solve_and_differentiate"]
