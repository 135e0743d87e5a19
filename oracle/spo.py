"""Oracle of the SPO+ surrogate loss (the LP surrogate gradient the paper uses
for decision-focused learning, Sec. 3.4): for a predicted cost c_hat and a true
cost c with optimum x*(c) and value z*(c) over the feasible set S,

    l(c_hat, c) = -min_{x in S} (2 c_hat - c)^T x + 2 c_hat^T x*(c) - z*(c),

convex in c_hat, zero at c_hat = c, with subgradient 2 (x*(c) - x~), x~ a
minimiser of (2 c_hat - c)^T x over S (Elmachtoub and Grigas, "Smart
'Predict, then Optimize'", Management Science 2022).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The inner LP is solved
by this oracle's own r^2HPDHG (pdhg.solve_lp)."""
from __future__ import annotations

import numpy as np

from .pdhg import Options, Problem, solve_lp


def spo_plus(p: Problem, c_hat, x_star, z_star, opts: Options = Options()):
    """(loss, subgradient, x~) of SPO+ at c_hat for the true cost p.c with optimum
    (x_star, z_star)."""
    c_hat = np.asarray(c_hat, dtype=np.float64)
    q = Problem(p.A, 2.0 * c_hat - p.c, p.lc, p.uc, p.l, p.u)
    r = solve_lp(q, opts)
    x_t = r.x
    loss = -float(q.c @ x_t) + 2.0 * float(c_hat @ x_star) - float(z_star)
    return loss, 2.0 * (np.asarray(x_star) - x_t), x_t
