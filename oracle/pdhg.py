"""Oracle for the restarted PDHG methods of the paper (FP64, CPU, numpy/scipy).

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never
imports this module, and this module never imports the CUDA library.

Problem (1) of Sec. 2:  min 1/2 x^T Q x + c^T x  s.t.  lc <= A x <= uc,  l <= x <= u.
Infinite bounds are IEEE +-inf.  Q = 0 gives an LP.

The paper states the iterations (eqs. 3-6, Algorithms 1 and 2) and names the
heuristics around them (diagonal preconditioning, adaptive restarts, step sizes,
primal-weight updates, relative-KKT termination; Sec. 3) without giving their
rules.  This oracle fixes one reading of each unstated rule; the CUDA path
implements the same written rules.  The readings are:

  * Scaling (Sec. 3): ``ruiz_iters`` rounds of Ruiz equilibration, each
    computing from the current scaled matrix K the row factors
    1/sqrt(max_j |K_ij|) and column factors 1/sqrt(max_i |K_ij|) (1 for an
    empty row/column) and applying both; then one Pock-Chambolle round with
    alpha = 1: factors 1/sqrt(sum_j |K_ij|) and 1/sqrt(sum_i |K_ij|).  For a QP
    the scaled diagonal Q~_jj joins column j's norm (max in the Ruiz rounds,
    sum in the Pock-Chambolle round) in place of Q's part of the KKT matrix;
    Q is scaled congruently (Q~ = D_c Q D_c).
    Scaled data: A~ = D_r A D_c, c~ = D_c c, Q~ = D_c Q D_c, [l~, u~] = [l, u]/D_c,
    [lc~, uc~] = D_r [lc, uc]; x = D_c x~, y = D_r y~.
  * Step sizes: eta = 0.998 / ||A~||_2 with ||A~||_2 from power iteration on
    A~^T A~ started at a fixed pseudo-random vector of entries in [-1, 1]
    (SplitMix64 of the index, see power_start).  After the Pock-Chambolle round
    ||A~||_2 <= 1 (Schur's test), and the iteration stops, using 1, once its
    extrapolated estimate is within 1e-3 of that bound; power_max_iter = 0
    takes that bound without any power round (on small instances the rounds
    cost as much as the solve).  The estimates rise towards the norm
    with geometrically shrinking increments d_t (ratio q); the iteration stops
    when d_t and the extrapolated remainder d_t q / (1 - q) are both at most
    1e-4 of the estimate (or after 1000 rounds) and returns the estimate plus
    the remainder.  (Stopping on the last change alone left the estimate up to
    2% low on matrices whose two top singular values are close, and a step with
    tau sigma ||A~||^2 > 1 diverges.)  LP: tau = eta/omega,
    sigma = eta*omega, fixed inside a restart cycle.  QP: sigma = eta*omega,
    tau = 0.998 / (||Q~||_2 + sigma ||A~||_2^2).
  * Primal weight: omega_0 = ||c~|| / ||b~|| when both exceed 1e-10, else 1,
    where b_i is the finite one of (lc_i, uc_i) (the larger in magnitude when
    both are finite, 0 when neither is).  At a restart,
    omega <- exp(0.5 log(||dy|| / ||dx||) + 0.5 log omega) where dx, dy are the
    moves of the restart anchor, applied only when both norms exceed 1e-10.
  * Checks run every ``check_every`` iterations (and at the iteration limit).
    LP restart metric: r = sqrt(omega ||x^ - x||^2 + ||y^ - y||^2 / omega)
    from the iterate z = (x, y) to its PDHG image z^ (scaled space).  QP
    restart metric: the relative KKT error of the averaged iterate.
    Restart when any of: r <= 0.2 r_anchor; r <= 0.8 r_anchor and r > r_prev;
    k >= 0.36 * t (k = steps in this cycle, t = all steps).  r_anchor is the
    metric at the restart that opened the cycle, r_prev the metric at the
    previous check of the cycle (r_anchor right after a restart).
  * Relative KKT error at (x, y) on the unscaled problem:
       r_p = A x - proj_[lc,uc](A x)
       lam = Q x + c - A^T y,   r_d = lam - proj_Lambda(lam)
       Lambda_j = R (l_j, u_j finite), R+ (only l_j), R- (only u_j), {0} (neither)
       p = 1/2 x^T Q x + c^T x
       d = -1/2 x^T Q x + sum lc_i y_i^+ - uc_i y_i^- + sum l_j lh_j^+ - u_j lh_j^-
           (lh = proj_Lambda(lam); terms with an infinite bound are dropped)
    converged iff ||r_p|| <= eps_abs + eps_rel ||b||, ||r_d|| <= eps_abs +
    eps_rel ||c||, |p - d| <= eps_abs + eps_rel (|p| + |d|).  The reported
    relative KKT error is the largest of ||r_p||/(1+||b||), ||r_d||/(1+||c||),
    |p-d|/(1+|p|+|d|).
  * Algorithm 1 writes A(2 x^{n,k+1} - x^{n,k}) in its dual line; eq. (3)
    uses the new PDHG primal point, which is what is done here: A(2 x^ - x).
  * rAPDHG schedules: beta_k = theta_k = 2/(k+2), k the inner counter.
  * Infeasibility detection (LP; Sec. 3 names it, the option table gives
    eps_primal_infeasible = eps_dual_infeasible = 1e-8): at every check the
    move of the cycle since its anchor, dx = D_c (x^ - x_anchor) and
    dy = D_r (y^ - y_anchor), is tested as a certificate.
      Primal infeasible (a Farkas ray): y = dy projected onto the recession
      cone of Y (y_i >= 0 where uc_i = +inf, y_i <= 0 where lc_i = -inf),
      lam = -A^T y, lh = proj_Lambda(lam); the ray's dual objective
      o = sum lc_i y_i^+ - uc_i y_i^- + sum l_j lh_j^+ - u_j lh_j^- (finite
      terms) must be positive and ||lam - lh|| <= eps_primal_infeasible * o.
      Dual infeasible (an unbounded primal ray): x = dx with
      ||A x - proj_R(A x)||^2 + ||x - proj_X(x)||^2 <= (eps_dual_infeasible c^T x)^2
      and c^T x < 0, where R and X are the recession cones of [lc, uc] and
      [l, u] (0 where both bounds are finite, R+ / R- where only the lower /
      upper one is, R where neither).
    The certificate is returned as Result.certificate.
  * Feasibility polishing (Sec. 3.3; off by default): see polish_lp.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

INF = math.inf


# -----------------------------------------------------------------------------
# Problem data
# -----------------------------------------------------------------------------

class DiagLowRankQ:
    """Q = diag(D) + F F^T, applied as an operator (F is n x r sparse)."""

    def __init__(self, D, F):
        self.D = np.asarray(D, dtype=np.float64)
        self.F = sp.csr_matrix(F, dtype=np.float64)

    def matvec(self, x):
        return self.D * x + self.F @ (self.F.T @ x)

    def congruent(self, d):
        """diag(d) Q diag(d)."""
        return DiagLowRankQ(d * d * self.D, sp.diags(d) @ self.F)

    def diagonal(self):
        return self.D + np.asarray(self.F.multiply(self.F).sum(axis=1)).ravel()

    def dense(self):
        return np.diag(self.D) + (self.F @ self.F.T).toarray()


class SparseQ:
    def __init__(self, Q):
        self.Q = sp.csr_matrix(Q, dtype=np.float64)

    def matvec(self, x):
        return self.Q @ x

    def congruent(self, d):
        return SparseQ(sp.diags(d) @ self.Q @ sp.diags(d))

    def diagonal(self):
        return self.Q.diagonal()

    def dense(self):
        return self.Q.toarray()


@dataclass
class Problem:
    A: sp.csr_matrix
    c: np.ndarray
    lc: np.ndarray
    uc: np.ndarray
    l: np.ndarray
    u: np.ndarray
    Q: object = None  # None, SparseQ or DiagLowRankQ

    @property
    def m(self):
        return self.A.shape[0]

    @property
    def n(self):
        return self.A.shape[1]

    def qx(self, x):
        return np.zeros_like(x) if self.Q is None else self.Q.matvec(x)


def problem_from_arrays(d: dict) -> Problem:
    """Build a Problem from a generator dictionary (synth.*)."""
    A = sp.csr_matrix((np.asarray(d["val"], dtype=np.float64), np.asarray(d["col"]),
                       np.asarray(d["row_ptr"])), shape=(d["m"], d["n"]))
    Q = None
    if "D" in d:
        F = sp.csr_matrix((d["f_val"], d["f_col"], d["f_row_ptr"]), shape=(d["n"], d["f_cols"]))
        Q = DiagLowRankQ(d["D"], F)
    elif "q_row_ptr" in d:
        Q = SparseQ(sp.csr_matrix((d["q_val"], d["q_col"], d["q_row_ptr"]),
                                  shape=(d["n"], d["n"])))
    return Problem(A, np.array(d["c"], dtype=np.float64), np.array(d["lc"], dtype=np.float64),
                   np.array(d["uc"], dtype=np.float64), np.array(d["l"], dtype=np.float64),
                   np.array(d["u"], dtype=np.float64), Q)


@dataclass
class Options:
    eps_abs: float = 1e-4
    eps_rel: float = 1e-4
    iteration_limit: int = 2**62
    check_every: int = 64
    ruiz_iters: int = 10
    pock_chambolle: bool = True
    reflection_gamma: float = 1.0
    restart_sufficient: float = 0.2
    restart_necessary: float = 0.8
    restart_artificial: float = 0.36
    primal_weight_smoothing: float = 0.5
    step_safety: float = 0.998
    power_max_iter: int = 1000
    power_tol: float = 1e-4
    eps_primal_infeasible: float = 1e-8
    eps_dual_infeasible: float = 1e-8


# -----------------------------------------------------------------------------
# Preconditioning (Sec. 3: Ruiz, then Pock-Chambolle with alpha = 1)
# -----------------------------------------------------------------------------

def _inv_sqrt_or_one(v):
    out = np.ones_like(v)
    pos = v > 0
    out[pos] = 1.0 / np.sqrt(v[pos])
    return out


def scaling_factors(A: sp.csr_matrix, ruiz_iters: int = 10, pock_chambolle: bool = True,
                    qdiag=None):
    """Diagonal factors (D_r, D_c) such that A~ = diag(D_r) A diag(D_c).

    For a QP, `qdiag` is the diagonal of Q; the scaled diagonal
    Q~_jj = D_c,j^2 Q_jj joins column j's norm (max with the column's
    infinity-norm in a Ruiz round, added to its 1-norm in the Pock-Chambolle
    round), standing in for Q's part of the KKT matrix."""
    m, n = A.shape
    Dr = np.ones(m)
    Dc = np.ones(n)
    K = sp.csr_matrix(A, copy=True)
    for _ in range(ruiz_iters):
        absK = abs(K)
        row_max = np.asarray(absK.max(axis=1).todense()).ravel() if m and n else np.zeros(m)
        col_max = np.asarray(absK.max(axis=0).todense()).ravel() if m and n else np.zeros(n)
        if qdiag is not None:
            col_max = np.maximum(col_max, Dc * Dc * qdiag)
        dr = _inv_sqrt_or_one(row_max)
        dc = _inv_sqrt_or_one(col_max)
        K = sp.csr_matrix(sp.diags(dr) @ K @ sp.diags(dc))
        Dr *= dr
        Dc *= dc
    if pock_chambolle:
        absK = abs(K)
        row_sum = np.asarray(absK.sum(axis=1)).ravel()
        col_sum = np.asarray(absK.sum(axis=0)).ravel()
        if qdiag is not None:
            col_sum = col_sum + Dc * Dc * qdiag
        dr = _inv_sqrt_or_one(row_sum)
        dc = _inv_sqrt_or_one(col_sum)
        Dr *= dr
        Dc *= dc
    return Dr, Dc


def scale_problem(p: Problem, Dr, Dc) -> Problem:
    A = sp.csr_matrix(sp.diags(Dr) @ p.A @ sp.diags(Dc))
    Q = None if p.Q is None else p.Q.congruent(Dc)
    return Problem(A, Dc * p.c, Dr * p.lc, Dr * p.uc, p.l / Dc, p.u / Dc, Q)


# -----------------------------------------------------------------------------
# Operator norms by power iteration
# -----------------------------------------------------------------------------

_M64 = (1 << 64) - 1
POWER_SEED = 0x6D706178  # counter base of the power iteration's start vector


def _splitmix64(x: int) -> int:
    """SplitMix64 (Steele, Lea and Flood, 2014) of the 64-bit counter x."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def power_start(n: int) -> np.ndarray:
    """Start vector of the power iterations: v_j = 2 u_j - 1 with u_j the top 53
    bits of SplitMix64(POWER_SEED + j) over 2^53, normalised.  A vector with
    entries of both signs and no structure has a component along every singular
    vector; the all-ones vector can be nearly orthogonal to the top one, and the
    iteration then settles on the second singular value first."""
    v = np.array([2.0 * ((_splitmix64(POWER_SEED + j) >> 11) * 2.0 ** -53) - 1.0
                  for j in range(n)])
    return v / np.linalg.norm(v)


def _power_stop(nu, nu_prev, d_prev, tol, cap=math.inf):
    """Stopping rule of the power iterations: the estimates nu_t rise towards the
    norm with increments d_t = nu_t - nu_{t-1} that shrink geometrically (ratio
    q = d_t / d_{t-1}) once the top singular vector dominates, so the distance
    still to go is about d_t q / (1 - q).  Stop when both the last increment and
    that remainder are at most tol * nu_t; the estimate is nu_t + remainder.
    With a certified upper bound `cap` on the norm, stop as soon as the
    extrapolated estimate is within 10 tol of the cap, and use the cap, once the
    increments are small (d_t <= 100 tol nu_t: before that the ratio q is not yet
    settled and the extrapolation overshoots); an estimate never exceeds the
    cap.  Returns (stop, estimate, d_t)."""
    d = nu - nu_prev
    if d <= 0.0:                      # no rise left (rounding): converged
        return True, min(nu, cap), d
    q = d / d_prev if d_prev > 0.0 else 1.0
    if q >= 1.0:                      # not yet in the geometric regime
        return False, nu, d
    rem = d * q / (1.0 - q)
    if d <= 100.0 * tol * nu and nu + rem >= (1.0 - 10.0 * tol) * cap:
        return True, cap, d
    if d <= tol * nu and rem <= tol * nu:
        return True, min(nu + rem, cap), d
    return False, nu, d


def power_norm_A(A: sp.csr_matrix, max_iter: int = 1000, tol: float = 1e-4,
                 cap: float = math.inf):
    """Estimate ||A||_2 = sqrt(lambda_max(A^T A)); start at power_start(n);
    nu_t = sqrt(||A^T A v_t||) with ||v_t|| = 1; stop by _power_stop with the
    certified bound `cap` (min(cap, last estimate) after max_iter rounds)."""
    n = A.shape[1]
    if n == 0 or A.nnz == 0:
        return 0.0, 0
    if max_iter == 0:                 # no power iteration: the certified bound itself
        if not math.isfinite(cap):
            raise ValueError("power_max_iter = 0 needs a certified bound on ||A~||_2")
        return cap, 0
    v = power_start(n)
    nu_prev, d_prev = None, 0.0
    for t in range(1, max_iter + 1):
        w = A @ v
        g = A.T @ w
        nrm = float(np.linalg.norm(g))
        if nrm == 0.0:
            return 0.0, t
        nu = math.sqrt(nrm)
        v = g / nrm
        if nu_prev is not None:
            stop, est, d_prev = _power_stop(nu, nu_prev, d_prev, tol, cap)
            if stop:
                return est, t
        nu_prev = nu
    return (cap if math.isfinite(cap) else nu), max_iter


def power_norm_Q(Q, n: int, max_iter: int = 1000, tol: float = 1e-4):
    """Estimate ||Q||_2 for symmetric PSD Q: start at power_start(n);
    nu_t = ||Q v_t||, ||v_t|| = 1; stop by _power_stop."""
    if Q is None or n == 0:
        return 0.0, 0
    v = power_start(n)
    nu_prev, d_prev = None, 0.0
    for t in range(1, max_iter + 1):
        g = Q.matvec(v)
        nu = float(np.linalg.norm(g))
        if nu == 0.0:
            return 0.0, t
        v = g / nu
        if nu_prev is not None:
            stop, est, d_prev = _power_stop(nu, nu_prev, d_prev, tol)
            if stop:
                return est, t
        nu_prev = nu
    return nu, max_iter


# -----------------------------------------------------------------------------
# Bound helpers
# -----------------------------------------------------------------------------

def bound_vector(lc, uc):
    """b_i: the finite one of (lc_i, uc_i); the larger magnitude when both are
    finite; 0 when neither is."""
    b = np.zeros_like(lc)
    fl = np.isfinite(lc)
    fu = np.isfinite(uc)
    b[fl & ~fu] = lc[fl & ~fu]
    b[fu & ~fl] = uc[fu & ~fl]
    both = fl & fu
    b[both] = np.where(np.abs(lc[both]) >= np.abs(uc[both]), lc[both], uc[both])
    return b


def initial_primal_weight(c_s, b_s):
    nc = float(np.linalg.norm(c_s))
    nb = float(np.linalg.norm(b_s))
    return nc / nb if (nc > 1e-10 and nb > 1e-10) else 1.0


def clamp(v, lo, hi):
    return np.minimum(np.maximum(v, lo), hi)


# -----------------------------------------------------------------------------
# One PDHG step (eqs. 3 and 5) and the Halpern/reflection update (eq. 4)
# -----------------------------------------------------------------------------

def dual_prox(y, s, sigma, lc, uc):
    """y - sigma s - sigma proj_[-uc,-lc](y/sigma - s), the dual line of eq. (3)
    with s = A(2 x^ - x)."""
    v = y / sigma - s
    return y - sigma * s - sigma * clamp(v, -uc, -lc)


def pdhg_step_lp(p: Problem, x, y, tau, sigma):
    """Eq. (3): returns (x^, y^, xbar) with xbar = 2 x^ - x."""
    x_hat = clamp(x - tau * (p.c - p.A.T @ y), p.l, p.u)
    xbar = 2.0 * x_hat - x
    y_hat = dual_prox(y, p.A @ xbar, sigma, p.lc, p.uc)
    return x_hat, y_hat, xbar


def halpern(z_hat, z, z_anchor, k, gamma):
    """Eq. (4): (k+1)/(k+2) ((1+gamma) z^ - gamma z) + 1/(k+2) z_anchor."""
    return (k + 1) / (k + 2) * ((1.0 + gamma) * z_hat - gamma * z) + z_anchor / (k + 2)


def apdhg_step_qp(p: Problem, x, y, xavg, yavg, k, tau, sigma):
    """One inner step of Algorithm 2 with beta_k = theta_k = 2/(k+2):
    momentum primal step (eq. 6), dual step of eq. (5), weighted averages.
    Returns (x+, y+, xavg+, yavg+, xref) with xref = 2 x+ - x."""
    beta = 2.0 / (k + 2)
    theta = 2.0 / (k + 2)
    x_md = (1.0 - beta) * xavg + beta * x
    g = p.qx(x_md) + p.c - p.A.T @ y
    x_new = clamp(x - tau * g, p.l, p.u)
    xref = 2.0 * x_new - x
    y_new = dual_prox(y, p.A @ xref, sigma, p.lc, p.uc)
    xavg_new = (1.0 - theta) * xavg + theta * x_new
    yavg_new = (1.0 - theta) * yavg + theta * y_new
    return x_new, y_new, xavg_new, yavg_new, xref


# -----------------------------------------------------------------------------
# Relative KKT error on the unscaled problem
# -----------------------------------------------------------------------------

def kkt(p: Problem, x, y, eps_abs=1e-4, eps_rel=1e-4):
    ax = p.A @ x
    r_p = ax - clamp(ax, p.lc, p.uc)
    qx = p.qx(x)
    lam = qx + p.c - p.A.T @ y
    fl = np.isfinite(p.l)
    fu = np.isfinite(p.u)
    lam_proj = np.where(fl & fu, lam,
                        np.where(fl, np.maximum(lam, 0.0),
                                 np.where(fu, np.minimum(lam, 0.0), 0.0)))
    r_d = lam - lam_proj
    xqx = float(x @ qx)
    p_obj = 0.5 * xqx + float(p.c @ x)
    yp = np.maximum(y, 0.0)
    ym = np.maximum(-y, 0.0)
    lp_ = np.maximum(lam_proj, 0.0)
    lm_ = np.maximum(-lam_proj, 0.0)
    lcf = np.where(np.isfinite(p.lc), p.lc, 0.0)
    ucf = np.where(np.isfinite(p.uc), p.uc, 0.0)
    lf = np.where(fl, p.l, 0.0)
    uf = np.where(fu, p.u, 0.0)
    d_obj = (-0.5 * xqx + float(lcf @ yp) - float(ucf @ ym)
             + float(lf @ lp_) - float(uf @ lm_))
    nb = float(np.linalg.norm(bound_vector(p.lc, p.uc)))
    nc = float(np.linalg.norm(p.c))
    nrp = float(np.linalg.norm(r_p))
    nrd = float(np.linalg.norm(r_d))
    gap = abs(p_obj - d_obj)
    rel = max(nrp / (1.0 + nb), nrd / (1.0 + nc), gap / (1.0 + abs(p_obj) + abs(d_obj)))
    ok = (nrp <= eps_abs + eps_rel * nb and nrd <= eps_abs + eps_rel * nc
          and gap <= eps_abs + eps_rel * (abs(p_obj) + abs(d_obj)))
    return dict(primal_res=nrp, dual_res=nrd, primal_obj=p_obj, dual_obj=d_obj, gap=gap,
                rel_kkt=rel, converged=bool(ok), b_norm=nb, c_norm=nc)


# -----------------------------------------------------------------------------
# Solvers
# -----------------------------------------------------------------------------

@dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    status: str
    iterations: int
    restarts: int
    kkt: dict
    omega: float
    eta: float
    norm_A: float
    norm_Q: float
    Dr: np.ndarray
    Dc: np.ndarray
    history: list = field(default_factory=list)
    certificate: np.ndarray | None = None
    # (total iterations, primal weight after the update) at every restart
    restart_log: list = field(default_factory=list)


# -----------------------------------------------------------------------------
# Infeasibility certificates (the reading in the module docstring)
# -----------------------------------------------------------------------------

def _recession(v, lo_finite, hi_finite):
    """Projection onto the recession cone of an interval with the given finite ends."""
    return np.where(lo_finite & hi_finite, 0.0,
                    np.where(lo_finite, np.maximum(v, 0.0),
                             np.where(hi_finite, np.minimum(v, 0.0), v)))


def primal_ray_test(p: Problem, dy):
    """(violation, objective) of the dual ray dy as a certificate of primal infeasibility."""
    flc, fuc = np.isfinite(p.lc), np.isfinite(p.uc)
    y = np.where(~fuc, np.maximum(dy, 0.0), dy)
    y = np.where(~flc, np.minimum(y, 0.0), y)
    lam = -(p.A.T @ y)
    fl, fu = np.isfinite(p.l), np.isfinite(p.u)
    lh = np.where(fl & fu, lam, np.where(fl, np.maximum(lam, 0.0),
                                         np.where(fu, np.minimum(lam, 0.0), 0.0)))
    obj = (float(np.where(flc, p.lc, 0.0) @ np.maximum(y, 0.0))
           - float(np.where(fuc, p.uc, 0.0) @ np.maximum(-y, 0.0))
           + float(np.where(fl, p.l, 0.0) @ np.maximum(lh, 0.0))
           - float(np.where(fu, p.u, 0.0) @ np.maximum(-lh, 0.0)))
    return float(np.linalg.norm(lam - lh)), obj, y


def dual_ray_test(p: Problem, dx):
    """(violation, c^T dx) of the primal ray dx as a certificate of dual infeasibility."""
    ax = p.A @ dx
    vr = ax - _recession(ax, np.isfinite(p.lc), np.isfinite(p.uc))
    vx = dx - _recession(dx, np.isfinite(p.l), np.isfinite(p.u))
    return math.sqrt(float(vr @ vr) + float(vx @ vx)), float(p.c @ dx)


def infeasibility(p: Problem, dx, dy, opts: Options):
    """'primal_infeasible' / 'dual_infeasible' with its certificate, or (None, None)."""
    if opts.eps_primal_infeasible > 0.0:
        vp, op, yray = primal_ray_test(p, dy)
        if op > 0.0 and vp <= opts.eps_primal_infeasible * op:
            return "primal_infeasible", yray
    if opts.eps_dual_infeasible > 0.0:
        vd, cd = dual_ray_test(p, dx)
        if cd < 0.0 and vd <= opts.eps_dual_infeasible * (-cd):
            return "dual_infeasible", dx
    return None, None


def prepare(p: Problem, opts: Options):
    """Scaling, operator norms and the initial primal weight."""
    qd = None if p.Q is None else p.Q.diagonal()
    Dr, Dc = scaling_factors(p.A, opts.ruiz_iters, opts.pock_chambolle, qd)
    ps = scale_problem(p, Dr, Dc)
    # after the Pock-Chambolle round (alpha = 1) A~_ij = K_ij / sqrt(r_i c_j) with
    # r, c the row and column 1-norms of the Ruiz-scaled K (c_j also holding Q's
    # scaled diagonal), and Schur's test with weights sqrt(r_i), sqrt(c_j) gives
    # ||A~||_2 <= 1
    cap = 1.0 if opts.pock_chambolle else math.inf
    nA, _ = power_norm_A(ps.A, opts.power_max_iter, opts.power_tol, cap)
    nQ, _ = power_norm_Q(ps.Q, ps.n, opts.power_max_iter, opts.power_tol)
    eta = opts.step_safety / nA if nA > 0 else 1.0
    omega = initial_primal_weight(ps.c, bound_vector(ps.lc, ps.uc))
    return ps, Dr, Dc, nA, nQ, eta, omega


def step_sizes(eta, omega, nA, nQ, opts: Options, is_qp: bool):
    if not is_qp:
        return eta / omega, eta * omega
    sigma = eta * omega
    denom = nQ + sigma * nA * nA
    tau = opts.step_safety / denom if denom > 0 else 1.0
    return tau, sigma


def _restart_decision(r, r_anchor, r_prev, k_cycle, total, opts: Options):
    if r_anchor is None:
        return True
    return (r <= opts.restart_sufficient * r_anchor
            or (r <= opts.restart_necessary * r_anchor and r > r_prev)
            or k_cycle >= opts.restart_artificial * total)


def _update_weight(omega, dx, dy, opts: Options):
    if dx > 1e-10 and dy > 1e-10:
        th = opts.primal_weight_smoothing
        return math.exp(th * math.log(dy / dx) + (1.0 - th) * math.log(omega))
    return omega


def solve_lp(p: Problem, opts: Options = Options(), x_init=None, y_init=None,
             keep_history=False, feasibility=None) -> Result:
    """r^2HPDHG (Algorithm 1) on the scaled LP.  feasibility = "primal" / "dual"
    ends the run on that residual alone (||r_p|| <= eps_abs + eps_rel ||b||, or
    ||r_d|| <= eps_abs + eps_rel ||c||): the polishing runs."""
    ps, Dr, Dc, nA, nQ, eta, omega = prepare(p, opts)
    x = np.zeros(p.n) if x_init is None else np.asarray(x_init, dtype=np.float64) / Dc
    y = np.zeros(p.m) if y_init is None else np.asarray(y_init, dtype=np.float64) / Dr
    xa, ya = x.copy(), y.copy()
    tau, sigma = step_sizes(eta, omega, nA, nQ, opts, False)
    k = 0
    total = 0
    restarts = 0
    r_anchor = None
    r_prev = None
    hist = []
    rlog = []
    while True:
        x_hat, y_hat, _ = pdhg_step_lp(ps, x, y, tau, sigma)
        total += 1
        if total % opts.check_every == 0 or total >= opts.iteration_limit:
            info = kkt(p, Dc * x_hat, Dr * y_hat, opts.eps_abs, opts.eps_rel)
            if keep_history:
                hist.append((total, info["rel_kkt"]))
            done = info["converged"]
            if feasibility == "primal":
                done = info["primal_res"] <= opts.eps_abs + opts.eps_rel * info["b_norm"]
            elif feasibility == "dual":
                done = info["dual_res"] <= opts.eps_abs + opts.eps_rel * info["c_norm"]
            if done or total >= opts.iteration_limit:
                status = "optimal" if done else "iteration_limit"
                return Result(Dc * x_hat, Dr * y_hat, status, total, restarts, info, omega,
                              eta, nA, nQ, Dr, Dc, hist, restart_log=rlog)
            status, cert = infeasibility(p, Dc * (x_hat - xa), Dr * (y_hat - ya), opts)
            if status is not None:
                return Result(Dc * x_hat, Dr * y_hat, status, total, restarts, info, omega,
                              eta, nA, nQ, Dr, Dc, hist, cert, restart_log=rlog)
            r = math.sqrt(omega * float(np.sum((x_hat - x) ** 2))
                          + float(np.sum((y_hat - y) ** 2)) / omega)
            if _restart_decision(r, r_anchor, r_prev, k + 1, total, opts):
                dx = float(np.linalg.norm(x_hat - xa))
                dy = float(np.linalg.norm(y_hat - ya))
                omega = _update_weight(omega, dx, dy, opts)
                rlog.append((total, omega))
                tau, sigma = step_sizes(eta, omega, nA, nQ, opts, False)
                x, y = x_hat, y_hat
                xa, ya = x_hat.copy(), y_hat.copy()
                k = 0
                restarts += 1
                r_anchor = r
                r_prev = r
                continue
            r_prev = r
        g = opts.reflection_gamma
        x, y = halpern(x_hat, x, xa, k, g), halpern(y_hat, y, ya, k, g)
        k += 1


def polish_lp(p: Problem, x, y, opts: Options = Options(), eps_feas_polish: float = 1e-6):
    """Feasibility polishing (Sec. 3.3: the feasibility-only problem, objective
    set to zero, solved by the same method from the current point).  Reading:
    primal phase -- min 0 s.t. the same constraints, from (x, 0), until
    ||r_p|| <= eps (1 + ||b||); dual phase -- the LP with every finite bound set
    to zero (the cones of Y and Lambda unchanged), from (0, y), until
    ||r_d|| <= eps (1 + ||c||).  Infeasibility tests are off in both.  Returns
    (x_polished, y_polished, primal Result, dual Result)."""
    import dataclasses
    o = dataclasses.replace(opts, eps_abs=eps_feas_polish, eps_rel=eps_feas_polish,
                            eps_primal_infeasible=0.0, eps_dual_infeasible=0.0)
    pp = Problem(p.A, np.zeros(p.n), p.lc, p.uc, p.l, p.u)
    rp = solve_lp(pp, o, x_init=x, y_init=np.zeros(p.m), feasibility="primal")
    z = lambda v: np.where(np.isfinite(v), 0.0, v)  # noqa: E731
    pd = Problem(p.A, p.c, z(p.lc), z(p.uc), z(p.l), z(p.u))
    rd = solve_lp(pd, o, x_init=np.zeros(p.n), y_init=y, feasibility="dual")
    return rp.x, rd.y, rp, rd


def solve_qp(p: Problem, opts: Options = Options(), x_init=None, y_init=None,
             keep_history=False, tape=None) -> Result:
    """rAPDHG (Algorithm 2) on the scaled QP.  With a list `tape`, every step
    appends ("step", k, tau, sigma, x, y, xavg, yavg) -- its inner counter,
    step sizes and the scaled state it starts from -- and every restart appends
    ("restart",); oracle.unrolled differentiates along that record."""
    ps, Dr, Dc, nA, nQ, eta, omega = prepare(p, opts)
    x = np.zeros(p.n) if x_init is None else np.asarray(x_init, dtype=np.float64) / Dc
    y = np.zeros(p.m) if y_init is None else np.asarray(y_init, dtype=np.float64) / Dr
    xavg, yavg = x.copy(), y.copy()
    xa, ya = x.copy(), y.copy()
    tau, sigma = step_sizes(eta, omega, nA, nQ, opts, True)
    k = 0
    total = 0
    restarts = 0
    r_anchor = None
    r_prev = None
    hist = []
    rlog = []
    while True:
        if tape is not None:
            tape.append(("step", k, tau, sigma, x.copy(), y.copy(), xavg.copy(), yavg.copy()))
        x, y, xavg, yavg, _ = apdhg_step_qp(ps, x, y, xavg, yavg, k, tau, sigma)
        total += 1
        k += 1
        if total % opts.check_every == 0 or total >= opts.iteration_limit:
            info = kkt(p, Dc * xavg, Dr * yavg, opts.eps_abs, opts.eps_rel)
            if keep_history:
                hist.append((total, info["rel_kkt"]))
            if info["converged"] or total >= opts.iteration_limit:
                status = "optimal" if info["converged"] else "iteration_limit"
                return Result(Dc * xavg, Dr * yavg, status, total, restarts, info, omega,
                              eta, nA, nQ, Dr, Dc, hist, restart_log=rlog)
            r = info["rel_kkt"]
            if _restart_decision(r, r_anchor, r_prev, k, total, opts):
                dx = float(np.linalg.norm(xavg - xa))
                dy = float(np.linalg.norm(yavg - ya))
                omega = _update_weight(omega, dx, dy, opts)
                rlog.append((total, omega))
                tau, sigma = step_sizes(eta, omega, nA, nQ, opts, True)
                x, y = xavg.copy(), yavg.copy()
                xa, ya = xavg.copy(), yavg.copy()
                k = 0
                restarts += 1
                r_anchor = r
                r_prev = r
                if tape is not None:
                    tape.append(("restart",))
                continue
            r_prev = r


def solve(p: Problem, opts: Options = Options(), **kw) -> Result:
    return solve_lp(p, opts, **kw) if p.Q is None else solve_qp(p, opts, **kw)
