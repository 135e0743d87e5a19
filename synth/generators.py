"""Seeded generators for the synthetic workloads.

Every instance is built from a master seed (20241212) and a per-instance seed
``SplitMix64(master ^ i)`` feeding numpy's PCG64.  The shapes follow the paper's
workload families (Sec. 4): sparse LPs with uniform or power-law (Zipf) row
lengths standing in for ``dlr1``-scale sparse LPs, a strictly convex QP with a
diagonal-plus-low-rank Q, a ragged batch of small LPs standing in for the
batched two-stage stochastic LPs, and a dense shared-matrix LP batch standing in
for the dense knapsack relaxation.

Construction of a feasible, bounded LP with a known optimum: pick a primal point
x0 in the box, a dual point y0 and a reduced-cost vector s that together satisfy
the optimality conditions of problem (1), then set the row bounds from A x0 and
the cost c = A^T y0 + s.  The "literal" variant puts x0 strictly inside the box
(so s = 0 and every feasible point is optimal); the "nondegenerate" variant puts
60% of x0 on a bound with strictly complementary reduced costs and makes half of
the inequality rows tight with strictly positive duals.  In both variants the
optimal value equals c^T x0.

Only instance-construction arithmetic lives here (products A x0, A^T y0); no step
of the PDHG method does.
"""
from __future__ import annotations

import numpy as np

MASTER_SEED = 20241212
_MASK64 = (1 << 64) - 1


def _splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014), on Python ints."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def instance_seed(i: int, master: int = MASTER_SEED) -> int:
    return _splitmix64((master ^ int(i)) & _MASK64)


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# ----------------------------------------------------------------------------
# CSR structure
# ----------------------------------------------------------------------------

def zipf_row_lengths(m: int, nnz: int, rng, s: float = 1.5, max_len: int = 10000,
                     n_cols: int | None = None) -> np.ndarray:
    """Row lengths L_i ~ Zipf(s) truncated to [1, max_len], rescaled so that
    sum(L) == nnz exactly (largest-remainder rounding, clamped to
    [1, min(max_len, n_cols)] with the excess or deficit redistributed)."""
    cap = max_len if n_cols is None else min(max_len, n_cols)
    if nnz < m or nnz > m * cap:
        raise ValueError("nnz out of range for the row count")
    k = np.arange(1, max_len + 1, dtype=np.float64)
    pmf = k ** (-s)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    raw = np.searchsorted(cdf, rng.random(m), side="right") + 1
    raw = np.minimum(raw, max_len).astype(np.float64)
    target = raw * (nnz / raw.sum())
    base = np.clip(np.floor(target), 1, cap).astype(np.int64)
    frac = target - np.floor(target)
    deficit = nnz - int(base.sum())
    # Redistribute in rounds so the clamp is always respected.
    while deficit != 0:
        if deficit > 0:
            room = np.flatnonzero(base < cap)
            order = room[np.argsort(-frac[room], kind="stable")]
            take = order[:deficit]
            base[take] += 1
        else:
            room = np.flatnonzero(base > 1)
            order = room[np.argsort(frac[room], kind="stable")]
            take = order[:-deficit]
            base[take] -= 1
        frac[take] = 0.5  # a row touched once is not preferred again
        deficit = nnz - int(base.sum())
    return base


def _distinct_sorted_columns(lengths: np.ndarray, n: int, rng) -> np.ndarray:
    """For each row, `lengths[i]` distinct column indices drawn uniformly from
    [0, n), sorted within the row.  Returns the concatenated column array."""
    m = lengths.shape[0]
    dense_rows = np.flatnonzero(lengths > n // 4)
    sparse_mask = lengths <= n // 4
    need = np.where(sparse_mask, lengths, 0).astype(np.int64)
    keys = np.empty(0, dtype=np.int64)
    while True:
        rows = np.repeat(np.arange(m, dtype=np.int64), need)
        cols = rng.integers(0, n, size=rows.shape[0], dtype=np.int64)
        keys = np.unique(np.concatenate([keys, rows * n + cols]))
        have = np.bincount(keys // n, minlength=m)
        need = np.where(sparse_mask, lengths - have, 0)
        if need.sum() == 0:
            break
    parts = [keys]
    for i in dense_rows:
        cols = np.sort(rng.choice(n, size=int(lengths[i]), replace=False)).astype(np.int64)
        parts.append(i * n + cols)
    keys = np.sort(np.concatenate(parts))
    return (keys % n).astype(np.int32)


def csr_random(m: int, n: int, rng, *, density: float | None = None, nnz: int | None = None,
               rows: str = "bernoulli", zipf_s: float = 1.5, zipf_max: int = 10000,
               min_row: int = 0, scale: float = 1.0):
    """Random CSR matrix with N(0, scale^2) values.

    rows="bernoulli": every entry present independently with probability
    `density` (row length Binomial(n, density), columns uniform without
    replacement), at least `min_row` entries per row.
    rows="zipf": power-law row lengths with exactly `nnz` entries.
    """
    if rows == "bernoulli":
        lengths = rng.binomial(n, density, size=m).astype(np.int64)
        lengths = np.clip(lengths, min(min_row, n), n)
    elif rows == "zipf":
        lengths = zipf_row_lengths(m, nnz, rng, s=zipf_s, max_len=zipf_max, n_cols=n)
    else:
        raise ValueError(rows)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    col = _distinct_sorted_columns(lengths, n, rng)
    val = rng.standard_normal(int(row_ptr[-1])) * scale
    return row_ptr, col, val


def _row_index(row_ptr: np.ndarray) -> np.ndarray:
    m = row_ptr.shape[0] - 1
    return np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))


def _matvec(row_ptr, col, val, x):
    m = row_ptr.shape[0] - 1
    return np.bincount(_row_index(row_ptr), weights=val * x[col], minlength=m)


def _rmatvec(row_ptr, col, val, y, n):
    return np.bincount(col, weights=val * y[_row_index(row_ptr)], minlength=n)


# ----------------------------------------------------------------------------
# LP instances
# ----------------------------------------------------------------------------

def lp_instance(m: int, n: int, *, seed: int, density: float | None = None,
                nnz: int | None = None, rows: str = "bernoulli", lo: float = 0.0,
                hi: float = 10.0, eq_frac: float = 0.5, variant: str = "literal",
                min_row: int = 0, tight_frac: float = 0.5) -> dict:
    """Feasible, bounded LP  min c^T x  s.t.  lc <= A x <= uc,  lo <= x <= hi.

    Rows [0, m_eq) are equalities lc = uc = A x0; rows [m_eq, m) are
    inequalities lc <= A x with uc = +inf.  In the nondegenerate variant exactly
    round(tight_frac * (m - m_eq)) inequality rows are tight at x0.
    """
    rng = _rng(seed)
    row_ptr, col, val = csr_random(m, n, rng, density=density, nnz=nnz, rows=rows,
                                   min_row=min_row)
    m_eq = int(round(eq_frac * m))
    l = np.full(n, lo, dtype=np.float64)
    u = np.full(n, hi, dtype=np.float64)
    s = np.zeros(n)
    if variant == "literal":
        x0 = lo + (hi - lo) * rng.random(n)
    elif variant == "nondegenerate":
        x0 = lo + (hi - lo) * rng.random(n)
        perm = rng.permutation(n)
        at_l = perm[: int(0.3 * n)]
        at_u = perm[int(0.3 * n): int(0.6 * n)]
        x0[at_l] = lo
        x0[at_u] = hi
        s[at_l] = rng.uniform(0.1, 1.0, size=at_l.shape[0])
        s[at_u] = -rng.uniform(0.1, 1.0, size=at_u.shape[0])
    else:
        raise ValueError(variant)
    ax0 = _matvec(row_ptr, col, val, x0)
    lc = np.empty(m)
    uc = np.empty(m)
    y0 = np.zeros(m)
    lc[:m_eq] = ax0[:m_eq]
    uc[:m_eq] = ax0[:m_eq]
    y0[:m_eq] = rng.standard_normal(m_eq)
    n_ineq = m - m_eq
    slack = rng.uniform(0.0, 1.0, size=n_ineq)
    if variant == "nondegenerate":
        tight = np.zeros(n_ineq, dtype=bool)
        tight[rng.permutation(n_ineq)[:int(round(tight_frac * n_ineq))]] = True
        slack[tight] = 0.0
        y0[m_eq:][tight] = np.abs(rng.standard_normal(int(tight.sum())))
    lc[m_eq:] = ax0[m_eq:] - slack
    uc[m_eq:] = np.inf
    c = _rmatvec(row_ptr, col, val, y0, n) + s
    return dict(kind="lp", m=m, n=n, nnz=int(row_ptr[-1]), row_ptr=row_ptr, col=col,
                val=val, c=c, lc=lc, uc=uc, l=l, u=u, x0=x0, y0=y0, s=s,
                opt_value=float(c @ x0), variant=variant, m_eq=m_eq)


# ----------------------------------------------------------------------------
# QP instance: Q = diag(D) + F F^T, equality rows b = A x0, box [lo, hi]
# ----------------------------------------------------------------------------

def qp_instance(n: int, m: int, *, seed: int, a_density: float = 1e-4, f_cols: int = 32,
                f_density: float = 0.01, lo: float = -1.0, hi: float = 1.0,
                min_row: int = 0) -> dict:
    rng = _rng(seed)
    row_ptr, col, val = csr_random(m, n, rng, density=a_density, min_row=min_row)
    f_ptr, f_col, f_val = csr_random(n, f_cols, rng, density=f_density)
    D = rng.uniform(0.1, 1.0, size=n)
    x0 = rng.uniform(lo, hi, size=n)
    b = _matvec(row_ptr, col, val, x0)
    c = rng.standard_normal(n)
    x_target = rng.uniform(lo, hi, size=n)
    return dict(kind="qp", m=m, n=n, nnz=int(row_ptr[-1]), row_ptr=row_ptr, col=col, val=val,
                c=c, lc=b.copy(), uc=b.copy(), l=np.full(n, lo), u=np.full(n, hi),
                D=D, f_cols=f_cols, f_row_ptr=f_ptr, f_col=f_col, f_val=f_val,
                x0=x0, x_target=x_target)


def qp_sparse_q_instance(n: int, m: int, *, seed: int, a_density: float = 1e-4,
                         b_density: float = 2e-4, lo: float = -1.0, hi: float = 1.0,
                         min_row: int = 0) -> dict:
    """Convex QP with a general sparse Q = B B^T + diag(U[0.1, 1]) (B n x n with
    N(0, 1) entries at `b_density`), stored as CSR with both triangles and sorted
    columns; A, the box, b = A x0 and c ~ N(0, 1) as in qp_instance."""
    import scipy.sparse as sp
    rng = _rng(seed)
    row_ptr, col, val = csr_random(m, n, rng, density=a_density, min_row=min_row)
    b_ptr, b_col, b_val = csr_random(n, n, rng, density=b_density)
    Bm = sp.csr_matrix((b_val, b_col, b_ptr), shape=(n, n))
    Q = sp.csr_matrix(Bm @ Bm.T + sp.diags(rng.uniform(0.1, 1.0, size=n)))
    Q.sort_indices()
    x0 = rng.uniform(lo, hi, size=n)
    b = _matvec(row_ptr, col, val, x0)
    c = rng.standard_normal(n)
    x_target = rng.uniform(lo, hi, size=n)
    return dict(kind="qp", m=m, n=n, nnz=int(row_ptr[-1]), row_ptr=row_ptr, col=col, val=val,
                c=c, lc=b.copy(), uc=b.copy(), l=np.full(n, lo), u=np.full(n, hi),
                q_row_ptr=Q.indptr.astype(np.int64), q_col=Q.indices.astype(np.int32),
                q_val=Q.data.astype(np.float64), x0=x0, x_target=x_target)


def grid_shortest_path_lp(k: int, B: int = 1, *, seed: int = MASTER_SEED,
                          lo: float = 0.1, hi: float = 1.0) -> dict:
    """Node-arc shortest-path LP on a k x k grid (the 2-D grid shortest path LP of
    the paper's Warcraft experiment, Sec. 4): nodes are cells, arcs join each cell
    to its up to 8 neighbours, flow conservation with supply 1 at the top-left
    cell (source) and demand 1 at the bottom-right one (sink), 0 <= x <= 1.  B
    cost vectors: node costs w_b ~ U[lo, hi] per cell, arc (u -> v) costs w_b[v]
    (the cost of entering v).  Rows: nodes (row v = out-flow minus in-flow);
    columns: arcs, listed cell by cell."""
    rng = _rng(seed)
    V = k * k
    tails, heads = [], []
    for r in range(k):
        for c in range(k):
            for dr in (-1, 0, 1):
                for dc in (-1, 0, 1):
                    rr, cc = r + dr, c + dc
                    if (dr or dc) and 0 <= rr < k and 0 <= cc < k:
                        tails.append(r * k + c)
                        heads.append(rr * k + cc)
    tails = np.asarray(tails, dtype=np.int64)
    heads = np.asarray(heads, dtype=np.int64)
    E = len(tails)
    # CSR by node: +1 on the arcs leaving it, -1 on the arcs entering it
    rows = np.concatenate([tails, heads])
    cols = np.concatenate([np.arange(E), np.arange(E)])
    vals = np.concatenate([np.ones(E), -np.ones(E)])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(V + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=V), out=row_ptr[1:])
    b = np.zeros(V)
    b[0], b[V - 1] = 1.0, -1.0
    W = rng.uniform(lo, hi, size=(B, V))
    return dict(kind="lp", m=V, n=E, nnz=2 * E, row_ptr=row_ptr, col=cols.astype(np.int32),
                val=vals, lc=b.copy(), uc=b.copy(), l=np.zeros(E), u=np.ones(E),
                C=W[:, heads], W=W, tails=tails, heads=heads, k=k, B=B)


# ----------------------------------------------------------------------------
# Ragged batch of independent LPs (packed CSR)
# ----------------------------------------------------------------------------

def ragged_lp_instances(B: int, which, *, seed: int = MASTER_SEED, m_lo: int = 50,
                        m_hi: int = 2000, density: float = 0.01, lo: float = 0.0,
                        hi: float = 10.0, variant: str = "literal") -> list:
    """Instances `which` (indices into 0..B-1) of the B-instance ragged batch
    below, each exactly as ragged_lp_batch builds it, without building the rest."""
    ms = _rng(seed).integers(m_lo, m_hi + 1, size=B)
    return [lp_instance(int(ms[i]), int(2 * ms[i]), seed=instance_seed(i, seed),
                        density=density, lo=lo, hi=hi, variant=variant) for i in which]


def ragged_lp_batch(B: int, *, seed: int = MASTER_SEED, m_lo: int = 50, m_hi: int = 2000,
                    density: float = 0.01, lo: float = 0.0, hi: float = 10.0,
                    variant: str = "literal") -> dict:
    """B LPs with m_i ~ U{m_lo..m_hi}, n_i = 2 m_i, packed back to back.

    Packed layout: row_ptr is global over the concatenated rows (length
    sum(m)+1), column indices are local to their instance, vectors are
    concatenated; m_off / n_off / nnz_off are exclusive prefix offsets.
    """
    insts = ragged_lp_instances(B, range(B), seed=seed, m_lo=m_lo, m_hi=m_hi, density=density,
                                lo=lo, hi=hi, variant=variant)
    m_off = np.zeros(B + 1, dtype=np.int64)
    n_off = np.zeros(B + 1, dtype=np.int64)
    nnz_off = np.zeros(B + 1, dtype=np.int64)
    np.cumsum([d["m"] for d in insts], out=m_off[1:])
    np.cumsum([d["n"] for d in insts], out=n_off[1:])
    np.cumsum([d["nnz"] for d in insts], out=nnz_off[1:])
    row_ptr = np.concatenate([[0]] + [d["row_ptr"][1:] + nnz_off[i] for i, d in enumerate(insts)])
    cat = lambda k: np.concatenate([d[k] for d in insts])  # noqa: E731
    return dict(kind="lp_batch", B=B, m_off=m_off, n_off=n_off, nnz_off=nnz_off,
                row_ptr=row_ptr.astype(np.int64), col=cat("col"), val=cat("val"),
                c=cat("c"), lc=cat("lc"), uc=cat("uc"), l=cat("l"), u=cat("u"),
                opt_value=np.array([d["opt_value"] for d in insts]), instances=insts)


# ----------------------------------------------------------------------------
# Dense shared-matrix LP batch
# ----------------------------------------------------------------------------

def shared_dense_lp_batch(m: int, n: int, B: int, *, seed: int = MASTER_SEED,
                          lo: float = 0.0, hi: float = 1.0, dtype=np.float32,
                          bound_frac: float = 0.0) -> dict:
    """Dense A (m x n) with N(0, 1/n) entries (std 1/sqrt(n)); equality rows
    b = A x0 with x0 ~ U[lo, hi]; B cost vectors c_k = A^T y_k + s_k, y_k ~ N(0,1).

    bound_frac = 0: s_k = 0 (every feasible point is optimal, value c_k^T x0).
    bound_frac > 0: that fraction of x0's coordinates is moved to a bound (half
    to lo, half to hi) and s_k carries reduced costs of the right sign there
    (U[0.1, 1] at lo, -U[0.1, 1] at hi), so x0 is the unique-valued optimum and
    (y_k, s_k) a dual certificate."""
    rng = _rng(seed)
    A = (rng.standard_normal((m, n), dtype=np.float32) / np.float32(np.sqrt(n))).astype(dtype)
    x0 = rng.uniform(lo, hi, size=n)
    Y = rng.standard_normal((B, m))
    if bound_frac > 0:
        r = rng.random(n)
        at_lo = r < 0.5 * bound_frac
        at_hi = (r >= 0.5 * bound_frac) & (r < bound_frac)
        x0[at_lo], x0[at_hi] = lo, hi
    A64 = A.astype(np.float64)
    b = A64 @ x0
    C = Y @ A64
    del A64
    if bound_frac > 0:
        C[:, at_lo] += rng.uniform(0.1, 1.0, size=(B, int(at_lo.sum())))
        C[:, at_hi] -= rng.uniform(0.1, 1.0, size=(B, int(at_hi.sum())))
    return dict(kind="lp_shared", m=m, n=n, B=B, A=A, b=b, C=C, x0=x0, Y=Y,
                l=np.full(n, lo), u=np.full(n, hi), opt_value=C @ x0)


# ----------------------------------------------------------------------------
# Seeded iterate states (for one-iteration parity from an identical state)
# ----------------------------------------------------------------------------

def random_state(n: int, m: int, *, seed: int, lo=None, hi=None) -> dict:
    rng = _rng(seed)
    def vec(k, a, b):
        return a + (b - a) * rng.random(k)
    xl = -1.0 if lo is None else lo
    xh = 1.0 if hi is None else hi
    return dict(x=vec(n, xl, xh), y=rng.standard_normal(m), x_anchor=vec(n, xl, xh),
                y_anchor=rng.standard_normal(m), xbar=vec(n, xl, xh),
                ybar=rng.standard_normal(m))


# ----------------------------------------------------------------------------
# Dense multi-dimensional knapsack relaxation (one instance)
# ----------------------------------------------------------------------------

def knapsack_lp(d: int, m: int, *, seed: int = MASTER_SEED, frac: float = 0.25) -> dict:
    """LP relaxation of a d-dimensional knapsack over m items:
        min -v^T x  s.t.  W x <= b,  0 <= x <= 1,
    W ~ U[0, 1] dense (d x m, FP32, row-major), item values v ~ U[0, 1], and
    capacities b = frac * W 1 (each dimension holds a fraction of all items).
    The objective is the negated value, so the LP is a maximisation of value as
    the knapsack relaxation intends."""
    rng = _rng(seed)
    W = rng.random((d, m), dtype=np.float32)
    v = rng.random(m)
    b = frac * W.astype(np.float64).sum(axis=1)
    return dict(kind="knapsack", d=d, m_items=m, A=W, c=-v, lc=np.full(d, -np.inf), uc=b,
                l=np.zeros(m), u=np.ones(m))
