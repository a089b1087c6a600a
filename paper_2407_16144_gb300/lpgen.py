"""Seeded synthetic LP generators.

Every LP here has the general form used throughout the package,

    min  c^T x + offset   s.t.   A x = b   (rows 0 .. m_eq-1)
                                 G x >= h  (rows m_eq .. m-1)
                                 l <= x <= u  (entries of l, u may be -inf / +inf),

stored as one CSR matrix K = [A; G] with rhs q = [b; h].  The paper's standard form
(Section 2, eq. lp: min c^T x, Ax = b, x >= 0) is the special case m_ineq = 0, l = 0, u = +inf.

The module holds only input generation (random draws and the algebra that plants a known
optimum, a Farkas vector or an unbounded ray).  It contains none of the solver's
arithmetic, so both the CUDA path and the FP64 oracle can draw their inputs from it.
All generators use numpy's PCG64 ``default_rng(seed)`` so an input is fixed by its seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

INF = np.inf


@dataclasses.dataclass
class LP:
    """A general-form LP in CSR layout (see module docstring)."""

    m_eq: int
    m_ineq: int
    n: int
    row_ptr: np.ndarray  # int64, m+1
    col_idx: np.ndarray  # int32, nnz, sorted within each row, no duplicates
    val: np.ndarray      # float64, nnz
    c: np.ndarray        # float64, n
    q: np.ndarray        # float64, m  (b then h)
    l: np.ndarray        # float64, n  (may hold -inf)
    u: np.ndarray        # float64, n  (may hold +inf)
    obj_offset: float = 0.0
    name: str = ""
    # planted data (None when not planted)
    x_star: Optional[np.ndarray] = None
    y_star: Optional[np.ndarray] = None
    farkas_y: Optional[np.ndarray] = None
    ray_d: Optional[np.ndarray] = None

    @property
    def m(self) -> int:
        return self.m_eq + self.m_ineq

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        """Dense copy of K (small problems only)."""
        K = np.zeros((self.m, self.n))
        for i in range(self.m):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            K[i, self.col_idx[s:e]] = self.val[s:e]
        return K

    def planted_objective(self) -> float:
        assert self.x_star is not None
        return float(self.c @ self.x_star + self.obj_offset)


def coo_to_csr(m: int, n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray):
    """Sort COO triplets into CSR (row-major, columns ascending).  Duplicates are not merged:
    callers never produce them."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order]
    vals = np.asarray(vals, dtype=np.float64)[order]
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), vals


def csr_matvec(row_ptr, col_idx, val, x):
    """y = K x for CSR K (used only to plant right-hand sides)."""
    m = len(row_ptr) - 1
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    return np.bincount(rows, weights=val * x[col_idx], minlength=m)


def csr_rmatvec(row_ptr, col_idx, val, y, n):
    """x = K^T y for CSR K (used only to plant objectives)."""
    m = len(row_ptr) - 1
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    return np.bincount(col_idx, weights=val * y[rows], minlength=n)


def _fix_empty_rows(rng, m, n, rows, cols, vals):
    """Give every empty row one random entry so no constraint is vacuous."""
    present = np.zeros(m, dtype=bool)
    present[rows] = True
    empty = np.flatnonzero(~present)
    if len(empty):
        extra_c = rng.integers(0, n, size=len(empty))
        extra_v = rng.standard_normal(len(empty))
        rows = np.concatenate([rows, empty])
        cols = np.concatenate([cols, extra_c])
        vals = np.concatenate([vals, extra_v])
    return rows, cols, vals


def _uniform_positions(rng, m: int, degrees: np.ndarray):
    """For each column j draw degrees[j] distinct row indices uniformly from [0, m).
    Returns COO (rows, cols) arrays."""
    all_rows, all_cols = [], []
    for d in np.unique(degrees):
        d = int(d)
        cols_d = np.flatnonzero(degrees == d)
        k = len(cols_d)
        if d == 0:
            continue
        if 4 * d * d <= m:
            # duplicates are rare (birthday bound < ~1/8): draw with replacement and redraw
            # the columns that hold a duplicate row
            r = rng.integers(0, m, size=(k, d))
            while d > 1:
                s = np.sort(r, axis=1)
                bad = np.flatnonzero((s[:, 1:] == s[:, :-1]).any(axis=1))
                if len(bad) == 0:
                    break
                r[bad] = rng.integers(0, m, size=(len(bad), d))
        else:
            r = np.stack([rng.choice(m, size=d, replace=False) for _ in range(k)])
        all_rows.append(r.reshape(-1))
        all_cols.append(np.repeat(cols_d, d))
    return np.concatenate(all_rows), np.concatenate(all_cols)


# ---------------------------------------------------------------------------------------------
# C1: standard-form LP with a planted optimum (200 x 500, 5 nnz per column)
# ---------------------------------------------------------------------------------------------

def make_standard_planted(seed: int = 0, m: int = 200, n: int = 500, col_nnz: int = 5,
                          zero_frac: float = 0.4) -> LP:
    """Standard-form LP (A x = b, x >= 0) with a planted primal-dual optimum.

    A has exactly ``col_nnz`` distinct uniformly placed rows per column with N(0,1) values
    (empty rows get one extra entry).  x* has ``zero_frac`` zeros, the rest U(0.5, 2);
    b = A x*; y* ~ N(0,1); s*_j = 0 where x*_j > 0 and U(0.5, 2) where x*_j = 0;
    c = A^T y* + s*, so (x*, y*) satisfies the KKT conditions exactly.
    """
    rng = np.random.default_rng(seed)
    deg = np.full(n, min(col_nnz, m), dtype=np.int64)
    rows, cols = _uniform_positions(rng, m, deg)
    vals = rng.standard_normal(len(rows))
    rows, cols, vals = _fix_empty_rows(rng, m, n, rows, cols, vals)
    row_ptr, col_idx, val = coo_to_csr(m, n, rows, cols, vals)
    x_star = rng.uniform(0.5, 2.0, size=n)
    zeros = rng.choice(n, size=int(round(zero_frac * n)), replace=False)
    x_star[zeros] = 0.0
    b = csr_matvec(row_ptr, col_idx, val, x_star)
    y_star = rng.standard_normal(m)
    s_star = np.zeros(n)
    s_star[zeros] = rng.uniform(0.5, 2.0, size=len(zeros))
    c = csr_rmatvec(row_ptr, col_idx, val, y_star, n) + s_star
    return LP(m_eq=m, m_ineq=0, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, c=c, q=b,
              l=np.zeros(n), u=np.full(n, INF), name=f"standard_planted_{m}x{n}_s{seed}",
              x_star=x_star, y_star=y_star)


def make_c1(seed: int = 0) -> LP:
    """The 200 x 500 planted standard-form LP (about 2,500 nonzeros)."""
    return make_standard_planted(seed=seed, m=200, n=500, col_nnz=5)


# ---------------------------------------------------------------------------------------------
# C2: general-form LP, power-law column degrees, mixed bounds, planted optimum
# ---------------------------------------------------------------------------------------------

def _powerlaw_degrees(rng, n: int, alpha: float, d_max: int, mean_target: float) -> np.ndarray:
    """Column degrees from a discrete power law P(d) ~ d^-alpha on [d_min, d_max], with the
    integer d_min whose mean is closest to ``mean_target``, then a final multiplicative
    adjustment of a random subset so the total is close to n * mean_target."""
    best = None
    for d_min in range(1, 64):
        d = np.arange(d_min, d_max + 1, dtype=np.float64)
        p = d ** (-alpha)
        p /= p.sum()
        mean = float((d * p).sum())
        if best is None or abs(mean - mean_target) < abs(best[1] - mean_target):
            best = (d_min, mean, d, p)
    d_min, mean, d, p = best
    deg = rng.choice(d.astype(np.int64), size=n, p=p)
    # nudge the total towards n * mean_target by adding/removing one at random columns
    target = int(round(n * mean_target))
    diff = target - int(deg.sum())
    if diff > 0:
        idx = rng.choice(n, size=min(diff, n), replace=False)
        deg[idx] = np.minimum(deg[idx] + 1, d_max)
    elif diff < 0:
        cand = np.flatnonzero(deg > d_min)
        idx = rng.choice(cand, size=min(-diff, len(cand)), replace=False)
        deg[idx] -= 1
    return deg


def make_general_planted(seed: int = 1, m_eq: int = 70_000, m_ineq: int = 30_000,
                         n: int = 250_000, mean_col_nnz: float = 10.0, alpha: float = 2.1,
                         d_max: int = 5000) -> LP:
    """General-form LP with a planted optimum (the 100k x 250k, ~2.5M nnz workload at the
    default sizes; smaller sizes give the same structure for tests).

    Columns: power-law degrees (alpha, max d_max), uniform distinct row positions.
    Values: 30% +-1, 30% +-U{1..10}, 40% +-lognormal(0,1), random signs.
    Bounds: 50% [0, inf), 30% [l, u] with l ~ U(-10, 0), u = l + U(1, 10), 20% free.
    Planted x*: [0,inf) columns 40% at 0 else U(0.5, 2); boxes 1/3 at l, 1/3 at u,
    1/3 interior; free columns N(0,1).  y*_eq ~ N(0,1); half the >= rows active
    (y* ~ U(0.5, 2), h = G x*) and half inactive (y* = 0, h = G x* - U(0.5, 2)).
    Reduced cost lambda* is U(0.5, 2) at an active lower bound, -U(0.5, 2) at an active
    upper bound, 0 otherwise; c = K^T y* + lambda*.
    """
    rng = np.random.default_rng(seed)
    m = m_eq + m_ineq
    d_max = min(d_max, m)
    deg = _powerlaw_degrees(rng, n, alpha, d_max, mean_col_nnz)
    rows, cols = _uniform_positions(rng, m, deg)
    nz = len(rows)
    kind = rng.random(nz)
    mag = np.where(kind < 0.3, 1.0,
                   np.where(kind < 0.6, rng.integers(1, 11, size=nz).astype(np.float64),
                            rng.lognormal(0.0, 1.0, size=nz)))
    sign = np.where(rng.random(nz) < 0.5, -1.0, 1.0)
    vals = mag * sign
    rows, cols, vals = _fix_empty_rows(rng, m, n, rows, cols, vals)
    row_ptr, col_idx, val = coo_to_csr(m, n, rows, cols, vals)

    btype = rng.random(n)
    lower = btype < 0.5
    boxed = (btype >= 0.5) & (btype < 0.8)
    free = btype >= 0.8
    l = np.full(n, -INF)
    u = np.full(n, INF)
    l[lower] = 0.0
    lb = rng.uniform(-10.0, 0.0, size=n)
    ub = lb + rng.uniform(1.0, 10.0, size=n)
    l[boxed] = lb[boxed]
    u[boxed] = ub[boxed]

    x_star = np.zeros(n)
    lam = np.zeros(n)
    # [0, inf)
    li = np.flatnonzero(lower)
    at0 = rng.random(len(li)) < 0.4
    x_star[li[~at0]] = rng.uniform(0.5, 2.0, size=int((~at0).sum()))
    lam[li[at0]] = rng.uniform(0.5, 2.0, size=int(at0.sum()))
    # boxes
    bi = np.flatnonzero(boxed)
    which = rng.integers(0, 3, size=len(bi))
    x_star[bi] = rng.uniform(l[bi], u[bi])
    atl = bi[which == 0]
    atu = bi[which == 1]
    x_star[atl] = l[atl]
    x_star[atu] = u[atu]
    lam[atl] = rng.uniform(0.5, 2.0, size=len(atl))
    lam[atu] = -rng.uniform(0.5, 2.0, size=len(atu))
    # free
    fi = np.flatnonzero(free)
    x_star[fi] = rng.standard_normal(len(fi))

    Kx = csr_matvec(row_ptr, col_idx, val, x_star)
    y_star = np.zeros(m)
    y_star[:m_eq] = rng.standard_normal(m_eq)
    active = rng.random(m_ineq) < 0.5
    y_ineq = np.zeros(m_ineq)
    y_ineq[active] = rng.uniform(0.5, 2.0, size=int(active.sum()))
    y_star[m_eq:] = y_ineq
    q = Kx.copy()
    slack = rng.uniform(0.5, 2.0, size=m_ineq)
    q[m_eq:] = np.where(active, Kx[m_eq:], Kx[m_eq:] - slack)
    c = csr_rmatvec(row_ptr, col_idx, val, y_star, n) + lam
    return LP(m_eq=m_eq, m_ineq=m_ineq, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, c=c,
              q=q, l=l, u=u, name=f"general_planted_{m}x{n}_s{seed}", x_star=x_star,
              y_star=y_star)


def make_c2(seed: int = 1, scale: float = 1.0) -> LP:
    """The 100k x 250k (70% equality rows, ~2.5M nnz) planted general-form LP; ``scale``
    shrinks every dimension for tests while keeping the structure."""
    m_eq = max(1, int(round(70_000 * scale)))
    m_ineq = max(1, int(round(30_000 * scale)))
    n = max(2, int(round(250_000 * scale)))
    return make_general_planted(seed=seed, m_eq=m_eq, m_ineq=m_ineq, n=n,
                                d_max=max(2, int(round(5000 * min(1.0, scale * 4)))))


# ---------------------------------------------------------------------------------------------
# C3: multicommodity flow
# ---------------------------------------------------------------------------------------------

def make_multicommodity_flow(seed: int = 2, nodes: int = 250_000, arcs: int = 2_000_000,
                             commodities: int = 20) -> LP:
    """Multicommodity min-cost flow on a random digraph: a random Hamiltonian cycle (so the
    graph is strongly connected) plus arcs - nodes uniform arcs u -> v, u != v, numbered in
    forward-star order (sorted by tail node, then head node).  Variables
    f_{k,a} >= 0 (column k * arcs + a).  Rows: flow conservation N f_k = s_k for every commodity
    and node (equality, row k * nodes + v, +1 on arcs leaving v and -1 on arcs entering it), then
    one shared capacity row per arc, -sum_k f_{k,a} >= -cap_a.  Arc costs U[1, 100] are shared by
    the commodities, capacities U[5, 50].  The supplies come from a planted flow
    f*_{k,a} ~ U(0, cap_a / commodities), so the LP is feasible; its optimum is not planted.
    Every coefficient is +-1 (exact in any floating type)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(nodes)
    tail = np.empty(arcs, dtype=np.int64)
    head = np.empty(arcs, dtype=np.int64)
    tail[:nodes] = perm
    head[:nodes] = np.roll(perm, -1)
    extra = arcs - nodes
    u = rng.integers(0, nodes, size=extra)
    v = rng.integers(0, nodes - 1, size=extra)
    v = v + (v >= u)                                   # uniform over v != u
    tail[nodes:] = u
    head[nodes:] = v
    # arcs numbered in forward-star order (by tail, then head), as a graph file lists them
    order = np.lexsort((head, tail))
    tail, head = tail[order], head[order]
    cost = rng.uniform(1.0, 100.0, size=arcs)
    cap = rng.uniform(5.0, 50.0, size=arcs)
    # one commodity's node-arc incidence in CSR (rows = nodes, sorted columns)
    rows1 = np.concatenate([tail, head])
    cols1 = np.concatenate([np.arange(arcs), np.arange(arcs)])
    vals1 = np.concatenate([np.ones(arcs), -np.ones(arcs)])
    order = np.lexsort((cols1, rows1))
    rows1, cols1, vals1 = rows1[order], cols1[order], vals1[order]
    ptr1 = np.zeros(nodes + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows1, minlength=nodes), out=ptr1[1:])
    del rows1, order
    nnz1 = 2 * arcs
    K = commodities
    m_eq, m_ineq, n = K * nodes, arcs, K * arcs
    nnz = K * nnz1 + K * arcs
    row_ptr = np.empty(m_eq + m_ineq + 1, dtype=np.int64)
    col_idx = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    for k in range(K):
        row_ptr[k * nodes:(k + 1) * nodes] = ptr1[:-1] + k * nnz1
        col_idx[k * nnz1:(k + 1) * nnz1] = cols1 + k * arcs
        val[k * nnz1:(k + 1) * nnz1] = vals1
    base = K * nnz1
    row_ptr[m_eq:m_eq + m_ineq] = base + K * np.arange(arcs, dtype=np.int64)
    row_ptr[-1] = nnz
    cap_cols = (np.arange(K, dtype=np.int64)[None, :] * arcs + np.arange(arcs)[:, None])
    col_idx[base:] = cap_cols.reshape(-1)
    val[base:] = -1.0
    del cap_cols
    # planted feasible flow and the supplies it implies
    f_star = rng.uniform(0.0, 1.0, size=(K, arcs)) * (cap / K)[None, :]
    supply = np.zeros((K, nodes))
    for k in range(K):
        supply[k] = (np.bincount(tail, weights=f_star[k], minlength=nodes) -
                     np.bincount(head, weights=f_star[k], minlength=nodes))
    q = np.concatenate([supply.reshape(-1), -cap])
    c = np.tile(cost, K)
    return LP(m_eq=m_eq, m_ineq=m_ineq, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, c=c,
              q=q, l=np.zeros(n), u=np.full(n, INF),
              name=f"multicommodity_{commodities}x{nodes}n{arcs}a_s{seed}",
              x_star=f_star.reshape(-1))


# ---------------------------------------------------------------------------------------------
# C4: infeasible LPs with planted certificates
# ---------------------------------------------------------------------------------------------

def make_primal_infeasible(seed: int = 3, m: int = 50_000, n: int = 100_000,
                           col_nnz: int = 6) -> LP:
    """Standard-form LP made primal infeasible by a planted Farkas vector y_F:
    A^T y_F <= 0 (columns whose product is positive are negated) and b^T y_F = 1."""
    rng = np.random.default_rng(seed)
    deg = np.full(n, min(col_nnz, m), dtype=np.int64)
    rows, cols = _uniform_positions(rng, m, deg)
    vals = rng.standard_normal(len(rows))
    rows, cols, vals = _fix_empty_rows(rng, m, n, rows, cols, vals)
    row_ptr, col_idx, val = coo_to_csr(m, n, rows, cols, vals)
    y_f = rng.standard_normal(m)
    aty = csr_rmatvec(row_ptr, col_idx, val, y_f, n)
    flip = aty > 0
    val = np.where(flip[col_idx], -val, val)
    aty = csr_rmatvec(row_ptr, col_idx, val, y_f, n)
    x_bar = rng.uniform(0.0, 1.0, size=n)
    gamma = (1.0 - float(x_bar @ aty)) / float(y_f @ y_f)
    b = csr_matvec(row_ptr, col_idx, val, x_bar) + gamma * y_f
    c = rng.standard_normal(n)
    return LP(m_eq=m, m_ineq=0, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, c=c, q=b,
              l=np.zeros(n), u=np.full(n, INF), name=f"primal_infeasible_{m}x{n}_s{seed}",
              farkas_y=y_f)


def make_dual_infeasible(seed: int = 3, m: int = 50_000, n: int = 100_000, col_nnz: int = 6,
                         support_frac: float = 0.01) -> LP:
    """Standard-form LP that is primal feasible but unbounded along a planted ray d >= 0
    (support ``support_frac``, U(0.5, 2)): A d = 0 and c^T d = -1."""
    rng = np.random.default_rng(seed + 100)
    deg = np.full(n, min(col_nnz, m), dtype=np.int64)
    rows, cols = _uniform_positions(rng, m, deg)
    vals = rng.standard_normal(len(rows))
    rows, cols, vals = _fix_empty_rows(rng, m, n, rows, cols, vals)
    row_ptr, col_idx, val = coo_to_csr(m, n, rows, cols, vals)
    k = max(2, int(round(support_frac * n)))
    supp = np.sort(rng.choice(n, size=k, replace=False))
    d = np.zeros(n)
    d[supp] = rng.uniform(0.5, 2.0, size=k)
    # for every row touching the support, reset one support coefficient so row . d = 0
    in_supp = np.zeros(n, dtype=bool)
    in_supp[supp] = True
    val = val.copy()
    for i in range(m):
        s, e = row_ptr[i], row_ptr[i + 1]
        js = col_idx[s:e]
        mask = in_supp[js]
        if not mask.any():
            continue
        pos = s + np.flatnonzero(mask)
        total = float(val[pos] @ d[col_idx[pos]])
        p0 = pos[0]
        rest = total - val[p0] * d[col_idx[p0]]
        val[p0] = -rest / d[col_idx[p0]]
        if val[p0] == 0.0:
            val[p0] = 0.0  # an explicit zero keeps the pattern; harmless
    x_bar = rng.uniform(0.0, 1.0, size=n)
    b = csr_matvec(row_ptr, col_idx, val, x_bar)
    c = rng.standard_normal(n)
    c[supp] += (-1.0 - float(c @ d)) * d[supp] / float(d[supp] @ d[supp])
    return LP(m_eq=m, m_ineq=0, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, c=c, q=b,
              l=np.zeros(n), u=np.full(n, INF), name=f"dual_infeasible_{m}x{n}_s{seed}",
              ray_d=d)


def make_dual_infeasible_twin(seed: int = 3, m: int = 50_000, n: int = 100_000,
                              col_nnz: int = 6) -> LP:
    """The LP dual of ``make_primal_infeasible(seed, m, n)``'s matrix, made dual infeasible with
    the planted Farkas vector y_F as its unbounded ray.  Variables w (m, free); n inequality rows
    -A^T w >= -(A^T y_bar + s) with y_bar ~ N(0, 1) and s ~ U(0, 1), so w = y_bar is feasible;
    objective min -b^T w.  Along d = y_F: -A^T d >= 0 and -b^T d = -1."""
    p = make_primal_infeasible(seed, m, n, col_nnz)
    rng = np.random.default_rng(seed + 200)
    y_bar = rng.standard_normal(m)
    s = rng.uniform(0.0, 1.0, size=n)
    aty = csr_rmatvec(p.row_ptr, p.col_idx, p.val, y_bar, n)
    # transpose of A by a stable sort on the column index (rows of A^T in order)
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(p.row_ptr))
    order = np.argsort(p.col_idx, kind="stable")
    t_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(p.col_idx, minlength=n), out=t_ptr[1:])
    return LP(m_eq=0, m_ineq=n, n=m, row_ptr=t_ptr, col_idx=rows[order].astype(np.int32),
              val=-p.val[order], c=-p.q, q=-(aty + s), l=np.full(m, -INF), u=np.full(m, INF),
              name=f"dual_infeasible_twin_{n}x{m}_s{seed}", ray_d=p.farkas_y.copy())


# ---------------------------------------------------------------------------------------------
# Tiny LPs for brute-force checks
# ---------------------------------------------------------------------------------------------

def make_tiny_standard(seed: int, m: int = 3, n: int = 6, density: float = 0.7) -> LP:
    """Small dense-ish standard-form LP that is feasible (b = A x_bar, x_bar >= 0) and bounded
    (c = A^T y + s with s >= 0), suitable for vertex enumeration."""
    rng = np.random.default_rng(10_000 + seed)
    while True:
        Kd = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
        if np.linalg.matrix_rank(Kd) == m and (Kd != 0).any(axis=0).all():
            break
    x_bar = rng.uniform(0.0, 2.0, size=n)
    b = Kd @ x_bar
    y = rng.standard_normal(m)
    s = rng.uniform(0.1, 2.0, size=n)
    c = Kd.T @ y + s
    rows, cols = np.nonzero(Kd)
    row_ptr, col_idx, val = coo_to_csr(m, n, rows, cols, Kd[rows, cols])
    return LP(m_eq=m, m_ineq=0, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, c=c, q=b,
              l=np.zeros(n), u=np.full(n, INF), name=f"tiny_{m}x{n}_s{seed}")


def make_tiny_general(seed: int, m_eq: int = 2, m_ineq: int = 2, n: int = 5) -> LP:
    """Small general-form LP (equalities, >= rows, mixed finite/infinite bounds) that is
    feasible and has finite bounds on every column, so it is bounded."""
    rng = np.random.default_rng(20_000 + seed)
    m = m_eq + m_ineq
    Kd = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.8)
    for j in range(n):
        if not Kd[:, j].any():
            Kd[rng.integers(0, m), j] = 1.0
    l = rng.uniform(-3.0, 0.0, size=n)
    u = l + rng.uniform(1.0, 4.0, size=n)
    x_bar = rng.uniform(l, u)
    q = Kd @ x_bar
    q[m_eq:] -= rng.uniform(0.0, 1.0, size=m_ineq)
    c = rng.standard_normal(n)
    rows, cols = np.nonzero(Kd)
    row_ptr, col_idx, val = coo_to_csr(m, n, rows, cols, Kd[rows, cols])
    return LP(m_eq=m_eq, m_ineq=m_ineq, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, c=c,
              q=q, l=l, u=u, name=f"tiny_general_s{seed}")


def make_long_lines(seed: int, m: int = 2400, n: int = 3000, dense_rows: int = 2,
                    dense_cols: int = 2, col_nnz: int = 3) -> LP:
    """Iterate-parity case for the long-row paths: an m x n general-form LP (half equality rows)
    whose first `dense_rows` rows hold every column and whose first `dense_cols` columns appear in
    every row (with the defaults, rows of 3000 and columns of 2400 entries, more than 8 chunks of
    256 each), the other columns holding col_nnz random entries; N(0,1) values, finite boxes on
    most columns, some free; c and q random (feasibility is not needed for iterate parity)."""
    rng = np.random.default_rng(40_000 + seed)
    rows, cols = [], []
    for i in range(dense_rows):
        rows.append(np.full(n, i))
        cols.append(np.arange(n))
    for j in range(dense_cols):
        rows.append(np.arange(dense_rows, m))
        cols.append(np.full(m - dense_rows, j))
    for j in range(dense_cols, n):
        r = rng.choice(np.arange(dense_rows, m), size=col_nnz, replace=False)
        rows.append(r)
        cols.append(np.full(col_nnz, j))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = rng.standard_normal(len(rows))
    row_ptr, col_idx, val = coo_to_csr(m, n, rows, cols, vals)
    l = rng.uniform(-2.0, 0.0, size=n)
    u = l + rng.uniform(0.5, 3.0, size=n)
    free = rng.random(n) < 0.1
    l[free], u[free] = -INF, INF
    m_eq = m // 2
    return LP(m_eq=m_eq, m_ineq=m - m_eq, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val,
              c=rng.standard_normal(n), q=rng.standard_normal(m), l=l, u=u,
              name=f"long_lines_s{seed}")


def make_box_lp(seed: int, n: int = 20) -> LP:
    """LP with no constraint rows (m = 0): min c^T x over a finite box, c_j != 0."""
    rng = np.random.default_rng(30_000 + seed)
    l = rng.uniform(-5.0, 0.0, size=n)
    u = l + rng.uniform(0.5, 5.0, size=n)
    c = rng.uniform(0.5, 2.0, size=n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return LP(m_eq=0, m_ineq=0, n=n, row_ptr=np.zeros(1, np.int64),
              col_idx=np.zeros(0, np.int32), val=np.zeros(0), c=c, q=np.zeros(0), l=l, u=u,
              name=f"box_{n}_s{seed}")


def make_fig1_lp() -> LP:
    """The one-variable LP behind Figure 1: min_{x>=0} max_y (x - 1) y, i.e. c = 0, A = 1,
    b = 1, whose unique primal-dual solution is (x, y) = (1, 0)."""
    return LP(m_eq=1, m_ineq=0, n=1, row_ptr=np.array([0, 1], np.int64),
              col_idx=np.array([0], np.int32), val=np.array([1.0]), c=np.array([0.0]),
              q=np.array([1.0]), l=np.array([0.0]), u=np.array([INF]), name="fig1",
              x_star=np.array([1.0]), y_star=np.array([0.0]))


def make_free_bilinear(seed: int, m: int = 6, n: int = 9) -> LP:
    """Equality-constrained LP with all variables free (l = -inf, u = +inf): the
    unconstrained bilinear saddle problem of Proposition 1 (eq. unconstrined)."""
    rng = np.random.default_rng(40_000 + seed)
    Kd = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.6)
    for j in range(n):
        if not Kd[:, j].any():
            Kd[rng.integers(0, m), j] = 1.0
    rows, cols = np.nonzero(Kd)
    row_ptr, col_idx, val = coo_to_csr(m, n, rows, cols, Kd[rows, cols])
    return LP(m_eq=m, m_ineq=0, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val,
              c=rng.standard_normal(n), q=rng.standard_normal(m), l=np.full(n, -INF),
              u=np.full(n, INF), name=f"free_bilinear_s{seed}")


def make_batch_stream(seed: int = 4, count: int = 2000, m_lo: int = 100, m_hi: int = 200_000,
                      rate_per_s: float = 50.0):
    """Request stream descriptor: per request (arrival time s, m, n = 2.5 m, tolerance, seed).
    Arrivals form a Poisson process (exponential gaps); m is log-uniform in [m_lo, m_hi];
    each request's tolerance is 1e-4 or 1e-6 with probability 1/2; its LP is
    ``make_standard_planted(seed=1000 + i, m, n, col_nnz=5)``."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)
    ms = np.floor(np.exp(rng.uniform(math.log(m_lo), math.log(m_hi), size=count))).astype(int)
    tol = np.where(rng.random(count) < 0.5, 1e-4, 1e-6)
    return [dict(arrival_s=float(t[i]), m=int(ms[i]), n=int(round(2.5 * ms[i])),
                 tol=float(tol[i]), seed=1000 + i) for i in range(count)]
