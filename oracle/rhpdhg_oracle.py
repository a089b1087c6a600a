"""Plain FP64 CPU oracle for restarted Halpern PDHG (rHPDHG, Algorithm 1) and reflected
restarted Halpern PDHG (r2HPDHG, Algorithm 2) of Lu & Yang, "Restarted Halpern PDHG for Linear
Programming" (arXiv 2407.16144).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the CPU-baseline
leg of the benchmark may import this module.  It shares no code with the CUDA library: it
reads the problem from the seeded generators and does every step itself, in numpy/scipy
float64, one step at a time, in the paper's order and notation.  Library primitives used as
steps: scipy.sparse matrix-vector products, numpy norms.

Problem form.  The paper treats the standard form (Section 2, eq. lp) min c^T x, Ax = b,
x >= 0 with saddle form eq. minmax.  This oracle takes the general form
    min c^T x  s.t.  A x = b,  G x >= h,  l <= x <= u
with K = [A; G], q = [b; h], X = [l, u], Y = R^{m_eq} x R_+^{m_ineq}, which reduces to eq. lp
for m_ineq = 0, l = 0, u = +inf.  The dual variable uses the Lagrangian sign
L(x, y) = c^T x - y^T (K x - q), i.e. the paper's y of eq. pdhg with y -> -y:
    x~ = proj_X(x - tau (c - K^T y))
    y~ = proj_Y(y + sigma (q - K (2 x~ - x)))                                   (eq. pdhg)
With tau = eta/omega and sigma = eta*omega the PDHG norm of Section 1.1 (Notation) becomes
||z||_P^2 = ||x||^2/tau + ||y||^2/sigma + 2 y^T K x.

Readings of silent or ambiguous passages (each listed with its reason in the design notes):
  * preprocessing "as cuPDLP" (Section 7, Algorithmic enhancements): Ruiz equilibration
    (R infinity-norm passes) then Pock-Chambolle scaling with alpha = 1;
  * constant step eta = safety / sigma_max(K^) with sigma_max from a fixed number of power
    iterations (Notation; the theory needs eta < 1/||A||);
  * primal weight omega_0 = ||c^||/||q^|| and, at each restart,
    omega <- exp(0.5 log(dy/dx) + 0.5 log omega) with dx, dy the anchor movements;
  * first-epoch length tau^0 of eq. (adaptive-restart) is a parameter, the n = 0 rule is
    "k > tau^0" as printed;
  * rel-KKT termination (Section 7, Termination criteria) is the l2 relative primal residual,
    dual residual and duality gap at the PDHG point (x~, y~), evaluated every C iterations;
  * two infeasibility candidates, the two limits of Lemma (sublinear-infeas) that Theorem
    (infeas) carries over to restarts: the displacement T(z) - z at each restart point
    z^{n,0} (n >= 1) and at each check iteration, and the anchor movement
    z^{n+1,0} - z^{n,0} at each restart; the first that passes the Farkas test is returned
    with its source (CERT_*).
Parity pinned by tests/test_oracle_pins.py (vertex enumeration, closed-form box LPs, an
independent LP solver's optimum, Proposition 1, Lemma (sublinear-feas), Corollary
(sublinear-feas-reflected), Lemma (iterates-feas)(i), planted optima and planted Farkas
certificates).  Parity unpinned: the primal-weight update (primal_weight_update), which the
paper names without defining it; the tests pin only its orientation and degree (the exact
covariance of the method under c -> alpha c and under (q, l, u) -> beta (q, l, u)), not its
smoothing exponent or which movement it measures.  Also unpinned: iteration counts to a
tolerance (the paper gives rates with unknown constants).
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Callable, Optional

import numpy as np
import scipy.sparse as sp

# status codes (same meaning as the C library's)
RUNNING, OPTIMAL, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE, ITERATION_LIMIT, TIME_LIMIT, \
    NUMERICAL_ERROR, CANCELLED = range(8)
# which candidate certified infeasibility: T(z) - z at a restart point, T(z) - z at a check
# iteration, or the anchor movement z^{n+1,0} - z^{n,0}
CERT_NONE, CERT_RESTART_POINT, CERT_CHECK, CERT_ANCHOR_MOVE = range(4)


@dataclasses.dataclass
class OracleParams:
    algorithm: int = 0            # 0 = rHPDHG (Algorithm 1), 1 = r2HPDHG (Algorithm 2)
    eps_rel_kkt: float = 1e-4
    eps_infeas: float = 1e-8
    max_iters: int = 100_000
    time_limit_s: float = 3600.0
    ruiz_iters: int = 10
    pock_chambolle_alpha: float = 1.0
    step_size: float = 0.0        # 0 = eta from power iteration
    step_safety: float = 0.9
    power_iters: int = 100
    primal_weight: float = 0.0    # 0 = ||c^||/||q^||
    primal_weight_update: int = 1
    first_epoch_len: int = 64     # tau^0 of eq. (adaptive-restart)
    max_epoch_len: int = 1000     # 0 = no cap; restart once k >= max_epoch_len
    restart_scheme: int = 0       # 0 = adaptive (eq. adaptive-restart), 1 = fixed (eq. fixed-restart),
    #                               2 = two-phase: the first epoch restarts at k >= first_epoch_len,
    #                               later ones at k >= max_epoch_len (remark after Theorem infeas)
    restart_beta: float = math.exp(-1.0)
    check_every: int = 64
    adaptive_step: int = 0        # 1 = the adaptive step rule (Section 7, "as cuPDLP")
    pow2_scaling: int = 0         # 1 = every factor of D and E rounded to the nearest power of
    #                               two after Ruiz and Pock-Chambolle (a preconditioner variant)
    x0: Optional[np.ndarray] = None
    y0: Optional[np.ndarray] = None


# ---------------------------------------------------------------------------------------------
# problem set-up
# ---------------------------------------------------------------------------------------------

def csr_matrix(lp) -> sp.csr_matrix:
    return sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))


def scale_problem(K: sp.csr_matrix, ruiz_iters: int, alpha: float):
    """Diagonal preconditioning K^ = D K E.

    Ruiz equilibration: each pass divides row i by sqrt(max_j |K^_ij|) and column j by
    sqrt(max_i |K^_ij|) (both norms taken on the same current matrix).  Then one
    Pock-Chambolle pass with parameter alpha divides row i by sqrt(sum_j |K^_ij|^alpha) and
    column j by sqrt(sum_i |K^_ij|^(2-alpha)).  A zero row or column keeps factor 1.
    Returns (K^, D, E) with D, E the accumulated diagonals.
    """
    m, n = K.shape
    Kh = K.copy().tocsr()
    D = np.ones(m)
    E = np.ones(n)
    for _ in range(ruiz_iters):
        A = abs(Kh)
        rmax = np.asarray(A.max(axis=1).todense()).ravel() if m else np.zeros(0)
        cmax = np.asarray(A.max(axis=0).todense()).ravel() if m else np.zeros(n)
        dr = np.ones(m)
        dc = np.ones(n)
        dr[rmax > 0] = 1.0 / np.sqrt(rmax[rmax > 0])
        dc[cmax > 0] = 1.0 / np.sqrt(cmax[cmax > 0])
        Kh = (sp.diags(dr) @ Kh @ sp.diags(dc)).tocsr()
        D *= dr
        E *= dc
    if alpha is not None and alpha >= 0:
        A = abs(Kh)
        rsum = np.asarray(A.power(alpha).sum(axis=1)).ravel() if m else np.zeros(0)
        csum = np.asarray(A.power(2.0 - alpha).sum(axis=0)).ravel() if m else np.zeros(n)
        dr = np.ones(m)
        dc = np.ones(n)
        dr[rsum > 0] = 1.0 / np.sqrt(rsum[rsum > 0])
        dc[csum > 0] = 1.0 / np.sqrt(csum[csum > 0])
        Kh = (sp.diags(dr) @ Kh @ sp.diags(dc)).tocsr()
        D *= dr
        E *= dc
    return Kh, D, E


def round_pow2(v: np.ndarray) -> np.ndarray:
    """Each positive entry rounded to the power of two nearest to it on a log scale
    (2^floor(log2 v + 1/2)): a scaling factor within a factor sqrt(2) of the original that only
    shifts exponents, so K^ = D K E keeps the significant bits of K."""
    m, e = np.frexp(v)                      # v = m 2^e with m in [0.5, 1)
    return np.ldexp(1.0, np.where(m >= np.sqrt(0.5), e, e - 1))


def scale_problem_pow2(K: sp.csr_matrix, ruiz_iters: int, alpha: float):
    """scale_problem, then D and E rounded to powers of two (round_pow2) and K^ = D K E
    recomputed from K with the rounded factors."""
    _, D, E = scale_problem(K, ruiz_iters, alpha)
    D, E = round_pow2(D), round_pow2(E)
    Kh = (sp.diags(D) @ K @ sp.diags(E)).tocsr()
    return Kh, D, E


def power_sigma_max(Kh: sp.csr_matrix, iters: int) -> float:
    """Largest singular value of K^ by power iteration on K^T K^ from the unit vector
    1/sqrt(n): v <- K^T K^ v / ||K^T K^ v||, ``iters`` times; returns ||K^ v||."""
    m, n = Kh.shape
    if m == 0 or Kh.nnz == 0:
        return 0.0
    v = np.full(n, 1.0 / math.sqrt(n))
    for _ in range(iters):
        w = Kh.T @ (Kh @ v)
        s = np.linalg.norm(w)
        if s == 0.0:
            return 0.0
        v = w / s
    return float(np.linalg.norm(Kh @ v))


# ---------------------------------------------------------------------------------------------
# operator, norms, checks
# ---------------------------------------------------------------------------------------------

def pdhg_T(Kh, KhT, c, q, l, u, m_eq, tau, sigma, x, y):
    """One PDHG step T(z) = (x~, y~) (eq. pdhg, Lagrangian sign), the plain definition:
    both products are formed explicitly."""
    xt = np.clip(x - tau * (c - KhT @ y), l, u)
    yt = y + sigma * (q - Kh @ (2.0 * xt - x))
    yt[m_eq:] = np.maximum(yt[m_eq:], 0.0)
    return xt, yt


def p_norm_sq(Kh, dx, dy, tau, sigma) -> float:
    """||(dx, dy)||_P^2 = ||dx||^2/tau + ||dy||^2/sigma + 2 dy^T K^ dx (the PDHG norm of
    Notation, with the square root the text omits restored by squaring)."""
    return float(dx @ dx / tau + dy @ dy / sigma + 2.0 * (dy @ (Kh @ dx)))


def lambda_projection(g, l, u):
    """Reduced cost lambda = proj_Lambda(g): Lambda_j = {0} (free), [0, inf) (only l finite),
    (-inf, 0] (only u finite), R (both finite)."""
    lf = np.isfinite(l)
    uf = np.isfinite(u)
    lam = np.zeros_like(g)
    both = lf & uf
    lam[both] = g[both]
    lo = lf & ~uf
    lam[lo] = np.maximum(g[lo], 0.0)
    up = uf & ~lf
    lam[up] = np.minimum(g[up], 0.0)
    return lam


def rel_kkt(lp, K, x, y):
    """Relative KKT error of an unscaled point (x, y) (Section 7, Termination criteria, read
    as the l2 form): returns dict(rel_p, rel_d, rel_gap, primal_obj, dual_obj, rel_kkt)."""
    m_eq = lp.m_eq
    q, c, l, u = lp.q, lp.c, lp.l, lp.u
    Kx = K @ x
    r = q - Kx
    r[m_eq:] = np.maximum(r[m_eq:], 0.0)
    rel_p = np.linalg.norm(r) / (1.0 + np.linalg.norm(q))
    g = c - K.T @ y
    lam = lambda_projection(g, l, u)
    rel_d = np.linalg.norm(g - lam) / (1.0 + np.linalg.norm(c))
    p_obj = float(c @ x) + lp.obj_offset
    lam_p = np.maximum(lam, 0.0)
    lam_m = np.maximum(-lam, 0.0)
    bound_terms = np.where(lam_p > 0, np.where(np.isfinite(l), l, 0.0) * lam_p, 0.0) \
        - np.where(lam_m > 0, np.where(np.isfinite(u), u, 0.0) * lam_m, 0.0)
    d_obj = float(q @ y) + float(bound_terms.sum()) + lp.obj_offset
    rel_gap = abs(p_obj - d_obj) / (1.0 + abs(p_obj) + abs(d_obj))
    return dict(rel_p=float(rel_p), rel_d=float(rel_d), rel_gap=float(rel_gap),
                primal_obj=p_obj, dual_obj=d_obj, rel_kkt=float(max(rel_p, rel_d, rel_gap)))


def primal_infeasibility_violation(lp, K, y):
    """Farkas test for primal infeasibility (Proposition full-infeas, dual part of v).
    A vector y (y_G >= 0) certifies Kx >=/= q has no solution in [l, u] when
    q^T y - sum_j [ (K^T y)_j^+ u_j - (K^T y)_j^- l_j ] > 0 with (K^T y)_j <= 0 where
    u_j = inf and (K^T y)_j >= 0 where l_j = -inf.  The candidate is scaled so this ray
    objective equals 1; the return value is the largest remaining violation (inf when the
    objective is not positive)."""
    kty = K.T @ y
    l, u = lp.l, lp.u
    pos = np.maximum(kty, 0.0)
    neg = np.maximum(-kty, 0.0)
    obj = float(lp.q @ y) - float(np.where(np.isfinite(u), pos * np.where(np.isfinite(u), u, 0.0), 0.0).sum()) \
        + float(np.where(np.isfinite(l), neg * np.where(np.isfinite(l), l, 0.0), 0.0).sum())
    if not obj > 0.0:
        return math.inf, obj
    s = 1.0 / obj
    viol = 0.0
    if (~np.isfinite(u)).any():
        viol = max(viol, float((pos[~np.isfinite(u)] * s).max(initial=0.0)))
    if (~np.isfinite(l)).any():
        viol = max(viol, float((neg[~np.isfinite(l)] * s).max(initial=0.0)))
    if lp.m_ineq:
        viol = max(viol, float((np.maximum(-y[lp.m_eq:], 0.0) * s).max(initial=0.0)))
    return viol, obj


def dual_infeasibility_violation(lp, K, d):
    """Test of an unbounded primal ray d (primal part of v): c^T d < 0, A d = 0, G d >= 0,
    d_j >= 0 where l_j is finite and d_j <= 0 where u_j is finite.  The ray is scaled so that
    c^T d = -1; returns the largest remaining violation (inf if c^T d >= 0)."""
    cd = float(lp.c @ d)
    if not cd < 0.0:
        return math.inf, cd
    s = 1.0 / (-cd)
    Kd = K @ d
    viol = 0.0
    if lp.m_eq:
        viol = max(viol, float(np.abs(Kd[:lp.m_eq]).max()) * s)
    if lp.m_ineq:
        viol = max(viol, float(np.maximum(-Kd[lp.m_eq:], 0.0).max()) * s)
    lf = np.isfinite(lp.l)
    uf = np.isfinite(lp.u)
    if lf.any():
        viol = max(viol, float(np.maximum(-d[lf], 0.0).max()) * s)
    if uf.any():
        viol = max(viol, float(np.maximum(d[uf], 0.0).max()) * s)
    return viol, cd


def infeasibility_test(lp, K, cx, cy, eps):
    """Farkas tests of one candidate (cx, cy) (unscaled): the y-part as a primal-infeasibility
    certificate first, then the x-part as an unbounded ray.  Returns (status, cert_x, cert_y)."""
    vy, _ = primal_infeasibility_violation(lp, K, cy)
    if vy <= eps:
        return PRIMAL_INFEASIBLE, None, cy
    vx, _ = dual_infeasibility_violation(lp, K, cx)
    if vx <= eps:
        return DUAL_INFEASIBLE, cx, None
    return RUNNING, None, None


def primal_weight_update(omega, dxa, dya):
    """Primal weight at a restart (Section 7 names the heuristic only; reading: the smoothed
    PDLP rule) from the anchor movements dxa = ||x^{n+1,0} - x^{n,0}||, dya = ||y^{n+1,0} -
    y^{n,0}||: omega <- exp(0.5 log(dya/dxa) + 0.5 log omega), kept when either movement is
    below 1e-10 or the ratio is not finite.  Parity unpinned beyond the covariance the method
    has under scaling of the objective and of the right-hand side (tests pin that)."""
    ratio = dya / dxa if dxa > 1e-10 else 0.0
    if dxa > 1e-10 and dya > 1e-10 and 0.0 < ratio < math.inf:
        return math.exp(0.5 * math.log(ratio) + 0.5 * math.log(omega))
    return omega


# ---------------------------------------------------------------------------------------------
# the solver
# ---------------------------------------------------------------------------------------------

@dataclasses.dataclass
class OracleResult:
    status: int
    iters: int
    restarts: int
    rel_p: float
    rel_d: float
    rel_gap: float
    primal_obj: float
    dual_obj: float
    x: np.ndarray
    y: np.ndarray
    cert_x: Optional[np.ndarray]
    cert_y: Optional[np.ndarray]
    cert_source: int
    eta: float
    omega: float
    sigma_max: float
    D: np.ndarray
    E: np.ndarray
    solve_seconds: float
    trace: list
    snapshots: dict
    telemetry: list = dataclasses.field(default_factory=list)
    steps: list = dataclasses.field(default_factory=list)


def solve(lp, params: OracleParams = OracleParams(), snapshot_iters=(),
          trace: bool = False, time_limit_s: Optional[float] = None) -> OracleResult:
    """Run rHPDHG / r2HPDHG on ``lp`` with ``params``.

    The iteration counter t counts PDHG evaluations T(z); iteration t evaluates T at the
    current iterate z^{n,k}.  ``snapshot_iters`` lists values of t after which the scaled
    iterate z^{n,k}, the PDHG point T(z^{n,k}) and the anchor z^{n,0} are recorded.
    ``trace`` records (t, n, k, ||z - T(z)||_P^2, restart, omega) per iteration.
    """
    t_start = time.perf_counter()
    rho = 2.0 if params.algorithm == 1 else 1.0
    m_eq, m, n = lp.m_eq, lp.m, lp.n
    K = csr_matrix(lp)
    scale = scale_problem_pow2 if params.pow2_scaling else scale_problem
    Kh, D, E = scale(K, params.ruiz_iters, params.pock_chambolle_alpha)
    KhT = Kh.T.tocsr()
    c = E * lp.c
    q = D * lp.q
    l = lp.l / E
    u = lp.u / E

    sigma_max = power_sigma_max(Kh, params.power_iters)
    if params.step_size > 0:
        eta = params.step_size
    elif sigma_max > 1e-12:
        eta = params.step_safety / sigma_max
    else:
        eta = 1.0
    if params.primal_weight > 0:
        omega = params.primal_weight
    else:
        cn, qn = np.linalg.norm(c), np.linalg.norm(q)
        omega = cn / qn if (cn > 1e-10 and qn > 1e-10) else 1.0
    tau, sigma = eta / omega, eta * omega

    # initial point z^{0,0} = (proj_X(0), 0) or the (unscaled) warm start mapped to scaled space
    x = np.clip(np.zeros(n), l, u) if params.x0 is None else np.asarray(params.x0, float) / E
    y = np.zeros(m) if params.y0 is None else np.asarray(params.y0, float) / D
    x0, y0 = x.copy(), y.copy()              # anchor z^{n,0}
    n_ep, k = 0, 0
    fpr0 = None
    tr = []
    snaps = {}
    snapshot_iters = set(snapshot_iters)
    beta2 = params.restart_beta * params.restart_beta
    limit = params.time_limit_s if time_limit_s is None else time_limit_s

    status = RUNNING
    xt = yt = None
    kkt = None
    cert_x = cert_y = None
    cert_source = CERT_NONE
    telemetry = []
    at_prev = np.zeros(n, dtype=bool)
    t = 0
    retries = 0
    eta_next = eta
    steps = []          # adaptive step: (t, eta tried, eta_bar, retries before it) per attempt
    while True:
        xt, yt = pdhg_T(Kh, KhT, c, q, l, u, m_eq, tau, sigma, x, y)
        dx, dy = x - xt, y - yt
        if params.adaptive_step:
            # the step is admissible while eta <= eta_bar = ||dz||_w^2 / (2 |dy^T K^ dx|) with
            # ||dz||_w^2 = omega ||dx||^2 + ||dy||^2 / omega; the next step is
            # min((1 - j^-0.3) eta_bar, (1 + j^-0.6) eta), j = t + 2; an inadmissible step is
            # retried with it (reading R22)
            cross = abs(float(dy @ (Kh @ dx)))
            num = omega * float(dx @ dx) + float(dy @ dy) / omega
            eta_bar = num / (2.0 * cross) if cross > 0.0 else math.inf
            j = t + 2.0
            eta_next = min((1.0 - j ** -0.3) * eta_bar, (1.0 + j ** -0.6) * eta)
            steps.append((t, eta, eta_bar, retries))
            if eta > eta_bar:
                retries += 1
                if retries > 64 or not np.isfinite(eta_next) or eta_next <= 0.0:
                    status = NUMERICAL_ERROR
                    break
                eta = eta_next
                tau, sigma = eta / omega, eta * omega
                continue
            retries = 0
        fpr2 = p_norm_sq(Kh, dx, dy, tau, sigma)
        if not np.isfinite(fpr2):
            status = NUMERICAL_ERROR
        if k == 0:
            fpr0 = fpr2
        if t in snapshot_iters:
            snaps[t] = dict(x=x.copy(), y=y.copy(), xt=xt.copy(), yt=yt.copy(), x0=x0.copy(),
                            y0=y0.copy(), n=n_ep, k=k, omega=omega, fpr2=fpr2)
        last = (t + 1 >= params.max_iters)
        is_check = (t + 1) % params.check_every == 0 or last
        # infeasibility, first candidate: the displacement T(z) - z, which tends to the
        # infimal displacement vector v (Lemma sublinear-infeas; linearly at restart points by
        # Theorem infeas), whose y-part certifies primal and x-part dual infeasibility
        # (Proposition full-infeas); tested at restart points and at check iterations
        if status == RUNNING and ((k == 0 and n_ep >= 1) or is_check):
            st, cx, cy = infeasibility_test(lp, K, E * (xt - x), D * (yt - y),
                                            params.eps_infeas)
            if st != RUNNING:
                status, cert_x, cert_y = st, cx, cy
                cert_source = CERT_RESTART_POINT if (k == 0 and n_ep >= 1) else CERT_CHECK
        if is_check:
            # active-set telemetry: columns whose PDHG point sits on a bound (the active set of
            # the partition of Section 4 as the iterates see it), and how many changed since
            # the previous check
            at = (xt == l) | (xt == u)
            telemetry.append((t, int(at.sum()), int((at != at_prev).sum())))
            at_prev = at
        if status == RUNNING and is_check:
            kkt = rel_kkt(lp, K, E * xt, D * yt)
            if kkt["rel_kkt"] <= params.eps_rel_kkt:
                status = OPTIMAL
            elif last:
                status = ITERATION_LIMIT
            elif time.perf_counter() - t_start > limit:
                status = TIME_LIMIT
        # restart test (eq. adaptive-restart / eq. fixed-restart, plus the epoch cap)
        if params.restart_scheme == 1:
            restart = params.max_epoch_len > 0 and k >= params.max_epoch_len
        elif params.restart_scheme == 2:
            restart = k >= (params.first_epoch_len if n_ep == 0 else params.max_epoch_len)
        else:
            restart = (n_ep == 0 and k > params.first_epoch_len) or \
                      (n_ep >= 1 and fpr2 <= beta2 * fpr0) or \
                      (params.max_epoch_len > 0 and k >= params.max_epoch_len)
        if trace:
            tr.append((t, n_ep, k, fpr2, bool(restart) and status == RUNNING, omega))
        t += 1
        if status != RUNNING:
            break
        if params.adaptive_step:
            eta = eta_next
            tau, sigma = eta / omega, eta * omega
        if restart:
            # z^{n+1,0} <- T(z^{n,k}).  Second candidate: the anchor movement
            # z^{n+1,0} - z^{n,0}, the restarted form of the normalised iterate
            # (2/k)(z^k - z^0) of Lemma sublinear-infeas (the test is scale free)
            st, cx, cy = infeasibility_test(lp, K, E * (xt - x0), D * (yt - y0),
                                            params.eps_infeas)
            if st != RUNNING:
                status, cert_x, cert_y, cert_source = st, cx, cy, CERT_ANCHOR_MOVE
                n_ep += 1          # the restart took place: z^{n+1,0} is the new anchor
                break
            if params.primal_weight_update:
                omega = primal_weight_update(omega, np.linalg.norm(xt - x0),
                                             np.linalg.norm(yt - y0))
                tau, sigma = eta / omega, eta * omega
            x, y = xt.copy(), yt.copy()
            x0, y0 = x.copy(), y.copy()
            n_ep += 1
            k = 0
        else:
            w = (k + 1.0) / (k + 2.0)
            if rho == 1.0:
                # eq. hpdhg: (k+1)/(k+2) T(z) + 1/(k+2) z^0
                x = w * xt + (1.0 - w) * x0
                y = w * yt + (1.0 - w) * y0
            else:
                # eq. hrpdhg: (k+1)/(k+2) (2 T(z) - z) + 1/(k+2) z^0
                x = w * (2.0 * xt - x) + (1.0 - w) * x0
                y = w * (2.0 * yt - y) + (1.0 - w) * y0
            k += 1

    if kkt is None:
        kkt = rel_kkt(lp, K, E * xt, D * yt)
    return OracleResult(status=status, iters=t, restarts=n_ep, rel_p=kkt["rel_p"],
                        rel_d=kkt["rel_d"], rel_gap=kkt["rel_gap"],
                        primal_obj=kkt["primal_obj"], dual_obj=kkt["dual_obj"], x=E * xt,
                        y=D * yt, cert_x=cert_x, cert_y=cert_y, cert_source=cert_source,
                        telemetry=telemetry, steps=steps,
                        eta=eta, omega=omega,
                        sigma_max=sigma_max, D=D, E=E,
                        solve_seconds=time.perf_counter() - t_start, trace=tr,
                        snapshots=snaps)


def vanilla_pdhg(lp, eta, omega, iters, x0=None, y0=None):
    """Plain fixed-point iteration z^{k+1} = T(z^k) on the unscaled problem (no scaling, no
    restart), used for the trajectory identity of Proposition 1."""
    K = csr_matrix(lp)
    KT = K.T.tocsr()
    tau, sigma = eta / omega, eta * omega
    x = np.zeros(lp.n) if x0 is None else x0.copy()
    y = np.zeros(lp.m) if y0 is None else y0.copy()
    out = [(x.copy(), y.copy())]
    for _ in range(iters):
        x, y = pdhg_T(K, KT, lp.c, lp.q, lp.l, lp.u, lp.m_eq, tau, sigma, x, y)
        out.append((x.copy(), y.copy()))
    return out


def halpern_pdhg(lp, eta, omega, iters, rho=1.0, x0=None, y0=None):
    """Halpern PDHG without restarts on the unscaled problem (eq. hpdhg, or eq. hrpdhg for
    rho = 2): returns the iterates z^0..z^iters and the PDHG points T(z^k)."""
    K = csr_matrix(lp)
    KT = K.T.tocsr()
    tau, sigma = eta / omega, eta * omega
    x = np.zeros(lp.n) if x0 is None else x0.copy()
    y = np.zeros(lp.m) if y0 is None else y0.copy()
    xa, ya = x.copy(), y.copy()
    zs, ts = [], []
    for k in range(iters + 1):
        xt, yt = pdhg_T(K, KT, lp.c, lp.q, lp.l, lp.u, lp.m_eq, tau, sigma, x, y)
        zs.append((x.copy(), y.copy()))
        ts.append((xt.copy(), yt.copy()))
        w = (k + 1.0) / (k + 2.0)
        if rho == 1.0:
            x, y = w * xt + (1 - w) * xa, w * yt + (1 - w) * ya
        else:
            x, y = w * (2 * xt - x) + (1 - w) * xa, w * (2 * yt - y) + (1 - w) * ya
    return zs, ts
