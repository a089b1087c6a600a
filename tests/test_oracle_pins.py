"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics, not by the
oracle itself:

* brute-force vertex enumeration of tiny standard-form LPs (eq. lp);
* the closed form of box LPs (x_j at l_j or u_j by the sign of c_j);
* an independent LP solver (scipy's HiGHS) on small general-form LPs;
* Proposition 1: Halpern PDHG equals averaged PDHG on the unconstrained bilinear problem;
* Lemma (sublinear-feas) and Corollary (sublinear-feas-reflected): fixed-point residual
  bounds at every inner iteration, in the PDHG norm;
* Lemma (iterates-feas)(i): PDHG-norm distance to an optimum never exceeds the epoch anchor's,
  and restart points approach it monotonically;
* the Figure 1 LP and its known solution (tests/golden/fig1_lp.txt);
* Pock-Chambolle scaling with alpha = 1 bounds the spectral norm by 1; power iteration agrees
  with an SVD;
* planted optima (zero gap, complementary slackness) and planted Farkas certificates.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

from oracle import rhpdhg_oracle as O
from paper_2407_16144_gb300 import lpgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def vertex_enumeration(lp):
    """min c^T x over {Ax = b, x >= 0} by trying every basis (tiny standard-form LPs)."""
    A = lp.dense()
    m, n = A.shape
    best = math.inf
    for B in itertools.combinations(range(n), m):
        AB = A[:, B]
        if abs(np.linalg.det(AB)) < 1e-12:
            continue
        xB = np.linalg.solve(AB, lp.q)
        if (xB >= -1e-11).all():
            best = min(best, float(lp.c[list(B)] @ xB))
    return best


def independent_linprog(lp):
    A = lp.dense()
    res = linprog(lp.c, A_eq=A[:lp.m_eq] if lp.m_eq else None,
                  b_eq=lp.q[:lp.m_eq] if lp.m_eq else None,
                  A_ub=-A[lp.m_eq:] if lp.m_ineq else None,
                  b_ub=-lp.q[lp.m_eq:] if lp.m_ineq else None,
                  bounds=list(zip([None if not np.isfinite(v) else v for v in lp.l],
                                  [None if not np.isfinite(v) else v for v in lp.u])),
                  method="highs", options=dict(primal_feasibility_tolerance=1e-10,
                                               dual_feasibility_tolerance=1e-10))
    assert res.status == 0
    return res.fun


def _p_norm(K, dx, dy, tau, sigma):
    v = dx @ dx / tau + dy @ dy / sigma + 2.0 * dy @ (K @ dx)
    return math.sqrt(max(v, 0.0))


# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("seed,m,n", [(0, 2, 5), (1, 3, 6), (2, 3, 7), (3, 4, 8), (4, 4, 8),
                                      (5, 2, 6), (6, 3, 8)])
def test_vertex_enumeration(seed, m, n, alg):
    lp = lpgen.make_tiny_standard(seed, m=m, n=n)
    best = vertex_enumeration(lp)
    r = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-11, max_iters=400_000,
                                   check_every=16))
    assert r.status == O.OPTIMAL
    assert abs(r.primal_obj - best) <= 1e-9 * (1 + abs(best))


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_box_lp_closed_form(seed, alg):
    lp = lpgen.make_box_lp(seed)
    r = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-12, max_iters=10_000,
                                   check_every=8))
    assert r.status == O.OPTIMAL
    expect = np.where(lp.c > 0, lp.l, lp.u)
    assert np.abs(r.x - expect).max() <= 1e-9
    assert r.y.shape == (0,)


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("seed", range(6))
def test_general_form_against_highs(seed, alg):
    lp = lpgen.make_tiny_general(seed, m_eq=2, m_ineq=3, n=7)
    ref = independent_linprog(lp)
    r = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-11, max_iters=400_000,
                                   check_every=16))
    assert r.status == O.OPTIMAL
    assert abs(r.primal_obj - ref) <= 1e-8 * (1 + abs(ref))


@pytest.mark.parametrize("alg", [0, 1])
def test_c2_structure_against_highs(alg):
    lp = lpgen.make_c2(1, scale=0.002)      # 140 + 60 rows, 500 columns, power-law columns
    ref = independent_linprog(lp)
    assert abs(ref - lp.planted_objective()) <= 1e-7 * (1 + abs(ref))
    r = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-10, max_iters=400_000))
    assert r.status == O.OPTIMAL
    assert abs(r.primal_obj - ref) <= 1e-8 * (1 + abs(ref))


def test_fig1_golden():
    with open(os.path.join(GOLDEN, "fig1_lp.txt")) as f:
        g = json.loads("".join(l for l in f if not l.startswith("#")))
    lp = lpgen.make_fig1_lp()
    assert lp.c.tolist() == g["c"] and lp.q.tolist() == g["b"] and lp.val.tolist() == g["A"]
    for alg in (0, 1):
        r = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-12, max_iters=100_000,
                                       check_every=4))
        assert r.status == O.OPTIMAL
        assert abs(r.x[0] - g["x_star"][0]) < 1e-10 and abs(r.y[0] - g["y_star"][0]) < 1e-10


def test_sign_convention_matches_paper_eq_pdhg():
    """One step of eq. pdhg as printed (y_p <- y_p + sigma A (2x+ - x) - sigma b) equals the
    oracle's Lagrangian-sign step with y = -y_p (reading A2)."""
    lp = lpgen.make_c1(3)
    K = O.csr_matrix(lp)
    rng = np.random.default_rng(0)
    x = np.abs(rng.standard_normal(lp.n))
    yp = rng.standard_normal(lp.m)
    tau, sigma = 0.3, 0.7
    xp_next = np.maximum(x - tau * (K.T @ yp) - tau * lp.c, 0.0)
    yp_next = yp + sigma * (K @ (2 * xp_next - x)) - sigma * lp.q
    xt, yt = O.pdhg_T(K, K.T.tocsr(), lp.c, lp.q, lp.l, lp.u, lp.m_eq, tau, sigma, x, -yp)
    assert np.allclose(xt, xp_next, rtol=0, atol=1e-13)
    assert np.allclose(yt, -yp_next, rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", range(3))
def test_prop1_halpern_equals_average_on_bilinear(seed):
    """Proposition 1: on the unconstrained bilinear problem, Halpern iterate z^k equals the
    average of the first k+1 vanilla PDHG iterates started at the same point."""
    lp = lpgen.make_free_bilinear(seed)
    smax = np.linalg.svd(lp.dense(), compute_uv=False)[0]
    eta = 0.5 / smax
    rng = np.random.default_rng(seed)
    x0, y0 = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
    van = O.vanilla_pdhg(lp, eta, 1.0, 60, x0, y0)
    hal, _ = O.halpern_pdhg(lp, eta, 1.0, 60, rho=1.0, x0=x0, y0=y0)
    for k in range(61):
        xa = np.mean([v[0] for v in van[:k + 1]], axis=0)
        ya = np.mean([v[1] for v in van[:k + 1]], axis=0)
        assert np.abs(hal[k][0] - xa).max() <= 1e-12 * (1 + np.abs(xa).max())
        assert np.abs(hal[k][1] - ya).max() <= 1e-12 * (1 + np.abs(ya).max())


def test_prop1_fails_with_projection():
    """The identity of Proposition 1 is specific to the unconstrained problem: with x >= 0
    (the Figure 1 LP) the two trajectories separate, as Section 2 states."""
    lp = lpgen.make_fig1_lp()
    start = dict(x0=np.array([0.0]), y0=np.array([-3.0]))    # the projection is active
    van = O.vanilla_pdhg(lp, 0.5, 1.0, 30, **start)
    hal, _ = O.halpern_pdhg(lp, 0.5, 1.0, 30, rho=1.0, **start)
    diffs = [abs(hal[k][0][0] - np.mean([v[0][0] for v in van[:k + 1]])) for k in range(31)]
    assert max(diffs) > 1e-3


@pytest.mark.parametrize("rho,const", [(1.0, 2.0), (2.0, 1.0)])
@pytest.mark.parametrize("maker", ["c1", "general", "c2small"])
def test_sublinear_fpr_bound_every_iteration(rho, const, maker):
    """Lemma (sublinear-feas): ||z^k - T(z^k)|| <= (2/k) ||z^k - z^0|| for Halpern PDHG;
    Corollary (sublinear-feas-reflected): <= (1/k) ||z^k - z^0|| for the reflected variant;
    PDHG norm, every k >= 1."""
    lp = {"c1": lambda: lpgen.make_c1(2),
          "general": lambda: lpgen.make_tiny_general(1, 3, 3, 8),
          "c2small": lambda: lpgen.make_c2(5, scale=0.002)}[maker]()
    K = O.csr_matrix(lp)
    smax = np.linalg.svd(lp.dense(), compute_uv=False)[0]
    eta, omega = 0.9 / smax, 1.7
    zs, ts = O.halpern_pdhg(lp, eta, omega, 400, rho=rho)
    tau, sigma = eta / omega, eta * omega
    for k in range(1, len(zs)):
        (x, y), (xt, yt) = zs[k], ts[k]
        lhs = _p_norm(K, x - xt, y - yt, tau, sigma)
        rhs = const / k * _p_norm(K, x - zs[0][0], y - zs[0][1], tau, sigma)
        assert lhs <= rhs * (1 + 1e-9) + 1e-13


@pytest.mark.parametrize("alg", [0, 1])
def test_sublinear_bound_inside_restarted_solver(alg):
    """The same bound holds inside every epoch of the restarted solver (scaled space)."""
    lp = lpgen.make_c1(1)
    its = range(0, 400)
    r = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-14, max_iters=400,
                                   primal_weight_update=0), snapshot_iters=its, trace=True)
    K = O.scale_problem(O.csr_matrix(lp), 10, 1.0)[0]
    const = 2.0 if alg == 0 else 1.0
    for t in its:
        s = r.snapshots[t]
        if s["k"] == 0:
            continue
        tau, sigma = r.eta / s["omega"], r.eta * s["omega"]
        lhs = _p_norm(K, s["x"] - s["xt"], s["y"] - s["yt"], tau, sigma)
        rhs = const / s["k"] * _p_norm(K, s["x"] - s["x0"], s["y"] - s["y0"], tau, sigma)
        assert lhs <= rhs * (1 + 1e-9) + 1e-13
        assert abs(lhs * lhs - s["fpr2"]) <= 1e-9 * (1 + s["fpr2"])


@pytest.mark.parametrize("alg", [0, 1])
def test_iterates_feas_distance_to_planted_optimum(alg):
    """Lemma (iterates-feas)(i): ||z^{n,k} - z*|| <= ||z^{n,0} - z*|| and
    ||z^{n+1,0} - z*|| <= ||z^{n,0} - z*|| for the planted optimum z* (fixed primal weight)."""
    lp = lpgen.make_c1(0)
    its = range(0, 900)
    r = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-15, max_iters=900,
                                   primal_weight_update=0, first_epoch_len=40),
                snapshot_iters=its, trace=True)
    Kh, D, E = O.scale_problem(O.csr_matrix(lp), 10, 1.0)
    xs, ys = lp.x_star / E, lp.y_star / D
    tau, sigma = r.eta / r.omega, r.eta * r.omega
    anchors = []
    for t in its:
        s = r.snapshots[t]
        dz = _p_norm(Kh, s["x"] - xs, s["y"] - ys, tau, sigma)
        da = _p_norm(Kh, s["x0"] - xs, s["y0"] - ys, tau, sigma)
        assert dz <= da * (1 + 1e-10) + 1e-12
        if s["k"] == 0:
            anchors.append(da)
    assert len(anchors) >= 3
    assert all(b <= a * (1 + 1e-10) + 1e-12 for a, b in zip(anchors, anchors[1:]))


def test_restart_rule_trace():
    """Restarts follow eq. (adaptive-restart): the first epoch ends at k = tau^0 + 1, later ones
    at the first k with FPR^2 <= beta^2 FPR0^2."""
    lp = lpgen.make_c1(0)
    p = O.OracleParams(eps_rel_kkt=1e-14, max_iters=2000, first_epoch_len=30, max_epoch_len=0)
    r = O.solve(lp, p, trace=True)
    tr = r.trace
    beta2 = math.exp(-2.0)
    fpr0 = None
    for (t, n, k, f, restart, _) in tr:
        if k == 0:
            fpr0 = f
        if n == 0:
            assert restart == (k > 30)
        else:
            assert restart == (f <= beta2 * fpr0)


def test_fixed_frequency_restart():
    lp = lpgen.make_c1(0)
    r = O.solve(lp, O.OracleParams(eps_rel_kkt=1e-14, max_iters=500, restart_scheme=1,
                                   max_epoch_len=50), trace=True)
    restarts = [t for (t, n, k, f, rs, _) in r.trace if rs]
    assert restarts == list(range(50, 500, 51))[:len(restarts)] and len(restarts) >= 9


def test_two_phase_restart_schedule():
    """The schedule of the remark after Theorem infeas: one long first epoch, then a fixed
    frequency.  With first epoch 80 and period 30 the restarts fall at t = 80, then every 31
    evaluations (the restart point itself opens the next epoch at k = 0)."""
    lp = lpgen.make_c1(0)
    r = O.solve(lp, O.OracleParams(eps_rel_kkt=1e-14, max_iters=400, restart_scheme=2,
                                   first_epoch_len=80, max_epoch_len=30), trace=True)
    restarts = [t for (t, n, k, f, rs, _) in r.trace if rs]
    assert restarts == list(range(80, 400, 31))[:len(restarts)] and len(restarts) >= 10


def test_two_phase_schedule_certifies_infeasibility():
    """The schedule's purpose is infeasibility detection: on a planted primal-infeasible LP it
    ends with a Farkas certificate that holds against the unscaled data."""
    lp = lpgen.make_primal_infeasible(3, m=500, n=1000)
    r = O.solve(lp, O.OracleParams(max_iters=50_000, restart_scheme=2, first_epoch_len=400,
                                   max_epoch_len=200))
    assert r.status == O.PRIMAL_INFEASIBLE
    y = r.cert_y
    K = O.csr_matrix(lp)
    by = lp.q @ y
    assert by > 0
    assert (K.T @ y).max() / by <= 1e-8          # A^T y <= 0, b^T y > 0 (Farkas)


def test_scaling_properties():
    lp = lpgen.make_c2(2, scale=0.002)
    K = O.csr_matrix(lp)
    Kh, D, E = O.scale_problem(K, 10, 1.0)
    Kd = Kh.toarray()
    # K^ = D K E
    assert np.allclose(Kd, (D[:, None] * lp.dense()) * E[None, :], rtol=1e-13, atol=0)
    # Pock-Chambolle (alpha = 1) guarantees ||D K E||_2 <= 1
    assert np.linalg.svd(Kd, compute_uv=False)[0] <= 1.0 + 1e-12
    # Ruiz alone equilibrates infinity norms towards 1
    Kr, _, _ = O.scale_problem(K, 40, -1.0)
    A = np.abs(Kr.toarray())
    assert np.abs(A.max(axis=1) - 1).max() < 1e-3 and np.abs(A.max(axis=0) - 1).max() < 1e-3


def test_scaled_problem_same_optimum():
    lp = lpgen.make_tiny_general(3, 2, 2, 6)
    ref = independent_linprog(lp)
    for ruiz, alpha in [(0, -1.0), (10, 1.0), (3, 0.5)]:
        r = O.solve(lp, O.OracleParams(eps_rel_kkt=1e-11, max_iters=400_000, ruiz_iters=ruiz,
                                       pock_chambolle_alpha=alpha))
        assert r.status == O.OPTIMAL and abs(r.primal_obj - ref) <= 1e-8 * (1 + abs(ref))


def test_power_iteration_matches_svd():
    lp = lpgen.make_c1(4)
    Kh, _, _ = O.scale_problem(O.csr_matrix(lp), 10, 1.0)
    s_true = np.linalg.svd(Kh.toarray(), compute_uv=False)[0]
    s100 = O.power_sigma_max(Kh, 100)
    assert s100 <= s_true * (1 + 1e-12)
    assert abs(O.power_sigma_max(Kh, 3000) - s_true) <= 1e-6 * s_true


def test_planted_point_has_zero_kkt():
    for lp in (lpgen.make_c1(0), lpgen.make_c2(1, scale=0.01)):
        k = O.rel_kkt(lp, O.csr_matrix(lp), lp.x_star, lp.y_star)
        assert k["rel_kkt"] <= 1e-14


def test_rel_kkt_closed_forms():
    """rel_p of a perturbed planted point is |delta| ||K_:j|| / (1 + ||q||); with every
    variable free the dual residual is ||c - K^T y|| / (1 + ||c||)."""
    lp = lpgen.make_c1(0)
    K = O.csr_matrix(lp)
    j = int(np.flatnonzero(lp.x_star > 0)[0])
    x = lp.x_star.copy()
    x[j] += 1e-3
    k = O.rel_kkt(lp, K, x, lp.y_star)
    colnorm = np.linalg.norm(K[:, j].toarray())
    assert abs(k["rel_p"] - 1e-3 * colnorm / (1 + np.linalg.norm(lp.q))) < 1e-15
    fb = lpgen.make_free_bilinear(0)
    Kf = O.csr_matrix(fb)
    y = np.ones(fb.m)
    k = O.rel_kkt(fb, Kf, np.zeros(fb.n), y)
    assert abs(k["rel_d"] - np.linalg.norm(fb.c - Kf.T @ y) / (1 + np.linalg.norm(fb.c))) < 1e-15


@pytest.mark.parametrize("alg", [0, 1])
def test_planted_c2_small_to_1e8(alg):
    lp = lpgen.make_c2(1, scale=0.01)
    r = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-8, max_iters=200_000))
    assert r.status == O.OPTIMAL
    ref = lp.planted_objective()
    assert abs(r.primal_obj - ref) <= 1e-7 * (1 + abs(ref))
    # complementary slackness at the returned point, checked independently
    K = O.csr_matrix(lp)
    slack = K @ r.x - lp.q
    bound = 1e-8 * (1 + np.linalg.norm(lp.q)) * (1 + np.abs(r.y).max())
    assert np.abs(slack[lp.m_eq:] * r.y[lp.m_eq:]).max() <= bound


@pytest.mark.parametrize("alg", [0, 1])
def test_primal_infeasible_certificate(alg):
    lp = lpgen.make_primal_infeasible(3, m=500, n=1000)
    r = O.solve(lp, O.OracleParams(algorithm=alg, max_iters=50_000, max_epoch_len=200))
    assert r.status == O.PRIMAL_INFEASIBLE
    y = r.cert_y
    K = O.csr_matrix(lp)
    by = lp.q @ y
    assert by > 0
    assert (K.T @ y).max() / by <= 1e-8          # A^T y <= 0, b^T y > 0 (Farkas)


@pytest.mark.parametrize("alg", [0, 1])
def test_dual_infeasible_certificate(alg):
    lp = lpgen.make_dual_infeasible(3, m=500, n=1000)
    r = O.solve(lp, O.OracleParams(algorithm=alg, max_iters=50_000, max_epoch_len=200))
    assert r.status == O.DUAL_INFEASIBLE
    d = r.cert_x
    K = O.csr_matrix(lp)
    cd = lp.c @ d
    assert cd < 0
    assert np.abs(K @ d).max() / -cd <= 1e-8 and (-d).max() / -cd <= 1e-8


@pytest.mark.parametrize("alg", [0, 1])
def test_dual_infeasible_twin_certificate(alg):
    """Free variables and inequality rows: the ray d must satisfy G d >= 0 and c^T d < 0."""
    lp = lpgen.make_dual_infeasible_twin(3, m=500, n=1000)
    r = O.solve(lp, O.OracleParams(algorithm=alg, max_iters=50_000))
    assert r.status == O.DUAL_INFEASIBLE
    d = r.cert_x
    cd = lp.c @ d
    assert cd < 0
    assert (-(O.csr_matrix(lp) @ d)).max() / -cd <= 1e-8


@pytest.mark.parametrize("case", [
    # (generator, algorithm, check cadence, epoch cap, expected source)
    ("primal", 0, 64, 200, O.CERT_CHECK),
    ("primal", 0, 100_000, 200, O.CERT_RESTART_POINT),
    ("primal", 1, 100_000, 200, O.CERT_ANCHOR_MOVE),
    ("dual", 1, 100_000, 200, O.CERT_ANCHOR_MOVE),
    ("twin", 0, 100_000, 1000, O.CERT_ANCHOR_MOVE),
])
def test_each_certificate_candidate_certifies(case):
    """Both candidates of Lemma sublinear-infeas (T(z) - z at restart points and checks, and the
    anchor movement z^{n+1,0} - z^{n,0}) end a solve on some instance, and every returned
    certificate passes the Farkas tests on the unscaled data."""
    name, alg, C, cap, src = case
    make = {"primal": lpgen.make_primal_infeasible, "dual": lpgen.make_dual_infeasible,
            "twin": lpgen.make_dual_infeasible_twin}[name]
    lp = make(3, m=500, n=1000)
    r = O.solve(lp, O.OracleParams(algorithm=alg, max_iters=50_000, max_epoch_len=cap,
                                   check_every=C))
    assert r.cert_source == src
    K = O.csr_matrix(lp)
    if name == "primal":
        assert r.status == O.PRIMAL_INFEASIBLE
        by = lp.q @ r.cert_y
        assert by > 0 and (K.T @ r.cert_y).max() / by <= 1e-8
    else:
        assert r.status == O.DUAL_INFEASIBLE
        v, cd = O.dual_infeasibility_violation(lp, K, r.cert_x)
        assert cd < 0 and v <= 1e-8
        # independent restatement of the ray test for this instance's form
        Kd = K @ r.cert_x
        if lp.m_eq:
            assert np.abs(Kd[:lp.m_eq]).max() <= 1e-8 * -cd
        if lp.m_ineq:
            assert (-Kd[lp.m_eq:]).max() <= 1e-8 * -cd


@pytest.mark.parametrize("case", ["c1", "c2_small"])
def test_active_set_identification(case):
    """Stage I of Section 4 (finite-time identification): on these planted LPs with strict
    complementarity, the set of PDHG-point coordinates on a bound settles on the planted active
    set and stops changing.  C1: exactly the planted zeros of x*."""
    lp = lpgen.make_c1(0) if case == "c1" else lpgen.make_c2(1, scale=0.01)
    r = O.solve(lp, O.OracleParams(algorithm=1, eps_rel_kkt=1e-10, max_iters=200_000))
    assert r.status == O.OPTIMAL
    tel = r.telemetry
    assert tel[0][1] == tel[0][2]                      # first check: all on-bound columns new
    planted = int(((lp.x_star == lp.l) | (lp.x_star == lp.u)).sum())
    assert tel[-1][1] == planted
    half = tel[len(tel) // 2:]
    assert all(c == 0 for (_, _, c) in half) and all(a == planted for (_, a, _) in half)
    if case == "c1":
        assert np.array_equal(r.x == 0.0, lp.x_star == 0.0)


@pytest.mark.parametrize("alg", [0, 1])
def test_adaptive_step_bound(alg):
    """Adaptive step rule: |dy^T K dx| <= ||K|| ||dx|| ||dy|| <= ||K|| ||dz||_w^2 / 2, so the
    admissibility bound eta_bar is never below 1 / ||K^|| (SVD); every accepted step satisfies
    eta <= eta_bar; and the solve still reaches the planted optimum."""
    lp = lpgen.make_c2(1, scale=0.01)
    r = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-8, max_iters=100_000,
                                   adaptive_step=1))
    Kh, _, _ = O.scale_problem(O.csr_matrix(lp), 10, 1.0)
    smax = np.linalg.svd(Kh.toarray(), compute_uv=False)[0]
    assert r.status == O.OPTIMAL
    assert r.steps and min(eb for (_, _, eb, _) in r.steps) >= (1.0 - 1e-12) / smax
    accepted = {}
    for (t, eta, eb, _) in r.steps:
        accepted[t] = (eta, eb)                        # the last attempt of t is the accepted one
    assert all(eta <= eb for (eta, eb) in accepted.values())
    ref = lp.planted_objective()
    assert abs(r.primal_obj - ref) <= 1e-6 * (1 + abs(ref))


def test_iteration_limit_status():
    lp = lpgen.make_c1(0)
    r = O.solve(lp, O.OracleParams(eps_rel_kkt=1e-12, max_iters=100))
    assert r.status == O.ITERATION_LIMIT and r.iters == 100


def _scaled_copy(lp, alpha=1.0, beta=1.0):
    """The LP with objective alpha c and right-hand side and bounds beta (q, l, u)."""
    import dataclasses
    return dataclasses.replace(lp, c=alpha * lp.c, q=beta * lp.q, l=beta * lp.l, u=beta * lp.u,
                               x_star=None, y_star=None)


def _covariance_gaps(lp, alpha, beta, T=300):
    """Largest relative deviation from exact covariance over T iterations of the restarted
    method with primal-weight updates: with c -> alpha c and (q, l, u) -> beta (q, l, u) the
    scaled iterates map as x -> beta x, y -> alpha y, the primal weight as omega -> omega
    alpha / beta and the PDHG-norm residual as FPR^2 -> alpha beta FPR^2, and the restart
    decisions are the same (the steps tau = eta / omega and sigma = eta omega absorb the
    scalings in eq. pdhg).  Iterations after the residual has fallen to 1e-12 of its start are
    rounding-dominated and are not compared.  Returns (restart flags equal, max omega gap, max FPR
    gap, max iterate gap at the last compared snapshot, restarts compared)."""
    common = dict(algorithm=1, eps_rel_kkt=1e-300, max_iters=T, first_epoch_len=20,
                  check_every=10 ** 6, primal_weight_update=1)
    snaps = list(range(25, T, 25))
    a = O.solve(lp, O.OracleParams(**common), trace=True, snapshot_iters=snaps)
    b = O.solve(_scaled_copy(lp, alpha, beta), O.OracleParams(**common), trace=True,
                snapshot_iters=snaps)
    f0 = a.trace[0][3]
    stop = next((i for i, r in enumerate(a.trace) if r[3] < 1e-12 * f0), len(a.trace))
    stop = min(stop, len(b.trace))
    ta, tb = a.trace[:stop], b.trace[:stop]
    same = [r[4] for r in ta] == [r[4] for r in tb]
    om = max(abs(rb[5] - ra[5] * alpha / beta) / (ra[5] * alpha / beta)
             for ra, rb in zip(ta, tb))
    fp = max(abs(rb[3] - ra[3] * alpha * beta) / max(ra[3] * alpha * beta, 1e-300)
             for ra, rb in zip(ta, tb))
    last = max((t for t in snaps if t < stop and t in a.snapshots and t in b.snapshots),
               default=None)
    it = np.inf
    if last is not None:
        sa, sb = a.snapshots[last], b.snapshots[last]
        it = max(np.abs(sb["xt"] - beta * sa["xt"]).max() /
                 max(1.0, np.abs(beta * sa["xt"]).max()),
                 np.abs(sb["yt"] - alpha * sa["yt"]).max() /
                 max(1.0, np.abs(alpha * sa["yt"]).max()))
    nrestarts = sum(r[4] for r in ta)
    return same, om, fp, it, nrestarts


@pytest.mark.parametrize("make", [lambda: lpgen.make_c1(0),
                                  lambda: lpgen.make_tiny_general(4, 3, 3, 8)])
def test_primal_weight_update_is_scale_covariant(make):
    """The primal-weight update (Section 7 names it without a definition; the oracle takes the
    smoothed rule omega <- sqrt(omega * dy / dx) over anchor movements) keeps the exact
    covariance of the method under c -> 2 c and under (q, l, u) -> 4 (q, l, u).  Powers of two
    keep every step exact except the update's logarithm and exponential, so the two runs agree
    to rounding.  The run has several restarts, so the update is exercised."""
    lp = make()
    for alpha, beta in ((2.0, 1.0), (1.0, 4.0), (2.0, 4.0)):
        same, om, fp, it, nr = _covariance_gaps(lp, alpha, beta)
        assert nr >= 3
        assert same and om < 1e-9 and fp < 1e-8 and it < 1e-9, (alpha, beta, om, fp, it)


def test_primal_weight_covariance_catches_a_wrong_update(monkeypatch):
    """The covariance pin above fails for plausible mistakes in the update, planted in the
    oracle: the ratio inverted (dx / dy), or the movement ratio taken without the old weight
    (not of degree one)."""
    lp = lpgen.make_c1(0)
    wrong = {
        "inverted": lambda om, dx, dy: math.exp(0.5 * math.log(dx / dy) + 0.5 * math.log(om)),
        "no smoothing of omega, ratio squared": lambda om, dx, dy: (dy / dx) ** 2,
    }
    for name, fn in wrong.items():
        monkeypatch.setattr(O, "primal_weight_update", fn)
        same, om, fp, it, nr = _covariance_gaps(lp, 2.0, 1.0)
        assert not (same and om < 1e-6 and it < 1e-6), name


def test_power_of_two_scaling_keeps_the_significant_bits():
    """round_pow2 gives powers of two within a factor sqrt(2) of the unrounded scaling, and with
    them every entry of K^ = D K E of a matrix of small integers has exactly the significant bits
    of the integer (it is the integer times a power of two), which is what makes such a K^ exact
    in a short floating-point format."""
    lp = lpgen.make_multicommodity_flow(2, 300, 2000, 3)
    K = O.csr_matrix(lp)
    _, D0, E0 = O.scale_problem(K, 10, 1.0)
    Kh, D, E = O.scale_problem_pow2(K, 10, 1.0)
    for v, v0 in ((D, D0), (E, E0)):
        mant, _ = np.frexp(v)
        assert np.all(mant == 0.5)                         # powers of two
        assert np.all(v / v0 <= np.sqrt(2) * (1 + 1e-15)) and np.all(v0 / v <= np.sqrt(2) * (1 + 1e-15))
    assert np.allclose(Kh.toarray(), D[:, None] * K.toarray() * E[None, :], rtol=0, atol=0)
    mant, _ = np.frexp(np.abs(Kh.data))
    assert np.all(mant == 0.5)                             # +-1 entries stay +-2^k
    # the rounded scaling is still a valid preconditioner: the oracle solves with it
    r = O.solve(lp, O.OracleParams(algorithm=1, eps_rel_kkt=1e-6, pow2_scaling=1,
                                   max_iters=200_000))
    assert r.status == O.OPTIMAL
    assert O.rel_kkt(lp, K, r.x, r.y)["rel_kkt"] <= 1e-6 * 1.0001
