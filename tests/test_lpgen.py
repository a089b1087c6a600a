"""The seeded generators: planted optima satisfy the KKT conditions exactly, planted
certificates satisfy Farkas' lemma, and the structure matches the stated recipe.
These checks use their own dense/sparse algebra, not the oracle's."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2407_16144_gb300 import lpgen


def _K(lp):
    return sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))


def _check_planted(lp, tol=1e-11):
    K = _K(lp)
    x, y = lp.x_star, lp.y_star
    Kx = K @ x
    scale = 1.0 + np.abs(lp.q).max()
    # primal feasibility
    assert np.abs(Kx[:lp.m_eq] - lp.q[:lp.m_eq]).max(initial=0) <= tol * scale
    assert (Kx[lp.m_eq:] - lp.q[lp.m_eq:]).min(initial=0) >= -tol * scale
    assert (x >= lp.l - 1e-15).all() and (x <= lp.u + 1e-15).all()
    # dual feasibility: y_G >= 0 and reduced costs of the right sign
    assert (y[lp.m_eq:] >= 0).all()
    lam = lp.c - K.T @ y
    at_l = np.isfinite(lp.l) & (x == lp.l)
    at_u = np.isfinite(lp.u) & (x == lp.u)
    interior = ~(at_l | at_u)
    cs = 1.0 + np.abs(lp.c).max()
    assert np.abs(lam[interior]).max(initial=0) <= tol * cs
    assert lam[at_l].min(initial=0) >= -tol * cs
    assert lam[at_u].max(initial=0) <= tol * cs
    # complementary slackness on rows
    slack = Kx[lp.m_eq:] - lp.q[lp.m_eq:]
    assert np.abs(slack * y[lp.m_eq:]).max(initial=0) <= tol * scale * (1 + np.abs(y).max())
    # zero duality gap
    p = lp.c @ x
    d = lp.q @ y + (lam[at_l] * lp.l[at_l]).sum() + (lam[at_u] * lp.u[at_u]).sum()
    assert abs(p - d) <= 1e-10 * (1 + abs(p))


def _check_csr(lp):
    assert lp.row_ptr[0] == 0 and lp.row_ptr[-1] == len(lp.col_idx) == len(lp.val)
    assert (np.diff(lp.row_ptr) >= 0).all()
    for i in range(min(lp.m, 2000)):
        cols = lp.col_idx[lp.row_ptr[i]:lp.row_ptr[i + 1]]
        assert (np.diff(cols) > 0).all()
    assert lp.col_idx.min(initial=0) >= 0 and lp.col_idx.max(initial=0) < lp.n


def test_c1_structure_and_planted():
    lp = lpgen.make_c1(0)
    assert (lp.m, lp.n) == (200, 500)
    assert 2500 <= lp.nnz <= 2600
    assert (np.bincount(lp.col_idx, minlength=lp.n) >= 5).all()
    assert (np.diff(lp.row_ptr) > 0).all()
    assert abs((lp.x_star == 0).mean() - 0.4) < 1e-9
    _check_csr(lp)
    _check_planted(lp)


def test_c1_deterministic():
    a, b = lpgen.make_c1(0), lpgen.make_c1(0)
    assert np.array_equal(a.val, b.val) and np.array_equal(a.c, b.c)
    c = lpgen.make_c1(1)
    assert not np.array_equal(a.c, c.c)


@pytest.mark.parametrize("scale", [0.004, 0.02])
def test_c2_small_planted(scale):
    lp = lpgen.make_c2(1, scale=scale)
    _check_csr(lp)
    _check_planted(lp)
    assert lp.m_eq > 0 and lp.m_ineq > 0
    assert np.isinf(lp.l).any() and np.isfinite(lp.u).any()


@pytest.mark.slow
def test_c2_full_structure():
    lp = lpgen.make_c2(1)
    assert (lp.m_eq, lp.m_ineq, lp.n) == (70_000, 30_000, 250_000)
    assert abs(lp.nnz - 2_500_000) < 50_000
    deg = np.bincount(lp.col_idx, minlength=lp.n)
    assert deg.max() <= 5000 and deg.max() > 1000       # heavy power-law tail
    rows = np.diff(lp.row_ptr)
    assert abs(rows.mean() - 25) < 1
    _check_planted(lp, tol=1e-10)


def test_primal_infeasible_farkas():
    lp = lpgen.make_primal_infeasible(3, m=300, n=600)
    K = _K(lp)
    y = lp.farkas_y
    assert (K.T @ y).max() <= 1e-12
    assert abs(lp.q @ y - 1.0) < 1e-9


def test_dual_infeasible_ray():
    lp = lpgen.make_dual_infeasible(3, m=300, n=600)
    K = _K(lp)
    d = lp.ray_d
    assert (d >= 0).all() and d.max() > 0
    assert np.abs(K @ d).max() <= 1e-12
    assert abs(lp.c @ d + 1.0) < 1e-9


def test_dual_infeasible_twin():
    """The twin is the transposed matrix of the primal-infeasible instance with its Farkas
    vector as a ray; it is primal feasible at the planted point."""
    p = lpgen.make_primal_infeasible(3, m=300, n=600)
    lp = lpgen.make_dual_infeasible_twin(3, m=300, n=600)
    assert (lp.m_eq, lp.m_ineq, lp.n) == (0, 600, 300)
    G = _K(lp)
    assert np.abs(G.toarray() + _K(p).toarray().T).max() == 0.0
    d = lp.ray_d
    assert (G @ d).min() >= -1e-12 and abs(lp.c @ d + 1.0) < 1e-9
    assert np.isinf(lp.l).all() and np.isinf(lp.u).all()
    rng = np.random.default_rng(3 + 200)
    y_bar = rng.standard_normal(300)
    assert (G @ y_bar - lp.q).min() > 0.0


def test_multicommodity_flow_structure():
    """Node-arc incidence per commodity plus shared capacity rows; the planted flow is feasible
    and every column holds exactly +1 (tail), -1 (head) and -1 (capacity)."""
    nodes, arcs, K = 300, 2000, 4
    lp = lpgen.make_multicommodity_flow(5, nodes, arcs, K)
    assert (lp.m_eq, lp.m_ineq, lp.n, lp.nnz) == (K * nodes, arcs, K * arcs, 3 * K * arcs)
    A = _K(lp).tocsc()
    cnt = np.diff(A.indptr)
    assert (cnt == 3).all()
    assert sorted(A.data.reshape(-1, 3)[:, :].sum(axis=1).tolist()) == [-1.0] * (K * arcs)
    for r in range(lp.m):
        seg = lp.col_idx[lp.row_ptr[r]:lp.row_ptr[r + 1]]
        assert (np.diff(seg) > 0).all()
    r = _K(lp) @ lp.x_star - lp.q
    assert np.abs(r[:lp.m_eq]).max() < 1e-9 and r[lp.m_eq:].min() >= 0.0
    assert (lp.x_star >= 0).all()


def test_tiny_and_box_generators():
    for s in range(5):
        lp = lpgen.make_tiny_standard(s)
        _check_csr(lp)
        assert np.linalg.matrix_rank(lp.dense()) == lp.m
        lpg = lpgen.make_tiny_general(s)
        _check_csr(lpg)
        assert np.isfinite(lpg.l).all() and np.isfinite(lpg.u).all()
    box = lpgen.make_box_lp(0)
    assert box.m == 0 and box.nnz == 0 and (box.c != 0).all()


def test_stream_descriptor():
    reqs = lpgen.make_batch_stream(4, count=2000)
    t = np.array([r["arrival_s"] for r in reqs])
    assert (np.diff(t) > 0).all()
    assert abs(len(t) / t[-1] - 50.0) < 5.0                      # Poisson at 50/s
    ms = np.array([r["m"] for r in reqs])
    assert ms.min() >= 100 and ms.max() <= 200_000
    tol = np.array([r["tol"] for r in reqs])
    assert set(np.unique(tol)) == {1e-4, 1e-6}
