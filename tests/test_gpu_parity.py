"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.

Tolerances (FP64 mode):
  * scaling vectors D, E: 1e-12 relative (same operations, different rounding order);
  * PDHG points (x~_t, y~_t) for t < 200: 1e-10 relative in the max norm, and the per-iteration
    fixed-point residual ||z - T(z)||_P^2: 1e-10 relative; restart iterations identical (a
    restart test within 1e-9 of its threshold is a tie and ends the comparison);
  * solutions to tolerance: same status; objective within 1e-8 relative of the oracle's and of
    the planted optimum at eps = 1e-8; the returned point's rel-KKT, recomputed on the host by
    the oracle's checker, within the tolerance.
"""
import math

import numpy as np
import pytest

import layout_rule
from oracle import rhpdhg_oracle as O
from paper_2407_16144_gb300 import lpgen

pytestmark = pytest.mark.gpu

TIE = 1e-9


@pytest.fixture(scope="module")
def rh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_16144_gb300 import _build, rhpdhg
    _build.build()
    rhpdhg.load()
    return rhpdhg


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if a.size == 0:
        return 0.0
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


def first_tie(trace, beta=math.exp(-1.0)):
    """Index of the first iteration whose restart test is within TIE of its threshold."""
    fpr0 = None
    for idx, rec in enumerate(trace):
        t, n, k, f = rec[:4]
        if k == 0:
            fpr0 = f
        if n >= 1 and fpr0 and abs(f / fpr0 - beta * beta) < TIE:
            return idx
    return len(trace)


CASES = {
    "c1": lambda: lpgen.make_c1(0),
    "c2_small": lambda: lpgen.make_c2(1, scale=0.01),
    "tiny_general": lambda: lpgen.make_tiny_general(2, 3, 4, 9),
    "c3_small": lambda: lpgen.make_multicommodity_flow(2, 500, 4000, 4),
    # two entries per column: the K^T walk takes four 64-entry tiles per work item, and 4001
    # columns leave a ragged last group (two tiles, the second with one row)
    "short_cols": lambda: lpgen.make_standard_planted(5, m=1000, n=4001, col_nnz=2),
    # rows of 3000 and columns of 2400 entries: long rows of 10-12 chunks on both sides
    "long_lines": lambda: lpgen.make_long_lines(0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_walk_layout(rh, case):
    """The device's tiles per work item on K^ and K^T match the rule restated from the CSR."""
    lp = CASES[case]()
    A = O.csr_matrix(lp)
    with rh.Solver(lp) as s:
        lay = s.layout()
    assert lay["tile_mult_row"] == layout_rule.expected_tile_mult(A.indptr)
    assert lay["tile_mult_col"] == layout_rule.expected_tile_mult(A.T.tocsr().indptr)
    # the device's layout is the host plan the C ABI reports
    for side, rp in (("row", A.indptr), ("col", A.T.tocsr().indptr)):
        rc, pl = rh.rhpdhg_plan_layout(rp)
        assert rc == 0 and pl["tile_mult"] == lay[f"tile_mult_{side}"]
        assert pl["long_rows"] == lay[f"long_rows_{side}"] and pl["chunks"] == lay[f"chunks_{side}"]
        assert pl["seg"] == lay[f"seg_{side}"]
        # warp-wide FP64 row sums where the tile cost model says they pay
        assert lay[f"wide_rows_{side}"] == pl["wide_rows"]
    if case == "short_cols":
        assert lay["tile_mult_col"] == 4
    if case == "c3_small":
        assert lay["tile_mult_col"] == 2
    assert lay["grid_row"] >= 1 and lay["grid_col"] >= 1
    assert lay["walk_row"] == 0 and lay["walk_col"] == 0          # FP64 handle
    with rh.Solver(lp, precision=1) as s:
        mx = s.layout()
    # mixed: grouped walks where tiles are grouped; the row side takes the wide staging round
    # only with long tiles and a grid set by the tile count
    assert (mx["walk_col"] == 2) == (mx["tile_mult_col"] > 1)
    assert (mx["walk_row"] == 2) == (mx["tile_mult_row"] > 1)
    if mx["walk_row"] == 1:
        assert A.nnz > 256 * ((A.shape[0] + 31) // 32)
    if case == "c2_small":
        assert mx["walk_row"] == 1


@pytest.mark.parametrize("case", list(CASES))
def test_scaling_and_step_match_oracle(rh, case):
    lp = CASES[case]()
    with rh.Solver(lp) as s:
        D, E, eta, om0, smax = s.scaling()
    Kh, Do, Eo = O.scale_problem(O.csr_matrix(lp), 10, 1.0)
    assert rel(D, Do) < 1e-12 and rel(E, Eo) < 1e-12
    so = O.power_sigma_max(Kh, 100)
    assert abs(smax - so) <= 1e-10 * so
    assert abs(eta - 0.9 / so) <= 1e-10 * eta
    c, q = Eo * lp.c, Do * lp.q
    assert abs(om0 - np.linalg.norm(c) / np.linalg.norm(q)) <= 1e-12 * om0


SNAP = [0, 1, 2, 3, 5, 10, 31, 62, 63, 64, 65, 100, 127, 128, 150, 199]


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("pw", [0, 1])
@pytest.mark.parametrize("case", list(CASES))
def test_iterates_match_oracle_first_200(rh, case, alg, pw):
    lp = CASES[case]()
    common = dict(algorithm=alg, eps_rel_kkt=1e-14, primal_weight_update=pw, first_epoch_len=20,
                  check_every=16)
    o = O.solve(lp, O.OracleParams(max_iters=200, **common), snapshot_iters=SNAP, trace=True)
    with rh.Solver(lp, max_iters=200, trace=1, trace_capacity=256, **common) as s:
        r = s.run()
        tr = s.trace()
        assert r.status == rh.STATUS_ITERATION_LIMIT and r.iters == 200
        stop = min(first_tie(o.trace), first_tie(tr))
        assert len(tr) == 200
        # ||z - T(z)||_P^2 is a sum of squared iterate differences: its rounding error is absolute
        # (about eps times the iterate scale), so agreement is relative down to 1e-8 of the
        # starting residual and absolute below it
        floor = 1e-8 * o.trace[0][3]
        for (a, b) in zip(tr[:stop], o.trace[:stop]):
            assert a[:3] == b[:3]                                   # t, n, k
            assert a[4] == b[4], f"restart flag differs at t={a[0]}"
            assert abs(a[3] - b[3]) <= 1e-10 * max(abs(b[3]), floor, 1e-300)
            assert abs(a[5] - b[5]) <= 1e-10 * b[5]                  # omega
        # active-set telemetry at the check iterations (on-bound columns, changes)
        tel = {t: (na, nc) for (t, na, nc) in o.telemetry}
        for a in tr[:stop]:
            if a[0] in tel:
                assert (a[6], a[7]) == tel[a[0]], (a[0], a[6:], tel[a[0]])
            else:
                assert (a[6], a[7]) == (-1, -1)
    # PDHG points at the snapshot iterations: rerun with max_iters = t + 1
    for t in SNAP:
        if t >= stop:
            break
        with rh.Solver(lp, max_iters=t + 1, **common) as s:
            r = s.run()
            xt, yt = s.state(1)
        assert r.iters == t + 1
        sn = o.snapshots[t]
        assert rel(xt, sn["xt"]) < 1e-10, (t, rel(xt, sn["xt"]))
        assert rel(yt, sn["yt"]) < 1e-10, (t, rel(yt, sn["yt"]))


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("case", ["c1", "c2_small"])
def test_solve_to_1e8_matches_oracle(rh, case, alg):
    lp = CASES[case]()
    o = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-8, max_iters=200_000))
    with rh.Solver(lp, algorithm=alg, eps_rel_kkt=1e-8) as s:
        r = s.run()
    assert r.status == rh.STATUS_OPTIMAL == o.status
    assert abs(r.primal_obj - o.primal_obj) <= 1e-8 * (1 + abs(o.primal_obj))
    ref = lp.planted_objective()
    assert abs(r.primal_obj - ref) <= 1e-7 * (1 + abs(ref))
    k = O.rel_kkt(lp, O.csr_matrix(lp), r.x, r.y)
    assert k["rel_kkt"] <= 1e-8 * 1.0001
    assert abs(k["rel_p"] - r.rel_p) <= 1e-6 * max(k["rel_p"], 1e-16) + 1e-15
    # error of the GPU solution against the oracle's solution (reported, loose bound)
    print(f"{case} alg={alg}: iters gpu {r.iters} oracle {o.iters}; |x-x_o|/|x_o| = "
          f"{np.linalg.norm(r.x - o.x) / max(1, np.linalg.norm(o.x)):.2e}")


@pytest.mark.parametrize("alg", [0, 1])
def test_full_size_c2_first_iterations(rh, alg):
    """The 100k x 250k (2.5M nnz) workload at full size, in the benchmark's launch
    configuration: PDHG points of the first iterations against the oracle."""
    lp = lpgen.make_c2(1)
    T = 12
    common = dict(algorithm=alg, eps_rel_kkt=1e-14, first_epoch_len=5, check_every=64)
    o = O.solve(lp, O.OracleParams(max_iters=T, **common), snapshot_iters=[T - 1])
    with rh.Solver(lp, max_iters=T, **common) as s:
        r = s.run()
        xt, yt = s.state(1)
    assert r.iters == T
    sn = o.snapshots[T - 1]
    assert rel(xt, sn["xt"]) < 1e-10 and rel(yt, sn["yt"]) < 1e-10


def _check_certificate(rh, lp, r, kind):
    """Host verification at 1e-8 against the unscaled data: a Farkas y (A^T y <= 0 on the
    equality-form instances, b^T y > 0) or a ray d (c^T d < 0, equality rows K d = 0, inequality
    rows K d >= 0, bound signs)."""
    K = O.csr_matrix(lp)
    if kind == "primal":
        assert r.status == rh.STATUS_PRIMAL_INFEASIBLE, r.status_name
        by = lp.q @ r.cert_y
        assert by > 0 and (K.T @ r.cert_y).max() / by <= 1e-8
        return
    assert r.status == rh.STATUS_DUAL_INFEASIBLE, r.status_name
    d = r.cert_x
    cd = lp.c @ d
    Kd = K @ d
    assert cd < 0
    if lp.m_eq:
        assert np.abs(Kd[:lp.m_eq]).max() / -cd <= 1e-8
    if lp.m_ineq:
        assert (-Kd[lp.m_eq:]).max() / -cd <= 1e-8
    lf, uf = np.isfinite(lp.l), np.isfinite(lp.u)
    if lf.any():
        assert (-d[lf]).max() / -cd <= 1e-8
    if uf.any():
        assert d[uf].max() / -cd <= 1e-8


_INFEASIBLE_KINDS = {
    "primal": ("primal", lpgen.make_primal_infeasible),
    "dual": ("dual", lpgen.make_dual_infeasible),
    "twin": ("dual", lpgen.make_dual_infeasible_twin),
}


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("cadence", [(64, 200), (100_000, 200), (100_000, 1000)])
def test_infeasibility_certificates(rh, alg, cadence):
    """Same status, iteration, restart count and certificate source as the oracle: with checks
    every 64 iterations T(z) - z at a check usually certifies first; without checks the restart
    point or the anchor movement does."""
    C, cap = cadence
    for name, (kind, make) in _INFEASIBLE_KINDS.items():
        lp = make(3, 500, 1000)
        o = O.solve(lp, O.OracleParams(algorithm=alg, max_iters=50_000, max_epoch_len=cap,
                                       check_every=C))
        with rh.Solver(lp, algorithm=alg, max_iters=50_000, max_epoch_len=cap,
                       check_every=C) as s:
            r = s.run()
        _check_certificate(rh, lp, r, kind)
        assert (r.status, r.iters, r.restarts, r.cert_source) == \
            (o.status, o.iters, o.restarts, o.cert_source)
        print(f"{name} alg={alg} C={C} cap={cap}: detected at {r.iters} "
              f"(oracle {o.iters}), source {r.cert_source}")


@pytest.mark.parametrize("precision", [0, 1])
def test_infeasibility_full_size(rh, precision):
    """The 50k x 100k (600k nonzeros) primal-infeasible instance and its dual twin (the
    transposed matrix, 100k inequality rows over 50k free variables, with the planted Farkas
    vector as its ray): certificates verified on the host at 1e-8 against the unscaled data."""
    for name in ("primal", "twin"):
        kind, make = _INFEASIBLE_KINDS[name]
        lp = make()
        with rh.Solver(lp, algorithm=1, precision=precision, max_iters=200_000,
                       time_limit_s=120.0) as s:
            r = s.run()
        _check_certificate(rh, lp, r, kind)
        print(f"full-size {name} precision={precision}: detected at {r.iters} iterations, "
              f"{r.restarts} restarts, {r.solve_seconds:.2f} s")


@pytest.mark.parametrize("alg", [0, 1])
def test_box_lp_and_fig1(rh, alg):
    lp = lpgen.make_box_lp(1, n=77)
    with rh.Solver(lp, algorithm=alg, eps_rel_kkt=1e-12, check_every=8) as s:
        r = s.run()
    assert r.status == rh.STATUS_OPTIMAL
    assert np.abs(r.x - np.where(lp.c > 0, lp.l, lp.u)).max() <= 1e-9
    lp = lpgen.make_fig1_lp()
    with rh.Solver(lp, algorithm=alg, eps_rel_kkt=1e-12, check_every=4) as s:
        r = s.run()
    assert r.status == rh.STATUS_OPTIMAL
    assert abs(r.x[0] - 1.0) < 1e-10 and abs(r.y[0]) < 1e-10


def test_empty_row_and_column(rh):
    """A row with no entries and a column that appears in no row (degenerate structure)."""
    base = lpgen.make_tiny_general(4, 2, 2, 6)
    m, n = base.m + 1, base.n + 1
    row_ptr = np.concatenate([base.row_ptr, [base.row_ptr[-1]]])      # empty last (>=) row
    lp = lpgen.LP(m_eq=base.m_eq, m_ineq=base.m_ineq + 1, n=n, row_ptr=row_ptr,
                  col_idx=base.col_idx, val=base.val, c=np.concatenate([base.c, [1.0]]),
                  q=np.concatenate([base.q, [-1.0]]), l=np.concatenate([base.l, [0.0]]),
                  u=np.concatenate([base.u, [2.0]]))
    o = O.solve(lp, O.OracleParams(algorithm=1, eps_rel_kkt=1e-10, max_iters=100_000))
    with rh.Solver(lp, algorithm=1, eps_rel_kkt=1e-10) as s:
        r = s.run()
    assert r.status == o.status == rh.STATUS_OPTIMAL
    assert abs(r.primal_obj - o.primal_obj) <= 1e-8 * (1 + abs(o.primal_obj))
    assert abs(r.x[-1]) < 1e-8                                        # c_j = 1 > 0, l_j = 0


def test_invalid_problems_rejected(rh):
    lp = lpgen.make_c1(0)
    bad = lpgen.make_c1(0)
    bad.col_idx = bad.col_idx.copy()
    s0, s1 = bad.row_ptr[3], bad.row_ptr[4]
    bad.col_idx[s0:s1] = bad.col_idx[s0:s1][::-1]                      # unsorted row
    with pytest.raises(rh.RHPDHGError, match="strictly increasing"):
        rh.Solver(bad)
    bad = lpgen.make_c1(0)
    bad.val = bad.val.copy()
    bad.val[7] = np.nan
    with pytest.raises(rh.RHPDHGError, match="non-finite"):
        rh.Solver(bad)
    bad = lpgen.make_c1(0)
    bad.l = bad.l.copy()
    bad.l[3] = 5.0
    bad.u = bad.u.copy()
    bad.u[3] = 1.0
    with pytest.raises(rh.RHPDHGError, match="l > u"):
        rh.Solver(bad)
    bad = lpgen.make_c1(0)
    bad.col_idx = bad.col_idx.copy()
    bad.col_idx[0] = lp.n + 4
    with pytest.raises(rh.RHPDHGError, match="out of range"):
        rh.Solver(bad)


def test_warm_start_at_planted_optimum(rh):
    lp = lpgen.make_c1(0)
    with rh.Solver(lp, eps_rel_kkt=1e-9, x0=lp.x_star, y0=lp.y_star) as s:
        r = s.run()
    assert r.status == rh.STATUS_OPTIMAL and r.iters == 64


def test_device_input_equals_host_input(rh):
    import torch
    lp = lpgen.make_c2(2, scale=0.01)
    dev = lpgen.LP(**{f: (torch.as_tensor(getattr(lp, f), device="cuda")
                          if isinstance(getattr(lp, f), np.ndarray) else getattr(lp, f))
                      for f in ("m_eq", "m_ineq", "n", "row_ptr", "col_idx", "val", "c", "q",
                                "l", "u")})
    with rh.Solver(lp, eps_rel_kkt=1e-7) as s:
        a = s.run()
    with rh.Solver(dev, device=True, stream=torch.cuda.current_stream().cuda_stream,
                   eps_rel_kkt=1e-7) as s:
        s.solve(1)
        xo = torch.empty(lp.n, dtype=torch.float64, device="cuda")
        yo = torch.empty(lp.m, dtype=torch.float64, device="cuda")
        b = s.poll(x=xo, y=yo, out_memory=rh.MEM_DEVICE)
    assert a.iters == b.iters and a.primal_obj == b.primal_obj
    assert np.array_equal(a.x, xo.cpu().numpy()) and np.array_equal(a.y, yo.cpu().numpy())


def test_deterministic_and_profile_mode_identical(rh):
    lp = lpgen.make_c2(3, scale=0.01)
    outs = []
    for prof in (0, 0, 1):
        with rh.Solver(lp, eps_rel_kkt=1e-7, profile=prof) as s:
            r = s.run()
            kt = s.kernel_times()
        outs.append(r)
        if prof:
            assert kt["launches_row"] == r.iters and kt["ms_row"] > 0 and kt["ms_col"] > 0
    for r in outs[1:]:
        assert r.iters == outs[0].iters and np.array_equal(r.x, outs[0].x)
        assert np.array_equal(r.y, outs[0].y)


def test_nonblocking_poll_cancel_and_limits(rh):
    lp = lpgen.make_c2(1, scale=0.05)
    with rh.Solver(lp, eps_rel_kkt=1e-15, max_iters=10_000_000) as s:
        for _ in range(2):                              # a handle can solve again
            s.solve(0)
            assert s.poll() is None                     # BUSY while running
            s.cancel()
            r = None
            while r is None:
                r = s.poll()
            assert r.status == rh.STATUS_CANCELLED
    with rh.Solver(lp, eps_rel_kkt=1e-15, time_limit_s=0.05) as s:
        r = s.run()
        assert r.status == rh.STATUS_TIME_LIMIT
    with rh.Solver(lp, eps_rel_kkt=1e-15, max_iters=1000) as s:
        r = s.run()
        assert r.status == rh.STATUS_ITERATION_LIMIT and r.iters == 1000


# ---------------------------------------------------------------------------------------------
# mixed precision (FP32 matrix values and iterate offsets, FP64 anchors and checks): no iterate
# parity is claimed; the solution must reach the tolerance as measured by the FP64 checker on the
# host, and its objective must agree with the FP64 oracle's to the accuracy the tolerance allows.

@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("tol", [1e-6, 1e-8])
@pytest.mark.parametrize("case", ["c1", "c2_small"])
def test_mixed_precision_reaches_tolerance(rh, case, tol, alg):
    lp = CASES[case]()
    o = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=tol, max_iters=400_000))
    with rh.Solver(lp, algorithm=alg, precision=1, eps_rel_kkt=tol, max_iters=400_000) as s:
        r = s.run()
    assert r.status == rh.STATUS_OPTIMAL, r.status_name
    k = O.rel_kkt(lp, O.csr_matrix(lp), r.x, r.y)
    assert k["rel_kkt"] <= tol * 1.05, k
    assert abs(r.primal_obj - o.primal_obj) <= 20 * tol * (1 + abs(o.primal_obj))
    print(f"mixed {case} tol={tol} alg={alg}: iters {r.iters} (fp64 oracle {o.iters}); "
          f"host rel-KKT {k['rel_kkt']:.2e}; |obj - obj_oracle|/(1+|obj|) = "
          f"{abs(r.primal_obj - o.primal_obj) / (1 + abs(o.primal_obj)):.2e}")


def test_mixed_precision_full_size_c2(rh):
    lp = lpgen.make_c2(1)
    with rh.Solver(lp, algorithm=1, precision=1, eps_rel_kkt=1e-6) as s:
        r = s.run()
    assert r.status == rh.STATUS_OPTIMAL
    k = O.rel_kkt(lp, O.csr_matrix(lp), r.x, r.y)
    assert k["rel_kkt"] <= 1.05e-6
    ref = lp.planted_objective()
    assert abs(r.primal_obj - ref) <= 1e-5 * (1 + abs(ref))


def test_multicommodity_flow_full_size(rh):
    """20 commodities on 250k nodes / 2M arcs (7M rows, 40M columns, 120M nonzeros) to 1e-4 in
    both precisions; the independent checker confirms rel-KKT on the unscaled data and the two
    objectives agree to the tolerance's duality gap."""
    lp = lpgen.make_multicommodity_flow()
    K = O.csr_matrix(lp)
    res = {}
    for prec in (1, 0):
        with rh.Solver(lp, algorithm=1, precision=prec, eps_rel_kkt=1e-4,
                       time_limit_s=300.0) as s:
            r = s.run()
        assert r.status == rh.STATUS_OPTIMAL, (prec, r.status_name)
        k = O.rel_kkt(lp, K, r.x, r.y)
        assert k["rel_kkt"] <= 1.05e-4, (prec, k)
        assert r.x.min() >= 0.0
        res[prec] = r
        print(f"C3 precision={prec}: {r.iters} iterations, {r.solve_seconds:.2f} s, "
              f"rel-KKT {k['rel_kkt']:.2e}, objective {r.primal_obj:.6e}")
    a, b = res[1].primal_obj, res[0].primal_obj
    assert abs(a - b) <= 4e-4 * (1 + abs(a) + abs(b))


@pytest.mark.parametrize("alg", [0, 1])
def test_mixed_precision_certificates(rh, alg):
    """FP32 offsets limit a certificate to about 1e-5; a near-certificate at a restart point
    moves the solve to FP64 from that point, which then certifies at 1e-8.  A second solve on
    the same handle starts in mixed precision again and repeats the first exactly."""
    for name, (kind, make) in _INFEASIBLE_KINDS.items():
        lp = make(3, 500, 1000)
        with rh.Solver(lp, algorithm=alg, precision=1, max_iters=100_000,
                       max_epoch_len=200) as s:
            r = s.run()
            r2 = s.run()
        assert (r2.status, r2.iters, r2.restarts) == (r.status, r.iters, r.restarts)
        assert np.array_equal(r2.cert_x, r.cert_x) and np.array_equal(r2.cert_y, r.cert_y)
        assert r.escalated == r2.escalated == 1      # the certificate comes from FP64
        _check_certificate(rh, lp, r, kind)
        print(f"mixed {name} alg={alg}: detected at {r.iters} iterations")


@pytest.mark.parametrize("precision", [0, 1])
def test_active_set_identification_on_device(rh, precision):
    """The device telemetry shows finite-time identification on C1 (Section 4, Stage I): the
    on-bound count settles on the planted zeros of x* and stops changing."""
    lp = lpgen.make_c1(0)
    with rh.Solver(lp, algorithm=1, precision=precision, eps_rel_kkt=1e-8, trace=1,
                   trace_capacity=1 << 14) as s:
        r = s.run()
        tr = s.trace(1 << 14)
    assert r.status == rh.STATUS_OPTIMAL
    checks = [(a[6], a[7]) for a in tr if a[6] >= 0]
    planted = int((lp.x_star == 0).sum())
    assert checks[-1] == (planted, 0)
    tol = 0.0 if precision == 0 else 1e-9      # FP32 offsets from an FP64 anchor
    assert np.array_equal(np.abs(r.x) <= tol, lp.x_star == 0.0)


@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("case", ["c1", "c2_small"])
def test_adaptive_step_matches_oracle(rh, case, alg):
    """Adaptive step rule (FP64): the same accepted steps, retries, restarts and FPR as the
    oracle over the first 100 iterations; then both solves reach 1e-8 at the planted optimum.
    Steps above 1/||K|| make the map locally expansive, so the two trajectories separate
    slowly after that and iteration counts to tolerance are compared only loosely."""
    lp = CASES[case]()
    T = 100
    common = dict(algorithm=alg, adaptive_step=1, eps_rel_kkt=1e-14, first_epoch_len=20,
                  check_every=16)
    o = O.solve(lp, O.OracleParams(max_iters=T, **common), trace=True)
    with rh.Solver(lp, max_iters=T, trace=1, trace_capacity=256, **common) as s:
        r = s.run()
        tr = s.trace()
    assert r.iters == T and len(tr) == T
    retries = {}
    for (t, eta, eb, rt) in o.steps:
        retries[t] = rt
    stop = min(first_tie(o.trace), first_tie(tr))
    for (a, b) in zip(tr[:stop], o.trace[:stop]):
        assert a[:3] == b[:3] and a[4] == b[4]
        assert abs(a[3] - b[3]) <= 1e-6 * max(abs(b[3]), 1e-300), (a[0], a[3], b[3])
        assert abs(a[5] - b[5]) <= 1e-9 * b[5]
        assert a[8] == retries[a[0]], (a[0], a[8], retries[a[0]])
    oo = O.solve(lp, O.OracleParams(algorithm=alg, adaptive_step=1, eps_rel_kkt=1e-8,
                                    max_iters=100_000))
    with rh.Solver(lp, algorithm=alg, adaptive_step=1, eps_rel_kkt=1e-8,
                   max_iters=100_000) as s:
        rr = s.run()
    assert rr.status == rh.STATUS_OPTIMAL == oo.status
    k = O.rel_kkt(lp, O.csr_matrix(lp), rr.x, rr.y)
    assert k["rel_kkt"] <= 1.05e-8
    ref = lp.planted_objective()
    assert abs(rr.primal_obj - ref) <= 1e-6 * (1 + abs(ref))
    print(f"adaptive {case} alg={alg}: {rr.iters} iterations (oracle {oo.iters}), "
          f"final eta {rr.eta:.4f}")


def test_adaptive_step_parameter_checks(rh):
    lp = lpgen.make_c1(0)
    with pytest.raises(rh.RHPDHGError, match="precision 0"):
        rh.Solver(lp, adaptive_step=1, precision=1)
    with rh.Batch(2, 64 << 20) as b:
        with pytest.raises(rh.RHPDHGError, match="constant step"):
            b.add(lp, adaptive_step=1)


@pytest.mark.parametrize("case", ["c2_small", "c3_small", "short_cols"])
def test_mixed_first_iterations_close_to_fp64(rh, case):
    """Before any restart the mixed path follows the FP64 trajectory to FP32 accuracy (one and
    several tiles per work item)."""
    lp = CASES[case]()
    T = 40
    common = dict(algorithm=1, eps_rel_kkt=1e-14, first_epoch_len=100, max_iters=T)
    with rh.Solver(lp, **common) as s:
        s.run()
        x64, y64 = s.state(1)
    with rh.Solver(lp, precision=1, **common) as s:
        s.run()
        x32, y32 = s.state(1)
    assert rel(x32, x64) < 1e-5 and rel(y32, y64) < 1e-5


def _device_lp(lp):
    import torch
    return lpgen.LP(**{f: (torch.as_tensor(getattr(lp, f), device="cuda")
                           if isinstance(getattr(lp, f), np.ndarray) else getattr(lp, f))
                       for f in ("m_eq", "m_ineq", "n", "row_ptr", "col_idx", "val", "c", "q",
                                 "l", "u", "obj_offset")})


@pytest.mark.parametrize("case", ["c1", "c2_small", "tiny_general"])
def test_kkt_eval_matches_oracle_checker(rh, case):
    """rhpdhg_kkt_eval (the termination measure for any point) against the oracle's checker."""
    import torch
    lp = CASES[case]()
    dlp = _device_lp(lp)
    prob = rh.device_problem(dlp)
    rng = np.random.default_rng(5)
    points = []
    if lp.x_star is not None:
        points.append((lp.x_star, lp.y_star))
    points.append((rng.uniform(0, 2, lp.n) * np.isfinite(lp.l) + np.where(np.isfinite(lp.l), 0, 0.3),
                   rng.standard_normal(lp.m)))
    with rh.Solver(lp, eps_rel_kkt=1e-6) as s:
        r = s.run()
    points.append((r.x, r.y))
    K = O.csr_matrix(lp)
    for x, y in points:
        xd = torch.as_tensor(np.ascontiguousarray(x), device="cuda")
        yd = torch.as_tensor(np.ascontiguousarray(y), device="cuda")
        rc, out = rh.rhpdhg_kkt_eval(prob, xd.data_ptr(), yd.data_ptr())
        assert rc == rh.OK
        ref = O.rel_kkt(lp, K, x, y)
        for got, key in zip(out, ["rel_p", "rel_d", "rel_gap", "primal_obj", "dual_obj"]):
            assert abs(got - ref[key]) <= 1e-12 * max(1.0, abs(ref[key])), (key, got, ref[key])
    # solver's own report agrees with the independent evaluation of its returned point
    assert abs(out[0] - r.rel_p) <= 1e-9 * max(r.rel_p, 1e-12) + 1e-15


@pytest.mark.parametrize("precision", [0, 1])
def test_repeated_handles_bit_identical(rh, precision):
    """Handles created after others were freed run on reused (dirty) device buffers: every solve
    of the same LP gives bit-identical results, so nothing relies on freshly zeroed memory."""
    lp = CASES["c3_small"]()
    outs = []
    for _ in range(3):
        with rh.Solver(lp, precision=precision, eps_rel_kkt=1e-6, max_iters=3000) as s:
            r = s.run()
        outs.append((r.status, r.iters, r.x.copy(), r.y.copy()))
        # a handle of another size in between, so the cache holds buffers of both
        with rh.Solver(CASES["c1"](), precision=precision, max_iters=50) as s2:
            s2.run()
    for st, it, x, y in outs[1:]:
        assert (st, it) == outs[0][:2]
        assert np.array_equal(x, outs[0][2]) and np.array_equal(y, outs[0][3])
    # the freed handles' buffers are cached; releasing them returns their bytes, then nothing
    assert rh.release_cached_memory() > 0
    assert rh.release_cached_memory() == 0


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("alg", [0, 1])
@pytest.mark.parametrize("case", ["c1", "c2_small", "c3_small"])
def test_restart_schemes_match_oracle(rh, case, alg, scheme, precision):
    """The fixed-frequency schedule (eq. fixed-restart) and the two-phase schedule of the remark
    after Theorem infeas (a first epoch of first_epoch_len, then every max_epoch_len) on the
    device: over 200 iterations the (t, n, k) sequence and the restart iterations equal the
    oracle's in both precisions (these schedules depend on k alone, so no tie can occur); in FP64
    the fixed-point residual and the primal weight also agree to 1e-10, in mixed precision to
    FP32 accuracy."""
    lp = CASES[case]()
    T = 200
    common = dict(algorithm=alg, eps_rel_kkt=1e-14, restart_scheme=scheme, first_epoch_len=45,
                  max_epoch_len=30, check_every=16)
    o = O.solve(lp, O.OracleParams(max_iters=T, **common), trace=True)
    with rh.Solver(lp, precision=precision, max_iters=T, trace=1, trace_capacity=256,
                   **common) as s:
        r = s.run()
        tr = s.trace()
    assert r.iters == T and len(tr) == T
    want = [b[0] for b in o.trace if b[4]]
    got = [a[0] for a in tr if a[4]]
    assert got == want, (got, want)
    first = 45 if scheme == 2 else 30
    assert want[0] == first and all(b - a == 31 for a, b in zip(want, want[1:]))
    tol, floor = (1e-10, 1e-8) if precision == 0 else (1e-3, 1e-6)
    for (a, b) in zip(tr, o.trace):
        assert a[:3] == b[:3]
        assert abs(a[3] - b[3]) <= tol * max(abs(b[3]), floor * o.trace[0][3], 1e-300), \
            (a[0], a[3], b[3])
        assert abs(a[5] - b[5]) <= tol * b[5], (a[0], a[5], b[5])
    assert r.restarts == o.restarts


def test_kkt_eval_reports_out_of_range_columns(rh):
    """The standalone KKT evaluation skips a column index outside [0, n) and a row with offsets
    beyond nnz, and returns RHPDHG_ERR_INVALID_ARG with a message; both entry points."""
    import torch
    lp = CASES["c1"]()
    x = torch.zeros(lp.n, dtype=torch.float64, device="cuda")
    y = torch.zeros(lp.m, dtype=torch.float64, device="cuda")
    for bad in ("column", "row"):
        dlp = _device_lp(lp)
        if bad == "column":
            dlp.col_idx = dlp.col_idx.clone()
            dlp.col_idx[5] = lp.n + 7
        else:
            dlp.row_ptr = dlp.row_ptr.clone()
            dlp.row_ptr[3] = int(lp.row_ptr[-1]) + 100
        prob = rh.device_problem(dlp)
        for fn in (rh.rhpdhg_kkt_eval, rh.rhpdhg_kkt_eval_noalloc):
            rc, _ = fn(prob, x.data_ptr(), y.data_ptr())
            assert rc == rh.ERR_INVALID_ARG, (bad, fn.__name__)
            assert "out of range" in rh.rhpdhg_last_error(None)
    # the library stays usable: a valid evaluation right after succeeds
    rc, out = rh.rhpdhg_kkt_eval(rh.device_problem(_device_lp(lp)), x.data_ptr(), y.data_ptr())
    assert rc == rh.OK


@pytest.mark.parametrize("precision", [0, 1])
def test_caller_allocator_supplies_device_memory(rh, precision):
    """With a caller allocator (here PyTorch's caching allocator through rhpdhg_params.dev_alloc
    / dev_free) every device buffer of the handle comes from it and goes back to it at free, and
    the solve is bit-identical to one on the library's own buffers."""
    import torch
    lp = CASES["c2_small"]()
    with rh.Solver(lp, precision=precision, eps_rel_kkt=1e-7) as s:
        ref = s.run()
    alloc = rh.TorchAllocator()
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    s = rh.Solver(lp, stream=stream, precision=precision, eps_rel_kkt=1e-7, allocator=alloc)
    held, held_bytes = len(alloc.live), sum(alloc.live.values())
    during = torch.cuda.memory_allocated()
    r = s.run()
    s.close()
    torch.cuda.synchronize()
    assert held >= 30, held                       # the handle's vectors, layouts and scratch
    assert during - before >= held_bytes
    assert not alloc.live and torch.cuda.memory_allocated() == before
    assert (r.status, r.iters) == (ref.status, ref.iters)
    assert np.array_equal(r.x, ref.x) and np.array_equal(r.y, ref.y)


@pytest.mark.parametrize("case,alg", [("c2_small", 0), ("c2_small", 1), ("c1", 0), ("c1", 1),
                                      ("c3_small", 1)])
def test_mixed_restart_decisions_fp32_vs_fp64_grade_sums(rh, case, alg):
    """The mixed path sums the restart test's norms in FP32 (df_sums = 0, the default: lane,
    warp, CTA and grid adds in FP32); df_sums = 1 carries double-float (FP64-grade) sums from the
    row up.  Over a full solve to 1e-6 the traced restart iterations, iteration counts and status
    are the same with both, and the traced residuals agree to FP32 summation accuracy.  (On the
    small multicommodity-flow LP plain rHPDHG does not reach 1e-6 within 200k iterations in any
    precision, FP64 included, so that case runs r2HPDHG only.)"""
    lp = CASES[case]()
    runs = {}
    for dfs in (0, 1):
        with rh.Solver(lp, algorithm=alg, precision=1, eps_rel_kkt=1e-6, df_sums=dfs,
                       max_iters=200_000, trace=1, trace_capacity=1 << 17) as s:
            r = s.run()
            tr = s.trace(1 << 17)
        assert r.status == rh.STATUS_OPTIMAL, (dfs, r.status_name)
        runs[dfs] = (r, tr)
    (r0, t0), (r1, t1) = runs[0], runs[1]
    assert r0.iters == r1.iters and r0.restarts == r1.restarts
    assert [a[0] for a in t0 if a[4]] == [a[0] for a in t1 if a[4]]
    # the FP32 sums carry an absolute error of about 1e-7 of the sum of the terms' magnitudes,
    # which the cross term's cancellation makes larger relative to a small residual: the
    # difference is bounded relative to the residual plus 1e-6 of the largest traced residual
    big = max(abs(b[3]) for b in t1)
    worst = max(abs(a[3] - b[3]) / (abs(b[3]) + 1e-6 * big) for a, b in zip(t0, t1))
    print(f"{case} alg={alg}: {r0.iters} iterations, {r0.restarts} restarts with both sums; "
          f"largest difference of the traced residual {worst:.1e} (relative, floored)")
    assert worst < 1e-3


@pytest.mark.parametrize("warps", [8, 16])
@pytest.mark.parametrize("case", ["c2_small", "c3_small", "short_cols", "long_lines"])
def test_cta_width_iterates_match_oracle(rh, case, warps):
    """Every CTA width the autotuner may choose computes the same method: with 8- and 16-warp
    CTAs the FP64 PDHG points after 200 iterations match the oracle's to 1e-10 and the restart
    iterations are the oracle's."""
    lp = CASES[case]()
    T = 200
    common = dict(algorithm=1, eps_rel_kkt=1e-14, first_epoch_len=20, check_every=16)
    o = O.solve(lp, O.OracleParams(max_iters=T, **common), snapshot_iters=[T - 1], trace=True)
    with rh.Solver(lp, max_iters=T, cta_warps=warps, trace=1, trace_capacity=256,
                   **common) as s:
        r = s.run()
        xt, yt = s.state(1)
        tr = s.trace()
        lay = s.layout()
    assert lay["cta_warps_row"] == warps and lay["cta_warps_col"] == warps
    assert r.iters == T
    stop = min(first_tie(o.trace), first_tie(tr))
    assert [a[0] for a in tr[:stop] if a[4]] == [b[0] for b in o.trace[:stop] if b[4]]
    if stop == len(tr):
        sn = o.snapshots[T - 1]
        assert rel(xt, sn["xt"]) < 1e-10 and rel(yt, sn["yt"]) < 1e-10


@pytest.mark.parametrize("case", ["c2_small", "c3_small", "short_cols"])
def test_tile_groups_iterates_match_oracle_and_each_other(rh, case):
    """Every tiles-per-item choice the autotuner may make computes the same method.  A forced
    tile_mult of 1, 2 or 4 is taken on each side whose longest group fits the staging area (the
    rule restated in Python decides which), and otherwise the side keeps the rule.  Before the
    first restart no reduction reaches the iterates, and the FP64 PDHG points of all choices
    are then bit-identical.  After 200 iterations they match the oracle's to 1e-10, with its
    restart iterations."""
    lp = CASES[case]()
    A = O.csr_matrix(lp)
    rps = {"row": A.indptr, "col": A.T.tocsr().indptr}
    common = dict(algorithm=1, eps_rel_kkt=1e-14, first_epoch_len=20, check_every=16)
    T = 200
    o = O.solve(lp, O.OracleParams(max_iters=T, **common), snapshot_iters=[T - 1], trace=True)
    early = None
    for m in (1, 2, 4):
        with rh.Solver(lp, max_iters=15, tile_mult=m, **common) as s:
            s.run()
            pts = s.state(1)
            lay = s.layout()
        for side, rp in rps.items():
            want = m if layout_rule.group_fits(rp, m) else layout_rule.expected_tile_mult(rp)
            assert lay[f"tile_mult_{side}"] == want, (side, m)
        if early is None:
            early = pts
        else:
            assert np.array_equal(pts[0], early[0]) and np.array_equal(pts[1], early[1]), m
        with rh.Solver(lp, max_iters=T, tile_mult=m, trace=1, trace_capacity=256,
                       **common) as s:
            r = s.run()
            xt, yt = s.state(1)
            tr = s.trace()
        assert r.iters == T
        stop = min(first_tie(o.trace), first_tie(tr))
        assert [a[0] for a in tr[:stop] if a[4]] == [b[0] for b in o.trace[:stop] if b[4]]
        if stop == len(tr):
            sn = o.snapshots[T - 1]
            assert rel(xt, sn["xt"]) < 1e-10 and rel(yt, sn["yt"]) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuner_choice_report_and_cache(rh, precision):
    """The autotuner times the candidate geometries at create, reports the rule's and the chosen
    candidate's iteration times (the choice is never slower than the rule, which is one of the
    candidates), caches the choice by the LP's structure for the next handle of the same shape,
    and the tuned handle solves to the same objective as the fixed rule."""
    lp = lpgen.make_c2(1, scale=0.05)
    with rh.Solver(lp, precision=precision, eps_rel_kkt=1e-7) as s:
        ref = s.run()
        rule = s.layout()
    assert rule["tuned"] == 0
    with rh.Solver(lp, precision=precision, eps_rel_kkt=1e-7, autotune=1) as s:
        a = s.layout()
        r = s.run()
    assert a["tuned"] in (1, 2)
    assert 0 < a["tune_ns_best"] <= a["tune_ns_rule"]
    assert a["cta_warps_row"] in (4, 8) and a["cta_warps_col"] in (4, 8)
    with rh.Solver(lp, precision=precision, eps_rel_kkt=1e-7, autotune=1) as s:
        b = s.layout()
    assert b["tuned"] == 2
    for k in ("cta_warps_row", "cta_warps_col", "walk_row", "grid_row", "grid_col"):
        assert a[k] == b[k], k
    assert r.status == ref.status == rh.STATUS_OPTIMAL
    assert abs(r.primal_obj - ref.primal_obj) <= 1e-6 * (1 + abs(ref.primal_obj))
    print(f"precision={precision}: rule {a['tune_ns_rule'] / 1e3:.1f} us, chosen "
          f"{a['tune_ns_best'] / 1e3:.1f} us per iteration (warps {a['cta_warps_row']}/"
          f"{a['cta_warps_col']}, row walk {a['walk_row']})")


# ---------------------------------------------------------------------------------------------
# BF16 matrix values (precision 2): power-of-two scaling keeps K^ exact in BF16 when K has at
# most 8 significant bits per value

def test_pow2_scaling_fp64_matches_oracle(rh):
    """The power-of-two scaling option in FP64: the same D and E as the oracle's rounding and
    the same PDHG points over 200 iterations (to 1e-10)."""
    lp = CASES["c3_small"]()
    Kh, Do, Eo = O.scale_problem_pow2(O.csr_matrix(lp), 10, 1.0)
    T = 200
    common = dict(algorithm=1, eps_rel_kkt=1e-14, first_epoch_len=20, check_every=16,
                  pow2_scaling=1)
    o = O.solve(lp, O.OracleParams(max_iters=T, **common), snapshot_iters=[T - 1])
    with rh.Solver(lp, max_iters=T, **common) as s:
        D, E, eta, om0, smax = s.scaling()
        r = s.run()
        xt, yt = s.state(1)
    assert np.array_equal(D, Do) and np.array_equal(E, Eo)
    sn = o.snapshots[T - 1]
    assert r.iters == T and rel(xt, sn["xt"]) < 1e-10 and rel(yt, sn["yt"]) < 1e-10


@pytest.mark.parametrize("alg", [0, 1])
def test_bf16_values_equal_fp32_values_under_pow2_scaling(rh, alg):
    """On an LP of +-1 coefficients the BF16 values of precision 2 are exactly the FP32 values
    of precision 1 with power-of-two scaling, so the two runs are bit-identical: same trace,
    iterations, restarts and point."""
    lp = CASES["c3_small"]()
    common = dict(algorithm=alg, eps_rel_kkt=1e-6, max_iters=30_000, trace=1,
                  trace_capacity=1 << 15)
    with rh.Solver(lp, precision=2, **common) as s:
        a = s.run()
        ta = s.trace(1 << 15)
    with rh.Solver(lp, precision=1, pow2_scaling=1, **common) as s:
        b = s.run()
        tb = s.trace(1 << 15)
    assert (a.status, a.iters, a.restarts) == (b.status, b.iters, b.restarts)
    assert ta == tb
    assert np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y)


def test_bf16_rejects_values_that_are_not_exact(rh):
    lp = CASES["c2_small"]()           # lognormal values: more than 8 significant bits
    with pytest.raises(rh.RHPDHGError, match="BF16"):
        rh.Solver(lp, precision=2)
    with pytest.raises(rh.RHPDHGError, match="parameter"):
        rh.Solver(CASES["c3_small"](), precision=2, df_sums=1)
