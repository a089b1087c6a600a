"""The workloads at their full sizes and stated tolerances, through the C ABI, checked against
the FP64 oracle and its independent rel-KKT checker (oracle.rel_kkt on the unscaled data).

  * 100k x 250k general-form LP (2.5M nonzeros, power-law columns, planted optimum): to 1e-8 in
    FP64 with the objective within 1e-8 relative of the oracle's own full solve (stored in
    tests/golden/oracle_solves.json by tests/golden/make_oracle_solves.py, which calls only the
    oracle), and in mixed precision with the checker's rel-KKT at 1e-8; to 1e-4 in both.
  * Multicommodity flow (20 commodities, 250k nodes, 2M arcs, 120M nonzeros): to 1e-6 in FP64,
    in mixed precision and with BF16 matrix values, checked by the checker, objectives agreeing
    to the tolerance's duality gap.
  * 50k x 100k primal-infeasible LP: certified at 1e-8 under the two-phase restart schedule of
    the remark after Theorem infeas, with the iteration count reported beside the adaptive rule's.

Each test prints every result's error against the FP64 oracle (or its checker)."""
import json
import os

import numpy as np
import pytest

from oracle import rhpdhg_oracle as O
from paper_2407_16144_gb300 import lpgen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_solves.json")


@pytest.fixture(scope="module")
def rh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_16144_gb300 import _build, rhpdhg
    _build.build()
    rhpdhg.load()
    return rhpdhg


@pytest.fixture(scope="module")
def c2():
    lp = lpgen.make_c2(1)
    return lp, O.csr_matrix(lp)


@pytest.mark.parametrize("precision", [0, 1])
def test_c2_full_size_to_1e8(rh, c2, precision):
    lp, K = c2
    with open(GOLDEN) as f:
        g = json.load(f)["c2_seed1_alg1_1e-8"]
    assert g["status"] == O.OPTIMAL
    with rh.Solver(lp, algorithm=1, precision=precision, eps_rel_kkt=1e-8) as s:
        r = s.run()
    assert r.status == rh.STATUS_OPTIMAL, r.status_name
    k = O.rel_kkt(lp, K, r.x, r.y)
    err = abs(r.primal_obj - g["primal_obj"]) / (1 + abs(g["primal_obj"]))
    print(f"C2 precision={precision} to 1e-8: {r.iters} iterations (oracle {g['iters']}), "
          f"{r.solve_seconds:.2f} s; checker rel-KKT {k['rel_kkt']:.2e}; "
          f"|obj - obj_oracle|/(1+|obj_oracle|) = {err:.2e}")
    if precision == 0:
        assert k["rel_kkt"] <= 1e-8 * 1.0001, k
        assert err <= 1e-8
    else:
        assert k["rel_kkt"] <= 1.05e-8, k
        assert err <= 2e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_c2_full_size_to_1e4(rh, c2, precision):
    lp, K = c2
    with rh.Solver(lp, algorithm=1, precision=precision, eps_rel_kkt=1e-4) as s:
        r = s.run()
    assert r.status == rh.STATUS_OPTIMAL, r.status_name
    k = O.rel_kkt(lp, K, r.x, r.y)
    ref = lp.planted_objective()
    err = abs(r.primal_obj - ref) / (1 + abs(ref))
    print(f"C2 precision={precision} to 1e-4: {r.iters} iterations; checker rel-KKT "
          f"{k['rel_kkt']:.2e}; |obj - planted|/(1+|planted|) = {err:.2e}")
    assert k["rel_kkt"] <= 1.05e-4, k
    assert err <= 1e-3


def test_multicommodity_flow_full_size_to_1e6(rh):
    lp = lpgen.make_multicommodity_flow()
    K = O.csr_matrix(lp)
    res = {}
    for prec in (2, 1, 0):
        with rh.Solver(lp, algorithm=1, precision=prec, eps_rel_kkt=1e-6,
                       time_limit_s=600.0) as s:
            r = s.run()
        assert r.status == rh.STATUS_OPTIMAL, (prec, r.status_name)
        k = O.rel_kkt(lp, K, r.x, r.y)
        print(f"C3 precision={prec} to 1e-6: {r.iters} iterations, {r.solve_seconds:.2f} s, "
              f"checker rel-KKT {k['rel_kkt']:.2e}, objective {r.primal_obj:.10e}")
        assert k["rel_kkt"] <= 1.05e-6, (prec, k)
        assert r.x.min() >= 0.0
        assert r.escalated == 0        # a feasible LP stays in its precision
        res[prec] = r
    a, b = res[1].primal_obj, res[0].primal_obj
    print(f"C3 objectives: |mixed - fp64| / (1 + |mixed| + |fp64|) = "
          f"{abs(a - b) / (1 + abs(a) + abs(b)):.2e}")
    assert abs(a - b) <= 4e-6 * (1 + abs(a) + abs(b))


@pytest.mark.parametrize("precision", [0, 1])
def test_infeasible_full_size_two_phase_restart(rh, precision):
    lp = lpgen.make_primal_infeasible()
    K = O.csr_matrix(lp)
    iters = {}
    for scheme, extra in ((0, {}), (2, dict(first_epoch_len=400, max_epoch_len=200))):
        with rh.Solver(lp, algorithm=1, precision=precision, restart_scheme=scheme,
                       max_iters=200_000, time_limit_s=120.0, **extra) as s:
            r = s.run()
        assert r.status == rh.STATUS_PRIMAL_INFEASIBLE, (scheme, r.status_name)
        y = r.cert_y
        by = lp.q @ y
        assert by > 0 and (K.T @ y).max() / by <= 1e-8
        iters[scheme] = (r.iters, r.restarts, r.cert_source)
    print(f"50k x 100k primal-infeasible, precision={precision}: adaptive restart "
          f"{iters[0][0]} iterations ({iters[0][1]} restarts, source {iters[0][2]}); two-phase "
          f"{iters[2][0]} iterations ({iters[2][1]} restarts, source {iters[2][2]})")
