"""Batched solver (one CTA per LP, one persistent launch for many LPs) against the FP64 oracle
and against itself in different mixes.

Parity: the batched path runs the same FP64 method as the single-LP path, so its PDHG points
after T iterations match the oracle's to 1e-10 (max-norm relative) and its solutions reach the
same objective to 1e-8; an LP's result is bit-identical alone and in any mix of other LPs,
because nothing in its CTA depends on them."""
import numpy as np
import pytest

from oracle import rhpdhg_oracle as O
from paper_2407_16144_gb300 import lpgen

pytestmark = pytest.mark.gpu


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
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(1.0, np.abs(b).max()))


def mix(seed0=0, k=6):
    lps = [lpgen.make_standard_planted(seed=seed0 + i, m=60 + 37 * i, n=150 + 90 * i)
           for i in range(k)]
    lps.append(lpgen.make_tiny_general(3, 3, 4, 9))
    lps.append(lpgen.make_c2(7, scale=0.004))
    return lps


@pytest.mark.parametrize("alg", [0, 1])
def test_batch_iterates_match_oracle(rh, alg):
    lps = mix()
    T = 150
    with rh.Batch(16, 256 << 20) as b:
        slots = [b.add(lp, algorithm=alg, eps_rel_kkt=1e-14, max_iters=T, check_every=16,
                       first_epoch_len=20) for lp in lps]
        res = b.run_all(slots, iters=40)
    for lp, s in zip(lps, slots):
        r = res[s]
        o = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-14, max_iters=T,
                                       check_every=16, first_epoch_len=20))
        assert r.status == rh.STATUS_ITERATION_LIMIT and r.iters == T
        assert rel(r.x, o.x) < 1e-10 and rel(r.y, o.y) < 1e-10, (lp.name, rel(r.x, o.x))


@pytest.mark.parametrize("alg", [0, 1])
def test_batch_solves_to_1e8(rh, alg):
    lps = mix(seed0=20)
    with rh.Batch(16, 256 << 20) as b:
        slots = [b.add(lp, algorithm=alg, eps_rel_kkt=1e-8) for lp in lps]
        res = b.run_all(slots, iters=64)
    for lp, s in zip(lps, slots):
        r = res[s]
        o = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=1e-8, max_iters=400_000))
        assert r.status == rh.STATUS_OPTIMAL == o.status, lp.name
        assert abs(r.primal_obj - o.primal_obj) <= 1e-8 * (1 + abs(o.primal_obj))
        k = O.rel_kkt(lp, O.csr_matrix(lp), r.x, r.y)
        assert k["rel_kkt"] <= 1e-8 * 1.0001
        # iteration counts to tolerance are not pinned (restart decisions near ties diverge)


def test_batch_alone_equals_in_mix(rh):
    target = lpgen.make_standard_planted(seed=77, m=300, n=750)
    with rh.Batch(4, 64 << 20) as b:
        s = b.add(target, eps_rel_kkt=1e-8)
        alone = b.run_all([s], iters=64)[s]
    others = mix(seed0=40)
    with rh.Batch(32, 512 << 20) as b:
        first = [b.add(lp, eps_rel_kkt=1e-8) for lp in others[:4]]
        b.step(100)                                   # others are mid-solve when it arrives
        s = b.add(target, eps_rel_kkt=1e-8)
        rest = [b.add(lp, eps_rel_kkt=1e-8) for lp in others[4:]]
        res = b.run_all(first + [s] + rest, iters=37)
    inmix = res[s]
    assert alone.status == inmix.status == rh.STATUS_OPTIMAL
    assert alone.iters == inmix.iters
    assert np.array_equal(alone.x, inmix.x) and np.array_equal(alone.y, inmix.y)


@pytest.mark.parametrize("C", [64, 100_000])
def test_batch_certificates(rh, C):
    """Batched slots detect infeasibility at the oracle's iteration with the oracle's
    certificate source (T(z) - z at checks or restart points, or the anchor movement)."""
    lps = [lpgen.make_primal_infeasible(3, 500, 1000), lpgen.make_dual_infeasible(3, 500, 1000),
           lpgen.make_dual_infeasible_twin(3, 500, 1000)]
    with rh.Batch(4, 256 << 20) as b:
        slots = [b.add(lp, max_iters=50_000, max_epoch_len=200, check_every=C) for lp in lps]
        res = b.run_all(slots, iters=256)
    for lp, sl in zip(lps, slots):
        r = res[sl]
        o = O.solve(lp, O.OracleParams(algorithm=1, max_iters=50_000, max_epoch_len=200,
                                       check_every=C))
        assert (r.status, r.iters, r.cert_source) == (o.status, o.iters, o.cert_source)
        K = O.csr_matrix(lp)
        if r.status == rh.STATUS_PRIMAL_INFEASIBLE:
            by = lp.q @ r.cert_y
            assert by > 0 and (K.T @ r.cert_y).max() / by <= 1e-8
        else:
            assert r.status == rh.STATUS_DUAL_INFEASIBLE
            v, cd = O.dual_infeasibility_violation(lp, K, r.cert_x)
            assert cd < 0 and v <= 1e-8


@pytest.mark.parametrize("scheme", [1, 2])
def test_batch_restart_schemes_match_oracle(rh, scheme):
    """Fixed-frequency and two-phase restart schedules in batched slots: after 150 iterations
    the PDHG points match the oracle's to 1e-10 and the restart counts are equal."""
    lps = mix(seed0=60)
    T = 150
    common = dict(algorithm=1, eps_rel_kkt=1e-14, max_iters=T, check_every=16,
                  restart_scheme=scheme, first_epoch_len=45, max_epoch_len=30)
    with rh.Batch(16, 256 << 20) as b:
        slots = [b.add(lp, **common) for lp in lps]
        res = b.run_all(slots, iters=40)
    for lp, s in zip(lps, slots):
        r = res[s]
        o = O.solve(lp, O.OracleParams(**common))
        assert r.status == rh.STATUS_ITERATION_LIMIT and r.iters == T
        assert r.restarts == o.restarts
        assert rel(r.x, o.x) < 1e-10 and rel(r.y, o.y) < 1e-10, (lp.name, rel(r.x, o.x))


def test_batch_capacity_limits(rh):
    lp = lpgen.make_c1(0)
    keep = []
    need = rh.rhpdhg_batch_bytes_needed(rh.host_problem(lp, keep))
    with rh.Batch(2, int(need * 1.5)) as b:
        s0 = b.add(lp)
        assert s0 >= 0
        with pytest.raises(rh.RHPDHGError, match="arena full"):
            b.add(lp)                                  # arena has room for one
    with rh.Batch(1, int(need * 3)) as b:
        assert b.add(lp) >= 0
        assert b.add(lp) == -1                         # no free slot (BUSY)
        b.remove(0)
        assert b.add(lp) == 0 and b.free_bytes() >= 0


# ---------------------------------------------------------------------------------------------
# mixed-precision slots (FP32 values and offsets in ordinary iterations, FP64 restarts, restart
# points and checks): accuracy parity with the FP64 oracle, as for the single-LP mixed path

@pytest.mark.parametrize("alg", [0, 1])
def test_batch_mixed_slots_reach_tolerance(rh, alg):
    lps = mix(seed0=80)
    tol = 1e-6
    with rh.Batch(16, 256 << 20) as b:
        slots = [b.add(lp, algorithm=alg, precision=1, eps_rel_kkt=tol, max_iters=400_000)
                 for lp in lps]
        res = b.run_all(slots, iters=64)
    for lp, s in zip(lps, slots):
        r = res[s]
        o = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=tol, max_iters=400_000))
        assert r.status == rh.STATUS_OPTIMAL, (lp.name, r.status_name)
        k = O.rel_kkt(lp, O.csr_matrix(lp), r.x, r.y)
        assert k["rel_kkt"] <= tol * 1.05, (lp.name, k)
        assert abs(r.primal_obj - o.primal_obj) <= 20 * tol * (1 + abs(o.primal_obj))


def test_batch_mixed_first_iterations_close_to_fp64(rh):
    """Before any restart a mixed slot follows its FP64 twin to FP32 accuracy."""
    lps = mix(seed0=90)
    T = 40
    common = dict(algorithm=1, eps_rel_kkt=1e-14, first_epoch_len=100, max_iters=T)
    with rh.Batch(32, 512 << 20) as b:
        s64 = [b.add(lp, precision=0, **common) for lp in lps]
        s32 = [b.add(lp, precision=1, **common) for lp in lps]
        res = b.run_all(s64 + s32, iters=16)
    for lp, a, c in zip(lps, s64, s32):
        ra, rc = res[a], res[c]
        assert ra.iters == rc.iters == T
        assert rel(rc.x, ra.x) < 1e-5 and rel(rc.y, ra.y) < 1e-5, (lp.name, rel(rc.x, ra.x))


def test_batch_mixed_alone_equals_in_mix(rh):
    target = lpgen.make_standard_planted(seed=78, m=300, n=750)
    with rh.Batch(4, 64 << 20) as b:
        s = b.add(target, precision=1, eps_rel_kkt=1e-7)
        alone = b.run_all([s], iters=64)[s]
    others = mix(seed0=45)
    with rh.Batch(32, 512 << 20) as b:
        first = [b.add(lp, precision=p % 2, eps_rel_kkt=1e-7) for p, lp in enumerate(others[:4])]
        b.step(100)
        s = b.add(target, precision=1, eps_rel_kkt=1e-7)
        rest = [b.add(lp, precision=1, eps_rel_kkt=1e-7) for lp in others[4:]]
        res = b.run_all(first + [s] + rest, iters=37)
    inmix = res[s]
    assert alone.status == inmix.status == rh.STATUS_OPTIMAL
    assert alone.iters == inmix.iters
    assert np.array_equal(alone.x, inmix.x) and np.array_equal(alone.y, inmix.y)


def test_batch_mixed_certificates(rh):
    """A mixed slot's near-certificate at a restart point moves the slot to FP64 inside the
    launch, which then certifies at 1e-8 (verified on the host against the unscaled data)."""
    lps = [lpgen.make_primal_infeasible(3, 500, 1000), lpgen.make_dual_infeasible_twin(3, 500, 1000)]
    with rh.Batch(4, 256 << 20) as b:
        slots = [b.add(lp, precision=1, max_iters=100_000, max_epoch_len=200) for lp in lps]
        res = b.run_all(slots, iters=256)
    K0 = O.csr_matrix(lps[0])
    r = res[slots[0]]
    assert r.status == rh.STATUS_PRIMAL_INFEASIBLE, r.status_name
    by = lps[0].q @ r.cert_y
    assert by > 0 and (K0.T @ r.cert_y).max() / by <= 1e-8
    K1 = O.csr_matrix(lps[1])
    r = res[slots[1]]
    assert r.status == rh.STATUS_DUAL_INFEASIBLE, r.status_name
    v, cd = O.dual_infeasibility_violation(lps[1], K1, r.cert_x)
    assert cd < 0 and v <= 1e-8
