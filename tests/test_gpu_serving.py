"""Serving loop (continuous batching under a device-memory budget): requests of different sizes
are admitted as memory and slots free up, small ones into the batched solver and large ones onto
their own single-LP handles, and each result is the same alone and in the mix."""
import time

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


def wait_all(srv, tickets, timeout=120.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, srv.stats()
        time.sleep(0.002)
    return out


def stream_lps(seed=0, k=10):
    rng = np.random.default_rng(seed)
    ms = np.floor(np.exp(rng.uniform(np.log(100), np.log(6000), k))).astype(int)
    return [lpgen.make_standard_planted(seed=1000 + seed * 100 + i, m=int(m), n=int(2.5 * m))
            for i, m in enumerate(ms)]


def test_serving_mixed_sizes(rh):
    lps = stream_lps(0)
    small_nnz = 20_000                      # the larger LPs take the single-LP path
    with rh.Server(8 << 30, small_nnz=small_nnz, max_slots=16, iters_per_step=64) as srv:
        ts = []
        for i, lp in enumerate(lps):
            prec = 0 if lp.nnz <= small_nnz else 1
            ts.append(srv.submit(lp, eps_rel_kkt=1e-6, precision=prec))
            time.sleep(0.003)              # arrivals while others run
        res = wait_all(srv, ts)
        st = srv.stats()
    assert st["admitted_batched"] > 0 and st["admitted_single"] > 0
    for lp, t in zip(lps, ts):
        r, lat = res[t]
        assert r.status == rh.STATUS_OPTIMAL, (lp.name, r.status_name)
        k = O.rel_kkt(lp, O.csr_matrix(lp), r.x, r.y)
        assert k["rel_kkt"] <= 1.05e-6
        assert lat >= r.solve_seconds >= 0.0


def test_serving_result_same_alone_and_in_mix(rh):
    small = lpgen.make_standard_planted(seed=5, m=400, n=1000)
    large = lpgen.make_standard_planted(seed=6, m=3000, n=7500)
    small_nnz = 10_000
    with rh.Server(4 << 30, small_nnz=small_nnz, max_slots=8) as srv:
        a = [srv.submit(small, eps_rel_kkt=1e-8), srv.submit(large, eps_rel_kkt=1e-6, precision=1)]
        alone = wait_all(srv, a)
    with rh.Server(4 << 30, small_nnz=small_nnz, max_slots=8) as srv:
        others = stream_lps(1, k=8)
        ts = [srv.submit(lp, eps_rel_kkt=1e-6, precision=0 if lp.nnz <= small_nnz else 1)
              for lp in others[:4]]
        time.sleep(0.02)
        b = [srv.submit(small, eps_rel_kkt=1e-8), srv.submit(large, eps_rel_kkt=1e-6, precision=1)]
        ts += [srv.submit(lp, eps_rel_kkt=1e-6, precision=0 if lp.nnz <= small_nnz else 1)
               for lp in others[4:]]
        mixed = wait_all(srv, ts + b)
    for ta, tb in zip(a, b):
        ra, rb = alone[ta][0], mixed[tb][0]
        assert ra.status == rb.status == rh.STATUS_OPTIMAL
        assert ra.iters == rb.iters
        assert np.array_equal(ra.x, rb.x) and np.array_equal(ra.y, rb.y)


def test_serving_respects_budget(rh):
    lps = [lpgen.make_standard_planted(seed=50 + i, m=2000, n=5000) for i in range(4)]
    # room for the arena plus about one single-LP handle at a time
    budget = (64 << 20) * 2 + (100 << 20)
    with rh.Server(budget, small_nnz=0, max_slots=1) as srv:
        ts = [srv.submit(lp, eps_rel_kkt=1e-6) for lp in lps]
        time.sleep(0.01)
        st0 = srv.stats()
        res = wait_all(srv, ts)
        st = srv.stats()
    assert st0["pending"] >= 1                     # not everything fits at once
    assert st["peak_bytes_in_use"] <= budget
    assert all(r.status == rh.STATUS_OPTIMAL for r, _ in res.values())


def test_serving_cancel(rh):
    big = lpgen.make_c2(3, scale=0.2)                 # takes the single-LP path (small_nnz = 0)
    with rh.Server(4 << 30, small_nnz=0, max_slots=2) as srv:
        t = srv.submit(big, eps_rel_kkt=1e-15, max_iters=10_000_000, precision=1)
        t0 = time.time()
        while srv.stats()["running_single"] < 1:     # wait until it runs on the device
            assert time.time() - t0 < 60
            time.sleep(0.001)
        srv.cancel(t)
        r, _ = wait_all(srv, [t])[t]
        assert r.status == rh.STATUS_CANCELLED
        # a request cancelled before admission
        t2 = srv.submit(big, eps_rel_kkt=1e-15, max_iters=10_000_000)
        srv.cancel(t2)
        r2, _ = wait_all(srv, [t2])[t2]
        assert r2.status == rh.STATUS_CANCELLED
