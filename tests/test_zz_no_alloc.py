"""rhpdhg_kkt_eval_noalloc: the KKT evaluation for callers that may not allocate device memory
(code inside a framework that owns every device allocation, or a latency-critical loop that
must not take cudaMalloc's synchronisation).  It runs on a fixed scratch array inside the
library.  Checked through the C ABI against rhpdhg_kkt_eval, which allocates its scratch, on two
calls in a row (the shared scratch keeps the previous call's contents, so the second call shows
that what must start at zero is cleared).  This file sorts last so a stop-at-first-failure run
has already run every other test."""
import numpy as np
import pytest

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


def _device(lp):
    import torch
    return lpgen.LP(**{f: (torch.as_tensor(getattr(lp, f), device="cuda")
                           if isinstance(getattr(lp, f), np.ndarray) else getattr(lp, f))
                       for f in ("m_eq", "m_ineq", "n", "row_ptr", "col_idx", "val", "c", "q",
                                 "l", "u", "obj_offset")})


def test_noalloc_matches_allocating_entry_point_twice(rh):
    import torch
    lps = [lpgen.make_c2(1, scale=0.02), lpgen.make_c1(0)]    # larger first, then smaller
    rng = np.random.default_rng(11)
    for lp in lps:
        dlp = _device(lp)
        prob = rh.device_problem(dlp)
        x = torch.as_tensor(np.where(np.isfinite(lp.l), lp.l, 0.0) + rng.uniform(0, 1, lp.n),
                            device="cuda")
        y = torch.as_tensor(rng.standard_normal(lp.m), device="cuda")
        rc, ref = rh.rhpdhg_kkt_eval(prob, x.data_ptr(), y.data_ptr())
        assert rc == rh.OK
        for _ in range(2):
            rc, got = rh.rhpdhg_kkt_eval_noalloc(prob, x.data_ptr(), y.data_ptr())
            assert rc == rh.OK, rh.rhpdhg_last_error(None)
            for g, r in zip(got, ref):
                assert abs(g - r) <= 1e-12 * max(1.0, abs(r)), (got, ref)


def test_noalloc_rejects_n_beyond_its_scratch(rh):
    prob = rh.rhpdhg_problem()
    prob.m_eq, prob.m_ineq, prob.n, prob.nnz = 0, 0, (1 << 20) + 1, 0
    prob.memory = rh.MEM_DEVICE
    prob.row_ptr = prob.c = prob.l = prob.u = 16     # never dereferenced: rejected first
    rc, _ = rh.rhpdhg_kkt_eval_noalloc(prob, 16, None)
    assert rc == rh.ERR_INVALID_ARG
    assert "exceeds the fixed scratch" in rh.rhpdhg_last_error(None)
