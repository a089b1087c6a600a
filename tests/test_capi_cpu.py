"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a and exports
every function include/rhpdhg.h declares, the Python structures match the C layout byte for
byte, defaults are as documented, and argument validation rejects bad calls before touching
the device."""
import ctypes as C
import os
import re
import shutil
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rhpdhg.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and
                                not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def rh():
    from paper_2407_16144_gb300 import _build, rhpdhg
    _build.build()
    rhpdhg.load()
    return rhpdhg


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rhpdhg_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(rh):
    names = declared_functions()
    assert len(names) >= 11
    lib = C.CDLL(rh.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", rh.LIB_PATH], capture_output=True,
                         text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n
    assert set(names) == set(rh.EXPORTED)


def test_struct_layout_matches_c(rh, tmp_path):
    """Compile a C program that prints sizeof/offsetof of every ABI struct and compare."""
    structs = {"rhpdhg_problem": rh.rhpdhg_problem, "rhpdhg_params": rh.rhpdhg_params,
               "rhpdhg_result": rh.rhpdhg_result, "rhpdhg_trace_rec": rh.rhpdhg_trace_rec}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rhpdhg.h"',
             'int main(void) {']
    for s, cls in structs.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for s, cls in structs.items():
        assert int(got[s]) == C.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_params_default(rh):
    p = rh.rhpdhg_params()
    assert rh.rhpdhg_params_default(p) == rh.OK
    assert p.algorithm == 1 and p.precision == 0
    assert p.eps_rel_kkt == 1e-4 and p.eps_infeas == 1e-8
    assert p.ruiz_iters == 10 and p.pock_chambolle_alpha == 1.0
    assert p.first_epoch_len == 64 and p.check_every == 64 and p.max_epoch_len == 1000
    assert abs(p.restart_beta - np.exp(-1.0)) < 1e-16
    assert rh.load().rhpdhg_params_default(None) == rh.ERR_INVALID_ARG


def test_create_rejects_bad_arguments_on_host(rh):
    p = rh.rhpdhg_params()
    rh.rhpdhg_params_default(p)
    prob = rh.rhpdhg_problem()
    prob.m_eq, prob.m_ineq, prob.n, prob.nnz = 1, 0, 0, 0        # n < 1
    rc, h = rh.rhpdhg_create(prob, p)
    assert rc == rh.ERR_INVALID_ARG and not h.value
    assert "n < 1" in rh.rhpdhg_last_error(None)
    prob.n = 3
    rc, h = rh.rhpdhg_create(prob, p)                             # missing arrays
    assert rc == rh.ERR_INVALID_ARG and "missing" in rh.rhpdhg_last_error(None)
    p.check_every = 0
    arr = np.zeros(8)
    rp = np.zeros(2, dtype=np.int64)
    prob.row_ptr, prob.c, prob.l, prob.u, prob.rhs = (rp.ctypes.data, arr.ctypes.data,
                                                      arr.ctypes.data, arr.ctypes.data,
                                                      arr.ctypes.data)
    rc, h = rh.rhpdhg_create(prob, p)                             # invalid parameter
    assert rc == rh.ERR_INVALID_ARG and "parameter" in rh.rhpdhg_last_error(None)
    rh.rhpdhg_free(None)                                          # NULL-safe


def test_binding_fails_loudly_without_library(tmp_path):
    code = ("import sys; sys.path.insert(0, %r); from paper_2407_16144_gb300 import rhpdhg; "
            "rhpdhg._lib = None\n"
            "try:\n    rhpdhg.load(%r)\nexcept RuntimeError as e:\n    print('raised', e)\n"
            % (ROOT, str(tmp_path / "missing.so")))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True).stdout
    assert out.startswith("raised")


def test_batch_slot_bytes_cover_the_data(rh):
    """A batched slot's size (host computation, no device) holds at least the LP's two CSR copies
    (int32 indices and FP64 values), both row-pointer arrays and the per-slot FP64 vectors, and
    grows with the LP."""
    from paper_2407_16144_gb300 import lpgen
    prev = 0
    for n in (50, 500, 5000):
        lp = lpgen.make_standard_planted(0, m=n // 2, n=n, col_nnz=3)
        keep = []
        need = rh.rhpdhg_batch_bytes_needed(rh.host_problem(lp, keep))
        m, nnz = lp.m_eq + lp.m_ineq, int(lp.row_ptr[-1])
        raw = 2 * nnz * (4 + 8) + 4 * (m + 1 + n + 1) + 8 * (n + m)
        assert need >= raw
        assert need > prev
        prev = need


def test_release_cached_memory_without_handles(rh):
    """With no handle ever freed the buffer cache is empty: releasing it frees nothing and needs
    no device."""
    assert rh.release_cached_memory() == 0


def test_restart_scheme_checked_on_host(rh):
    """Restart schemes 0, 1 (fixed frequency) and 2 (two-phase) are accepted; any other value,
    and a fixed or two-phase schedule without a positive period, are rejected before the device
    is touched."""
    arr = np.zeros(8)
    rp = np.zeros(2, dtype=np.int64)
    prob = rh.rhpdhg_problem()
    prob.m_eq, prob.m_ineq, prob.n, prob.nnz = 1, 0, 3, 0
    prob.row_ptr, prob.c, prob.l, prob.u, prob.rhs = (rp.ctypes.data, arr.ctypes.data,
                                                      arr.ctypes.data, arr.ctypes.data,
                                                      arr.ctypes.data)
    for scheme, cap in ((3, 100), (-1, 100), (1, 0), (2, 0)):
        p = rh.rhpdhg_params()
        rh.rhpdhg_params_default(p)
        p.restart_scheme, p.max_epoch_len = scheme, cap
        rc, h = rh.rhpdhg_create(prob, p)
        assert rc == rh.ERR_INVALID_ARG and not h.value, (scheme, cap)
        assert "parameter" in rh.rhpdhg_last_error(None)


@pytest.mark.parametrize("entry", ["rhpdhg_kkt_eval", "rhpdhg_kkt_eval_noalloc"])
def test_kkt_eval_rejects_bad_arguments_with_a_message(rh, entry):
    """Both KKT entry points reject host-memory problems, missing arrays and a CSR with entries
    but no column indices on the host, and say why in rhpdhg_last_error(NULL)."""
    fn = getattr(rh, entry)
    arr = np.zeros(8)
    rp = np.array([0, 2], dtype=np.int64)
    prob = rh.rhpdhg_problem()
    prob.m_eq, prob.m_ineq, prob.n, prob.nnz = 1, 0, 3, 2
    prob.memory = rh.MEM_HOST
    prob.row_ptr, prob.c, prob.l, prob.u, prob.rhs = (rp.ctypes.data, arr.ctypes.data,
                                                      arr.ctypes.data, arr.ctypes.data,
                                                      arr.ctypes.data)
    prob.col_idx, prob.val = 16, 16
    rc, _ = fn(prob, arr.ctypes.data, arr.ctypes.data)
    assert rc == rh.ERR_INVALID_ARG and "device memory" in rh.rhpdhg_last_error(None)
    prob.memory = rh.MEM_DEVICE
    prob.col_idx = None
    rc, _ = fn(prob, arr.ctypes.data, arr.ctypes.data)
    assert rc == rh.ERR_INVALID_ARG and "missing" in rh.rhpdhg_last_error(None)
    prob.col_idx = 16
    prob.nnz = -1
    rc, _ = fn(prob, arr.ctypes.data, arr.ctypes.data)
    assert rc == rh.ERR_INVALID_ARG and "negative" in rh.rhpdhg_last_error(None)


def test_allocator_hook_given_whole_or_not_at_all(rh):
    """rhpdhg_params.dev_alloc and dev_free come as a pair: one without the other is rejected on
    the host, before any device work."""
    arr = np.zeros(8)
    rp = np.zeros(2, dtype=np.int64)
    prob = rh.rhpdhg_problem()
    prob.m_eq, prob.m_ineq, prob.n, prob.nnz = 1, 0, 3, 0
    prob.row_ptr, prob.c, prob.l, prob.u, prob.rhs = (rp.ctypes.data, arr.ctypes.data,
                                                      arr.ctypes.data, arr.ctypes.data,
                                                      arr.ctypes.data)
    p = rh.rhpdhg_params()
    rh.rhpdhg_params_default(p)
    assert not p.dev_alloc and not p.dev_free and not p.alloc_ctx      # defaults: no hook
    p.dev_alloc = rh.DEV_ALLOC_FN(lambda n, s, c: None)
    rc, h = rh.rhpdhg_create(prob, p)
    assert rc == rh.ERR_INVALID_ARG and not h.value
    assert "dev_alloc and dev_free" in rh.rhpdhg_last_error(None)
