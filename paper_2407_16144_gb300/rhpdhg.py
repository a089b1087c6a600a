"""Python binding of the rHPDHG C ABI (include/rhpdhg.h): argument marshalling only.

Every function named ``rhpdhg_*`` below calls the C function of the same name in the in-tree
``librhpdhg.so``; all arithmetic of the solver runs in that library's CUDA kernels.  The module
raises ``RuntimeError`` when the library is missing or cannot be loaded: there is no fallback.

``Solver`` is a convenience wrapper that creates a handle from an ``lpgen.LP`` held in host
numpy arrays or in device memory (torch CUDA tensors), runs the solve and reads the result.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librhpdhg.so")

OK, BUSY = 0, 1
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_STATE = -1, -2, -3, -4, -5
(STATUS_RUNNING, STATUS_OPTIMAL, STATUS_PRIMAL_INFEASIBLE, STATUS_DUAL_INFEASIBLE,
 STATUS_ITERATION_LIMIT, STATUS_TIME_LIMIT, STATUS_NUMERICAL_ERROR, STATUS_CANCELLED) = range(8)
MEM_HOST, MEM_DEVICE = 0, 1
STATUS_NAMES = ["RUNNING", "OPTIMAL", "PRIMAL_INFEASIBLE", "DUAL_INFEASIBLE",
                "ITERATION_LIMIT", "TIME_LIMIT", "NUMERICAL_ERROR", "CANCELLED"]
# which candidate certified infeasibility (rhpdhg_result.cert_source)
CERT_NONE, CERT_RESTART_POINT, CERT_CHECK, CERT_ANCHOR_MOVE = range(4)

_dp = C.POINTER(C.c_double)


class rhpdhg_problem(C.Structure):
    _fields_ = [("m_eq", C.c_int32), ("m_ineq", C.c_int32), ("n", C.c_int32),
                ("memory", C.c_int32), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p), ("c", C.c_void_p),
                ("rhs", C.c_void_p), ("l", C.c_void_p), ("u", C.c_void_p),
                ("obj_offset", C.c_double)]


DEV_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
DEV_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class rhpdhg_params(C.Structure):
    _fields_ = [("algorithm", C.c_int32), ("precision", C.c_int32),
                ("eps_rel_kkt", C.c_double), ("eps_infeas", C.c_double),
                ("max_iters", C.c_int64), ("time_limit_s", C.c_double),
                ("ruiz_iters", C.c_int32), ("pock_chambolle_alpha", C.c_double),
                ("step_size", C.c_double), ("step_safety", C.c_double),
                ("power_iters", C.c_int32), ("primal_weight", C.c_double),
                ("primal_weight_update", C.c_int32), ("first_epoch_len", C.c_int32),
                ("max_epoch_len", C.c_int64), ("restart_scheme", C.c_int32),
                ("restart_beta", C.c_double), ("check_every", C.c_int32),
                ("use_graphs", C.c_int32), ("trace", C.c_int32), ("profile", C.c_int32),
                ("trace_capacity", C.c_int64), ("x0", C.c_void_p), ("y0", C.c_void_p),
                ("adaptive_step", C.c_int32), ("cta_warps", C.c_int32),
                ("df_sums", C.c_int32), ("dev_alloc", DEV_ALLOC_FN), ("dev_free", DEV_FREE_FN),
                ("alloc_ctx", C.c_void_p), ("autotune", C.c_int32), ("pow2_scaling", C.c_int32),
                ("tile_mult", C.c_int32)]


class rhpdhg_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("out_memory", C.c_int32), ("cert_source", C.c_int32),
                ("escalated", C.c_int32), ("iters", C.c_int64),
                ("restarts", C.c_int64), ("rel_p", C.c_double), ("rel_d", C.c_double),
                ("rel_gap", C.c_double), ("primal_obj", C.c_double), ("dual_obj", C.c_double),
                ("solve_seconds", C.c_double), ("eta", C.c_double), ("omega", C.c_double),
                ("sigma_max", C.c_double), ("x", C.c_void_p), ("y", C.c_void_p),
                ("cert_x", C.c_void_p), ("cert_y", C.c_void_p)]


class rhpdhg_trace_rec(C.Structure):
    _fields_ = [("t", C.c_int64), ("epoch", C.c_int64), ("k", C.c_int64),
                ("fpr_sq", C.c_double), ("omega", C.c_double), ("restart", C.c_int32),
                ("retries", C.c_int32), ("active", C.c_int64), ("changed", C.c_int64)]


EXPORTED = ["rhpdhg_params_default", "rhpdhg_create", "rhpdhg_solve", "rhpdhg_poll",
            "rhpdhg_cancel", "rhpdhg_free", "rhpdhg_last_error", "rhpdhg_get_state",
            "rhpdhg_get_scaling", "rhpdhg_get_trace", "rhpdhg_get_layout", "rhpdhg_plan_layout",
            "rhpdhg_release_cached_memory",
            "rhpdhg_kernel_times",
            "rhpdhg_launch_count", "rhpdhg_kkt_eval", "rhpdhg_kkt_eval_noalloc",
            "rhpdhg_batch_create", "rhpdhg_batch_add", "rhpdhg_batch_step", "rhpdhg_batch_poll",
            "rhpdhg_batch_remove", "rhpdhg_batch_slot_status", "rhpdhg_batch_free_bytes",
            "rhpdhg_batch_bytes_needed", "rhpdhg_batch_launch_count", "rhpdhg_batch_free",
            "rhpdhg_server_create", "rhpdhg_server_submit", "rhpdhg_server_poll",
            "rhpdhg_server_cancel", "rhpdhg_server_stats", "rhpdhg_server_free",
            "rhpdhg_probe_fp64_fma_rate", "rhpdhg_probe_l2_read_bandwidth"]

_lib = None


def load(path: str = LIB_PATH):
    """Load librhpdhg.so (built by ``__graft_entry__.build()``) and declare the signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    H = C.c_void_p
    sig = {
        "rhpdhg_params_default": (C.c_int, [C.POINTER(rhpdhg_params)]),
        "rhpdhg_create": (C.c_int, [C.POINTER(rhpdhg_problem), C.POINTER(rhpdhg_params),
                                    C.c_void_p, C.POINTER(H)]),
        "rhpdhg_solve": (C.c_int, [H, C.c_int]),
        "rhpdhg_poll": (C.c_int, [H, C.POINTER(rhpdhg_result)]),
        "rhpdhg_cancel": (C.c_int, [H]),
        "rhpdhg_free": (None, [H]),
        "rhpdhg_last_error": (C.c_char_p, [H]),
        "rhpdhg_get_state": (C.c_int, [H, C.c_int, _dp, _dp]),
        "rhpdhg_get_scaling": (C.c_int, [H, _dp, _dp, _dp, _dp, _dp]),
        "rhpdhg_get_trace": (C.c_int, [H, C.POINTER(rhpdhg_trace_rec), C.c_int64,
                                       C.POINTER(C.c_int64)]),
        "rhpdhg_get_layout": (C.c_int, [H, C.POINTER(C.c_int64), C.c_int32]),
        "rhpdhg_plan_layout": (C.c_int, [C.POINTER(C.c_int64), C.c_int32, C.POINTER(C.c_int64),
                                         C.c_int32]),
        "rhpdhg_release_cached_memory": (C.c_int64, []),
        "rhpdhg_kernel_times": (C.c_int, [H, _dp, _dp, C.POINTER(C.c_int64),
                                          C.POINTER(C.c_int64), _dp, _dp]),
        "rhpdhg_launch_count": (C.c_int64, [H]),
        "rhpdhg_kkt_eval": (C.c_int, [C.POINTER(rhpdhg_problem), C.c_void_p, C.c_void_p,
                                      C.c_void_p, _dp]),
        "rhpdhg_kkt_eval_noalloc": (C.c_int, [C.POINTER(rhpdhg_problem), C.c_void_p,
                                              C.c_void_p, C.c_void_p, _dp]),
        "rhpdhg_batch_create": (C.c_int, [C.c_int32, C.c_int64, C.c_void_p, C.POINTER(H)]),
        "rhpdhg_batch_add": (C.c_int, [H, C.POINTER(rhpdhg_problem), C.POINTER(rhpdhg_params),
                                       C.POINTER(C.c_int32)]),
        "rhpdhg_batch_step": (C.c_int, [H, C.c_int32]),
        "rhpdhg_batch_poll": (C.c_int, [H, C.c_int32, C.POINTER(rhpdhg_result)]),
        "rhpdhg_batch_remove": (C.c_int, [H, C.c_int32]),
        "rhpdhg_batch_slot_status": (C.c_int, [H, C.c_int32]),
        "rhpdhg_batch_free_bytes": (C.c_int64, [H]),
        "rhpdhg_batch_bytes_needed": (C.c_int64, [C.POINTER(rhpdhg_problem), C.c_int32]),
        "rhpdhg_batch_launch_count": (C.c_int64, [H]),
        "rhpdhg_batch_free": (None, [H]),
        "rhpdhg_server_create": (C.c_int, [C.c_int64, C.c_int64, C.c_int32, C.c_int32,
                                           C.POINTER(H)]),
        "rhpdhg_server_submit": (C.c_int, [H, C.POINTER(rhpdhg_problem),
                                           C.POINTER(rhpdhg_params), C.POINTER(C.c_int64)]),
        "rhpdhg_server_poll": (C.c_int, [H, C.c_int64, C.POINTER(rhpdhg_result), _dp]),
        "rhpdhg_server_cancel": (C.c_int, [H, C.c_int64]),
        "rhpdhg_server_stats": (C.c_int, [H, C.POINTER(C.c_int64)]),
        "rhpdhg_server_free": (None, [H]),
        "rhpdhg_probe_fp64_fma_rate": (C.c_int, [C.c_void_p, _dp]),
        "rhpdhg_probe_l2_read_bandwidth": (C.c_int, [C.c_int64, C.c_void_p, _dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


# ---- same-named wrappers ---------------------------------------------------------------------

def rhpdhg_params_default(p: rhpdhg_params) -> int:
    return load().rhpdhg_params_default(C.byref(p))


def rhpdhg_create(lp: rhpdhg_problem, params: rhpdhg_params, stream: int = 0):
    h = C.c_void_p()
    rc = load().rhpdhg_create(C.byref(lp), C.byref(params), C.c_void_p(stream or None),
                              C.byref(h))
    return rc, h


def rhpdhg_solve(h, blocking: int = 1) -> int:
    return load().rhpdhg_solve(h, blocking)


def rhpdhg_poll(h, r: rhpdhg_result) -> int:
    return load().rhpdhg_poll(h, C.byref(r))


def rhpdhg_cancel(h) -> int:
    return load().rhpdhg_cancel(h)


def rhpdhg_free(h) -> None:
    load().rhpdhg_free(h)


def rhpdhg_last_error(h=None) -> str:
    s = load().rhpdhg_last_error(h)
    return s.decode() if s else ""


def rhpdhg_get_state(h, which: int, x, y) -> int:
    return load().rhpdhg_get_state(h, which, _ptr(x), _ptr(y))


def rhpdhg_get_scaling(h, D, E):
    eta, om, sm = C.c_double(), C.c_double(), C.c_double()
    rc = load().rhpdhg_get_scaling(h, _ptr(D), _ptr(E), C.byref(eta), C.byref(om), C.byref(sm))
    return rc, eta.value, om.value, sm.value


def rhpdhg_get_trace(h, capacity: int):
    recs = (rhpdhg_trace_rec * max(capacity, 1))()
    cnt = C.c_int64()
    rc = load().rhpdhg_get_trace(h, recs, capacity, C.byref(cnt))
    return rc, [recs[i] for i in range(min(cnt.value, capacity))]


LAYOUT_FIELDS = ("grid_row", "grid_col", "tile_mult_row", "tile_mult_col", "long_rows_row",
                 "long_rows_col", "chunks_row", "chunks_col", "seg_row", "seg_col", "walk_row",
                 "walk_col", "cta_warps_row", "cta_warps_col", "tuned", "tune_ns_rule",
                 "tune_ns_best", "wide_rows_row", "wide_rows_col")


def rhpdhg_get_layout(h):
    out = (C.c_int64 * len(LAYOUT_FIELDS))()
    rc = load().rhpdhg_get_layout(h, out, len(LAYOUT_FIELDS))
    return rc, dict(zip(LAYOUT_FIELDS, list(out)))


def release_cached_memory() -> int:
    """Frees the device buffers cached from freed handles; returns the bytes freed."""
    return int(load().rhpdhg_release_cached_memory())


PLAN_FIELDS = ("tiles", "tile_mult", "long_rows", "chunks", "seg", "nnz_short", "nnz_long",
               "wide_rows")


def rhpdhg_plan_layout(row_ptr):
    """Layout plan of an operator side from its CSR row pointers (host only, no device)."""
    rp = np.ascontiguousarray(np.asarray(row_ptr, dtype=np.int64))
    out = (C.c_int64 * len(PLAN_FIELDS))()
    rc = load().rhpdhg_plan_layout(rp.ctypes.data_as(C.POINTER(C.c_int64)), len(rp) - 1, out,
                                   len(PLAN_FIELDS))
    return rc, dict(zip(PLAN_FIELDS, list(out)))


def rhpdhg_kernel_times(h):
    a, b, e, f = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    c, d = C.c_int64(), C.c_int64()
    rc = load().rhpdhg_kernel_times(h, C.byref(a), C.byref(b), C.byref(c), C.byref(d),
                                    C.byref(e), C.byref(f))
    return rc, dict(ms_row=a.value, ms_col=b.value, launches_row=c.value,
                    launches_col=d.value, bytes_row=e.value, bytes_col=f.value)


def rhpdhg_launch_count(h) -> int:
    return load().rhpdhg_launch_count(h)


def rhpdhg_kkt_eval(lp: rhpdhg_problem, x, y, stream: int = 0):
    """x, y: device pointers (int).  Returns (rc, [rel_p, rel_d, rel_gap, primal_obj,
    dual_obj])."""
    out = (C.c_double * 5)()
    rc = load().rhpdhg_kkt_eval(C.byref(lp), C.c_void_p(x), C.c_void_p(y or None),
                                C.c_void_p(stream or None), out)
    return rc, list(out)


def rhpdhg_kkt_eval_noalloc(lp: rhpdhg_problem, x, y, stream: int = 0):
    """As rhpdhg_kkt_eval, on the library's fixed scratch (allocates no device memory)."""
    out = (C.c_double * 5)()
    rc = load().rhpdhg_kkt_eval_noalloc(C.byref(lp), C.c_void_p(x), C.c_void_p(y or None),
                                        C.c_void_p(stream or None), out)
    return rc, list(out)


def rhpdhg_probe_fp64_fma_rate(stream: int = 0):
    """Returns (rc, FP64 FMA rate in TFLOP/s of the current device)."""
    v = C.c_double()
    rc = load().rhpdhg_probe_fp64_fma_rate(C.c_void_p(stream or None), C.byref(v))
    return rc, v.value


def rhpdhg_probe_l2_read_bandwidth(nbytes: int, stream: int = 0):
    """Returns (rc, read bandwidth in GB/s of a device buffer of nbytes)."""
    v = C.c_double()
    rc = load().rhpdhg_probe_l2_read_bandwidth(nbytes, C.c_void_p(stream or None), C.byref(v))
    return rc, v.value


def rhpdhg_batch_create(max_slots: int, arena_bytes: int, stream: int = 0):
    h = C.c_void_p()
    rc = load().rhpdhg_batch_create(max_slots, arena_bytes, C.c_void_p(stream or None),
                                    C.byref(h))
    return rc, h


def rhpdhg_batch_add(b, lp: rhpdhg_problem, params: Optional[rhpdhg_params]):
    slot = C.c_int32(-1)
    rc = load().rhpdhg_batch_add(b, C.byref(lp), C.byref(params) if params else None,
                                 C.byref(slot))
    return rc, slot.value


def rhpdhg_batch_step(b, iters: int) -> int:
    return load().rhpdhg_batch_step(b, iters)


def rhpdhg_batch_poll(b, slot: int, r: rhpdhg_result) -> int:
    return load().rhpdhg_batch_poll(b, slot, C.byref(r))


def rhpdhg_batch_remove(b, slot: int) -> int:
    return load().rhpdhg_batch_remove(b, slot)


def rhpdhg_batch_slot_status(b, slot: int) -> int:
    return load().rhpdhg_batch_slot_status(b, slot)


def rhpdhg_batch_free_bytes(b) -> int:
    return load().rhpdhg_batch_free_bytes(b)


def rhpdhg_batch_bytes_needed(lp: rhpdhg_problem, precision: int = 0) -> int:
    return load().rhpdhg_batch_bytes_needed(C.byref(lp), precision)


def rhpdhg_batch_launch_count(b) -> int:
    return load().rhpdhg_batch_launch_count(b)


def rhpdhg_batch_free(b) -> None:
    load().rhpdhg_batch_free(b)


def rhpdhg_server_create(budget_bytes: int, small_nnz: int, max_slots: int,
                         iters_per_step: int):
    h = C.c_void_p()
    rc = load().rhpdhg_server_create(budget_bytes, small_nnz, max_slots, iters_per_step,
                                     C.byref(h))
    return rc, h


def rhpdhg_server_submit(s, lp: rhpdhg_problem, params: Optional[rhpdhg_params]):
    t = C.c_int64(0)
    rc = load().rhpdhg_server_submit(s, C.byref(lp), C.byref(params) if params else None,
                                     C.byref(t))
    return rc, t.value


def rhpdhg_server_poll(s, ticket: int, r: rhpdhg_result):
    lat = C.c_double(0.0)
    rc = load().rhpdhg_server_poll(s, ticket, C.byref(r), C.byref(lat))
    return rc, lat.value


def rhpdhg_server_cancel(s, ticket: int) -> int:
    return load().rhpdhg_server_cancel(s, ticket)


def rhpdhg_server_stats(s) -> dict:
    out = (C.c_int64 * 10)()
    load().rhpdhg_server_stats(s, out)
    keys = ["pending", "running_batched", "running_single", "completed", "bytes_in_use",
            "peak_bytes_in_use", "budget", "batched_launches", "admitted_batched",
            "admitted_single"]
    return dict(zip(keys, list(out)))


def rhpdhg_server_free(s) -> None:
    load().rhpdhg_server_free(s)


class Server:
    """Owns a serving loop (rhpdhg_server_*)."""

    def __init__(self, budget_bytes: int, small_nnz: int = 200_000, max_slots: int = 256,
                 iters_per_step: int = 64):
        rc, self.s = rhpdhg_server_create(budget_bytes, small_nnz, max_slots, iters_per_step)
        _check(rc, None, "rhpdhg_server_create")
        self._shape = {}

    def submit(self, lp, **params) -> int:
        keep = []
        prob = host_problem(lp, keep)
        p = default_params(**params)
        rc, t = rhpdhg_server_submit(self.s, prob, p)
        _check(rc, None, "rhpdhg_server_submit")
        self._shape[t] = (int(lp.n), int(lp.m_eq) + int(lp.m_ineq))
        return t

    def poll(self, ticket: int):
        n, m = self._shape[ticket]
        r = rhpdhg_result()
        x, y = np.empty(n), np.empty(max(m, 1))
        cx, cy = np.zeros(n), np.zeros(max(m, 1))
        r.x, r.y, r.cert_x, r.cert_y = x.ctypes.data, y.ctypes.data, cx.ctypes.data, cy.ctypes.data
        rc, lat = rhpdhg_server_poll(self.s, ticket, r)
        if rc == BUSY:
            return None
        _check(rc, None, "rhpdhg_server_poll")
        self._shape.pop(ticket)
        res = Result(status=r.status, cert_source=r.cert_source, escalated=r.escalated,
                     iters=r.iters, restarts=r.restarts, rel_p=r.rel_p,
                     rel_d=r.rel_d, rel_gap=r.rel_gap, primal_obj=r.primal_obj,
                     dual_obj=r.dual_obj, solve_seconds=r.solve_seconds, eta=r.eta,
                     omega=r.omega, sigma_max=r.sigma_max, x=x, y=y[:m], cert_x=cx,
                     cert_y=cy[:m])
        return res, lat

    def cancel(self, ticket: int):
        rhpdhg_server_cancel(self.s, ticket)

    def stats(self) -> dict:
        return rhpdhg_server_stats(self.s)

    def close(self):
        if getattr(self, "s", None):
            rhpdhg_server_free(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def host_problem(lp, keep: list) -> rhpdhg_problem:
    """rhpdhg_problem over an lpgen.LP's host arrays (contiguous copies appended to keep)."""
    prob = rhpdhg_problem()
    prob.m_eq, prob.m_ineq, prob.n = int(lp.m_eq), int(lp.m_ineq), int(lp.n)
    prob.memory = MEM_HOST
    prob.obj_offset = float(getattr(lp, "obj_offset", 0.0))
    arrs = dict(row_ptr=np.ascontiguousarray(lp.row_ptr, dtype=np.int64),
                col_idx=np.ascontiguousarray(lp.col_idx, dtype=np.int32),
                val=np.ascontiguousarray(lp.val, dtype=np.float64),
                c=np.ascontiguousarray(lp.c, dtype=np.float64),
                rhs=np.ascontiguousarray(lp.q, dtype=np.float64),
                l=np.ascontiguousarray(lp.l, dtype=np.float64),
                u=np.ascontiguousarray(lp.u, dtype=np.float64))
    keep.append(arrs)
    prob.nnz = int(arrs["row_ptr"][-1])
    for f, a in arrs.items():
        setattr(prob, f, a.ctypes.data if a.size else None)
    if prob.row_ptr is None:
        prob.row_ptr = arrs["row_ptr"].ctypes.data
    return prob


class Batch:
    """Owns a batched solver (rhpdhg_batch_*): add LPs, step, poll results."""

    def __init__(self, max_slots: int, arena_bytes: int, stream: int = 0):
        rc, self.b = rhpdhg_batch_create(max_slots, arena_bytes, stream)
        _check(rc, None, "rhpdhg_batch_create")
        self._keep = {}
        self._shape = {}

    def add(self, lp, **params) -> int:
        keep = []
        prob = host_problem(lp, keep)
        p = default_params(**params)
        rc, slot = rhpdhg_batch_add(self.b, prob, p)
        if rc == BUSY:
            return -1
        _check(rc, None, "rhpdhg_batch_add")
        self._keep[slot] = keep
        self._shape[slot] = (int(lp.n), int(lp.m_eq) + int(lp.m_ineq))
        return slot

    def step(self, iters: int = 64):
        _check(rhpdhg_batch_step(self.b, iters), None, "rhpdhg_batch_step")

    def status(self, slot: int) -> int:
        return rhpdhg_batch_slot_status(self.b, slot)

    def poll(self, slot: int, remove: bool = True):
        n, m = self._shape[slot]
        r = rhpdhg_result()
        x, y = np.empty(n), np.empty(max(m, 1))
        cx, cy = np.zeros(n), np.zeros(max(m, 1))
        r.x, r.y, r.cert_x, r.cert_y = x.ctypes.data, y.ctypes.data, cx.ctypes.data, cy.ctypes.data
        rc = rhpdhg_batch_poll(self.b, slot, r)
        if rc == BUSY:
            return None
        _check(rc, None, "rhpdhg_batch_poll")
        res = Result(status=r.status, cert_source=r.cert_source, escalated=r.escalated,
                     iters=r.iters, restarts=r.restarts, rel_p=r.rel_p,
                     rel_d=r.rel_d, rel_gap=r.rel_gap, primal_obj=r.primal_obj,
                     dual_obj=r.dual_obj, solve_seconds=0.0, eta=r.eta, omega=r.omega,
                     sigma_max=r.sigma_max, x=x, y=y[:m], cert_x=cx, cert_y=cy[:m])
        if remove:
            self.remove(slot)
        return res

    def remove(self, slot: int):
        _check(rhpdhg_batch_remove(self.b, slot), None, "rhpdhg_batch_remove")
        self._keep.pop(slot, None)

    def free_bytes(self) -> int:
        return rhpdhg_batch_free_bytes(self.b)

    def launch_count(self) -> int:
        return rhpdhg_batch_launch_count(self.b)

    def run_all(self, slots, iters: int = 64, max_steps: int = 100_000):
        out = {}
        for _ in range(max_steps):
            self.step(iters)
            for s in slots:
                if s not in out and self.status(s) != STATUS_RUNNING:
                    out[s] = self.poll(s)
            if len(out) == len(slots):
                return out
        raise RHPDHGError("batch did not finish")

    def close(self):
        if getattr(self, "b", None):
            rhpdhg_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def device_problem(lp) -> rhpdhg_problem:
    """rhpdhg_problem describing an LP whose arrays are torch CUDA tensors (the caller keeps
    them alive)."""
    prob = rhpdhg_problem()
    prob.m_eq, prob.m_ineq, prob.n = int(lp.m_eq), int(lp.m_ineq), int(lp.n)
    prob.memory = MEM_DEVICE
    prob.nnz = int(lp.row_ptr[-1].item())
    for f in ("row_ptr", "col_idx", "val", "c", "l", "u"):
        setattr(prob, f, int(getattr(lp, f).data_ptr()))
    prob.rhs = int(lp.q.data_ptr()) if prob.m_eq + prob.m_ineq else None
    prob.obj_offset = float(getattr(lp, "obj_offset", 0.0))
    return prob


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data_as(_dp)
    return C.cast(C.c_void_p(int(a)), _dp)


# ---- convenience wrapper ---------------------------------------------------------------------

class RHPDHGError(RuntimeError):
    pass


def _check(rc, h=None, what=""):
    if rc < 0:
        raise RHPDHGError(f"{what} failed ({rc}): {rhpdhg_last_error(h)}")
    return rc


class TorchAllocator:
    """Device allocator callbacks for rhpdhg_params.dev_alloc / dev_free that take a handle's
    device memory from PyTorch's caching allocator (torch.cuda.caching_allocator_alloc on the
    handle's stream, caching_allocator_delete to give it back), so the solver's buffers count in
    torch's memory statistics and are reused by torch after the handle is freed.  Keep the
    object alive as long as any handle created with it."""

    def __init__(self, device=None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.live = {}

        def _alloc(nbytes, stream, ctx):
            try:
                ptr = self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                               int(stream or 0))
            except Exception:
                return None
            self.live[ptr] = int(nbytes)
            return ptr

        def _free(ptr, stream, ctx):
            if ptr in self.live:
                del self.live[ptr]
                self._torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = DEV_ALLOC_FN(_alloc)
        self.free_fn = DEV_FREE_FN(_free)

    def apply(self, p: "rhpdhg_params"):
        p.dev_alloc = self.alloc_fn
        p.dev_free = self.free_fn
        p.alloc_ctx = None


def default_params(**kw) -> rhpdhg_params:
    p = rhpdhg_params()
    _check(rhpdhg_params_default(p))
    for k, v in kw.items():
        if k in ("x0", "y0"):
            continue
        if k == "allocator":
            v.apply(p)
            continue
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


@dataclasses.dataclass
class Result:
    status: int
    iters: int
    restarts: int
    rel_p: float
    rel_d: float
    rel_gap: float
    primal_obj: float
    dual_obj: float
    solve_seconds: float
    eta: float
    omega: float
    sigma_max: float
    x: np.ndarray
    y: np.ndarray
    cert_x: np.ndarray
    cert_y: np.ndarray
    cert_source: int = 0     # CERT_* of an infeasibility status
    escalated: int = 0       # 1 if a mixed-precision solve continued in FP64

    @property
    def status_name(self) -> str:
        return STATUS_NAMES[self.status]

    @property
    def rel_kkt(self) -> float:
        return max(self.rel_p, self.rel_d, self.rel_gap)


class Solver:
    """Owns one library handle for one LP.

    ``lp`` is an ``lpgen.LP`` (host numpy arrays) or a mapping of torch CUDA tensors with the
    same field names (``device=True``).  ``stream`` is a CUDA stream handle (int) or 0.
    """

    def __init__(self, lp, stream: int = 0, device: bool = False, **params):
        self._keep = []
        self.m_eq, self.m_ineq, self.n = int(lp.m_eq), int(lp.m_ineq), int(lp.n)
        self.m = self.m_eq + self.m_ineq
        prob = rhpdhg_problem()
        prob.m_eq, prob.m_ineq, prob.n = self.m_eq, self.m_ineq, self.n
        prob.memory = MEM_DEVICE if device else MEM_HOST
        prob.obj_offset = float(getattr(lp, "obj_offset", 0.0))
        if device:
            prob.nnz = int(lp.row_ptr[-1].item())
            for f in ("row_ptr", "col_idx", "val", "c", "l", "u"):
                setattr(prob, f, int(getattr(lp, f).data_ptr()))
            prob.rhs = int(lp.q.data_ptr()) if self.m else None
        else:
            rp = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
            ci = np.ascontiguousarray(lp.col_idx, dtype=np.int32)
            va = np.ascontiguousarray(lp.val, dtype=np.float64)
            arrs = dict(row_ptr=rp, col_idx=ci, val=va,
                        c=np.ascontiguousarray(lp.c, dtype=np.float64),
                        rhs=np.ascontiguousarray(lp.q, dtype=np.float64),
                        l=np.ascontiguousarray(lp.l, dtype=np.float64),
                        u=np.ascontiguousarray(lp.u, dtype=np.float64))
            self._keep.append(arrs)
            prob.nnz = int(rp[-1])
            for f, a in arrs.items():
                setattr(prob, f, a.ctypes.data if a.size else None)
            if prob.row_ptr is None:
                prob.row_ptr = arrs["row_ptr"].ctypes.data
        p = default_params(**params)
        x0, y0 = params.get("x0"), params.get("y0")
        if x0 is not None:
            x0 = np.ascontiguousarray(x0, dtype=np.float64)
            self._keep.append(x0)
            p.x0 = x0.ctypes.data
        if y0 is not None:
            y0 = np.ascontiguousarray(y0, dtype=np.float64)
            self._keep.append(y0)
            p.y0 = y0.ctypes.data
        self.params = p
        rc, self.h = rhpdhg_create(prob, p, stream)
        _check(rc, None, "rhpdhg_create")

    def solve(self, blocking: int = 1) -> int:
        return _check(rhpdhg_solve(self.h, blocking), self.h, "rhpdhg_solve")

    def poll(self, x=None, y=None, cert_x=None, cert_y=None, out_memory=MEM_HOST):
        r = rhpdhg_result()
        r.out_memory = out_memory
        if out_memory == MEM_HOST:
            x = np.empty(self.n) if x is None else x
            y = np.empty(self.m) if y is None else y
            cert_x = np.zeros(self.n) if cert_x is None else cert_x
            cert_y = np.zeros(self.m) if cert_y is None else cert_y
            r.x, r.y = x.ctypes.data, (y.ctypes.data if self.m else None)
            r.cert_x = cert_x.ctypes.data
            r.cert_y = cert_y.ctypes.data if self.m else None
        else:
            for f, a in (("x", x), ("y", y), ("cert_x", cert_x), ("cert_y", cert_y)):
                setattr(r, f, int(a.data_ptr()) if a is not None else None)
        rc = rhpdhg_poll(self.h, r)
        if rc == BUSY:
            return None
        _check(rc, self.h, "rhpdhg_poll")
        return Result(status=r.status, cert_source=r.cert_source, escalated=r.escalated,
                      iters=r.iters, restarts=r.restarts, rel_p=r.rel_p,
                      rel_d=r.rel_d, rel_gap=r.rel_gap, primal_obj=r.primal_obj,
                      dual_obj=r.dual_obj, solve_seconds=r.solve_seconds, eta=r.eta,
                      omega=r.omega, sigma_max=r.sigma_max, x=x, y=y, cert_x=cert_x,
                      cert_y=cert_y)

    def run(self) -> Result:
        self.solve(1)
        return self.poll()

    def state(self, which: int = 1):
        x, y = np.empty(self.n), np.empty(max(self.m, 1))
        _check(rhpdhg_get_state(self.h, which, x, y), self.h, "rhpdhg_get_state")
        return x, y[:self.m]

    def scaling(self):
        D, E = np.empty(max(self.m, 1)), np.empty(self.n)
        rc, eta, om, sm = rhpdhg_get_scaling(self.h, D, E)
        _check(rc, self.h, "rhpdhg_get_scaling")
        return D[:self.m], E, eta, om, sm

    def trace(self, capacity: int = 1 << 16):
        rc, recs = rhpdhg_get_trace(self.h, capacity)
        _check(rc, self.h, "rhpdhg_get_trace")
        return [(r.t, r.epoch, r.k, r.fpr_sq, bool(r.restart), r.omega, r.active, r.changed,
                 r.retries) for r in recs]

    def layout(self):
        """Launch geometry and walk layout chosen at create (see LAYOUT_FIELDS)."""
        rc, d = rhpdhg_get_layout(self.h)
        _check(rc, self.h, "rhpdhg_get_layout")
        return d

    def kernel_times(self):
        rc, d = rhpdhg_kernel_times(self.h)
        _check(rc, self.h, "rhpdhg_kernel_times")
        return d

    def launch_count(self) -> int:
        return rhpdhg_launch_count(self.h)

    def cancel(self):
        rhpdhg_cancel(self.h)

    def close(self):
        if getattr(self, "h", None):
            rhpdhg_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
