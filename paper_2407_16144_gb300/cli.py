"""Command-line solve of a generated workload through the C ABI.

    python -m paper_2407_16144_gb300.cli --workload c2 --tol 1e-6 [--precision 1]
        [--algorithm 0|1] [--max-iters N] [--scale S] [--repeat R] [--autotune 1]
        [--cta-warps 4|8|16] [--df-sums 0|1]

Workloads (all from lpgen, seeded): c1 = 200 x 500 planted standard form; c2 = 100k x 250k
general form with power-law columns (--scale shrinks it); c3 = multicommodity flow, 20
commodities on 250k nodes / 2M arcs (120M nonzeros; --scale shrinks the graph); c4p = 50k x 100k primal-infeasible
LP with a planted Farkas vector; c4d = its dual twin (100k inequality rows over 50k free
variables, unbounded along the planted vector); c4s = a 50k x 100k standard-form LP unbounded
along a sparse planted ray.  Prints one JSON line per solve.
"""
from __future__ import annotations

import argparse
import json
import time


def make(workload: str, scale: float):
    from . import lpgen
    if workload == "c1":
        return lpgen.make_c1(0)
    if workload == "c2":
        return lpgen.make_c2(1, scale=scale)
    if workload == "c3":
        return lpgen.make_multicommodity_flow(2, max(10, int(250_000 * scale)),
                                              max(20, int(2_000_000 * scale)))
    if workload == "c4p":
        return lpgen.make_primal_infeasible(3, int(50_000 * scale), int(100_000 * scale))
    if workload == "c4d":
        return lpgen.make_dual_infeasible_twin(3, int(50_000 * scale), int(100_000 * scale))
    if workload == "c4s":
        return lpgen.make_dual_infeasible(3, int(50_000 * scale), int(100_000 * scale))
    raise SystemExit(f"unknown workload {workload}")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--algorithm", type=int, default=1)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--max-iters", type=int, default=10_000_000)
    ap.add_argument("--max-epoch-len", type=int, default=1000)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--profile", type=int, default=0)
    ap.add_argument("--time-limit", type=float, default=3600.0)
    ap.add_argument("--autotune", type=int, default=0)
    ap.add_argument("--cta-warps", type=int, default=0)
    ap.add_argument("--df-sums", type=int, default=0)
    a = ap.parse_args(argv)
    from . import rhpdhg
    rhpdhg.load()
    lp = make(a.workload, a.scale)
    for _ in range(a.repeat):
        t0 = time.perf_counter()
        with rhpdhg.Solver(lp, algorithm=a.algorithm, precision=a.precision, eps_rel_kkt=a.tol,
                           max_iters=a.max_iters, max_epoch_len=a.max_epoch_len,
                           profile=a.profile, time_limit_s=a.time_limit,
                           autotune=a.autotune, cta_warps=a.cta_warps, df_sums=a.df_sums) as s:
            t1 = time.perf_counter()
            r = s.run()
            kt = s.kernel_times() if a.profile else None
        print(json.dumps(dict(workload=a.workload, m=lp.m, n=lp.n, nnz=lp.nnz,
                              status=r.status_name, iters=r.iters, restarts=r.restarts,
                              rel_kkt=r.rel_kkt, primal_obj=r.primal_obj,
                              dual_obj=r.dual_obj, create_s=t1 - t0,
                              solve_s=r.solve_seconds, iters_per_s=r.iters / r.solve_seconds,
                              kernel_times=kt)), flush=True)


if __name__ == "__main__":
    main()
