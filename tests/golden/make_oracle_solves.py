"""Writes tests/golden/oracle_solves.json: full solves of the FP64 oracle (and nothing else) on
seeded workloads too large to solve inside a GPU test run on the test machine's host cores.

Each entry records the oracle's status, iteration and restart counts, objectives and rel-KKT
parts at the returned point for one (workload, algorithm, tolerance).  The GPU tests compare the
library's objective with these values.  Re-run after any change to the oracle's arithmetic or to
the generators:

    python tests/golden/make_oracle_solves.py
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import rhpdhg_oracle as O  # noqa: E402
from paper_2407_16144_gb300 import lpgen  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_solves.json")

RUNS = [
    # (key, generator call, algorithm, tolerance)
    ("c2_seed1_alg1_1e-8", "make_c2(1)", 1, 1e-8),
]


def main():
    res = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            res = json.load(f)
    for key, gen, alg, tol in RUNS:
        lp = eval("lpgen." + gen)
        t0 = time.perf_counter()
        r = O.solve(lp, O.OracleParams(algorithm=alg, eps_rel_kkt=tol, max_iters=1_000_000))
        res[key] = {"generator": gen, "algorithm": alg, "eps_rel_kkt": tol,
                    "status": r.status, "iters": r.iters, "restarts": r.restarts,
                    "primal_obj": r.primal_obj, "dual_obj": r.dual_obj, "rel_p": r.rel_p,
                    "rel_d": r.rel_d, "rel_gap": r.rel_gap,
                    "planted_objective": float(lp.planted_objective()),
                    "oracle_seconds": round(time.perf_counter() - t0, 1)}
        print(key, res[key], flush=True)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
