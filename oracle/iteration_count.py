"""Record the oracle's own CGNR iteration count on a benchmark workload.

The CPU baseline of bench.py times a bounded sample of oracle iterations on
the full workload; this script runs the oracle solve to completion once and
stores how many iterations it needed, so the sample can be scaled to
seconds per solve.  It calls only oracle/ and the seeded input generators.

    python -m oracle.iteration_count            # 16^3x32, Ls=16 workload
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1706_05843_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "iteration_counts.json")

WORKLOADS = {
    "16^3x32_Ls16": dict(dims=(16, 16, 16, 32), Ls=16, eps=0.5, gauge_seed=1, rhs_seed=1001,
                         action=dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04,
                                     beta=-1.0, pm=1, t_bc=-1)),
}


def run(name: str, tol: float = 1e-10) -> dict:
    w = WORKLOADS[name]
    U = I.gauge_field(w["dims"], w["eps"], w["gauge_seed"])
    phi = I.gaussian_fermion(w["dims"], w["Ls"], w["rhs_seed"])
    o = oracle.Oracle(oracle.Action(dims=w["dims"], Ls=w["Ls"], **w["action"]), U)
    t0 = time.time()
    _, st = o.solve_h(phi, tol=tol, maxit=200000)
    return {"iters": st.iters, "converged": bool(st.converged), "true_res": st.true_res,
            "recur_res": st.recur_res, "tol": tol, "seconds": time.time() - t0,
            "threads": oracle.num_threads(), "solver": "oracle CGNR, unpreconditioned, H form"}


def main():
    names = sys.argv[1:] or list(WORKLOADS)
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for n in names:
        data[n] = run(n)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(n, data[n], flush=True)


if __name__ == "__main__":
    main()
