"""Store a sample of the FP64 oracle's solution of the 16^3x32, Ls=16
benchmark solve, for the element-by-element GPU comparison.

The oracle (unpreconditioned CGNR on the full-lattice H-form system of Eq.
generic_eofa_system) solves phi = (H(m1) + beta Delta_+(m2, m3) P_+) psi to a
relative residual of 1e-12, and the solution psi at 48 fixed 4D sites (all
Ls slices, spins and colours) is written to oracle_psi_16x16x16x32_Ls16.npz
beside this script, with the sites, the residual and the iteration count.
It calls only oracle/ and the seeded input generators; it runs for hours on
the host cores.

    python tests/golden/oracle_solution_sample.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1706_05843_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "oracle_psi_16x16x16x32_Ls16.npz")
DIMS, LS, EPS, GAUGE_SEED, RHS_SEED = (16, 16, 16, 32), 16, 0.5, 1, 1001
ACTION = dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, beta=-1.0, pm=1, t_bc=-1)
TOL = 1e-12
N_SITES, SITE_SEED = 48, 5


def sample_sites():
    V = int(np.prod(DIMS))
    return np.sort(np.random.default_rng(SITE_SEED).choice(V, N_SITES, replace=False))


def main():
    oracle.build()
    U = I.gauge_field(DIMS, EPS, GAUGE_SEED)
    phi = I.gaussian_fermion(DIMS, LS, RHS_SEED)
    o = oracle.Oracle(oracle.Action(dims=DIMS, Ls=LS, **ACTION), U)
    t0 = time.time()
    psi, st = o.solve_h(phi, tol=TOL, maxit=400000)
    res = float(np.linalg.norm(phi - o.hsys(psi)) / np.linalg.norm(phi))
    sites = sample_sites()
    np.savez_compressed(OUT, sites=sites, psi=psi.reshape(-1, LS, 4, 3)[sites], residual=res,
                        iters=st.iters, converged=bool(st.converged), tol=TOL, seconds=time.time() - t0,
                        threads=oracle.num_threads())
    print(f"stored {OUT}: residual {res:.3e} after {st.iters} iterations, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
