"""Host-side tuning around the EOFA heatbath (Sec. III.B, Sec. V.B).

The heatbath itself, phi = M_EOFA^(-1/2) eta by Eq. (eofa_heatbath), runs in
the library (``Solver.heatbath``): 2 N_p H-form solves on the GPU.  This
module holds the set-up a caller performs around it:

  * an estimate of the largest eigenvalue of M_EOFA by power iteration with
    the library's M_EOFA application, for the interval of the rational
    approximation (the smallest is close to 1 for EOFA, Sec. III.B);
  * the heatbath error epsilon of Eq. (heatbath_rel_err);
  * the paper's per-solve stopping-tolerance tuning (Sec. V.B): for each
    of the 2 N_p solves in turn, relax its tolerance while the heatbath error
    stays below a target.

Inner products of the 4D fields are the solver's (``solver.dot``: the
library's FP64 device reduction), so no field leaves the device.
"""
from __future__ import annotations

import math


def heatbath_error(solver, eta, phi, m_phi) -> float:
    """epsilon = |eta^dag eta - phi^dag M_EOFA phi| / eta^dag eta."""
    ee = solver.dot(eta, eta).real
    return abs(ee - solver.dot(phi, m_phi).real) / ee


def largest_eigenvalue(solver, m1, m2, start, iters=12, **opts):
    """Power-iteration estimate of the largest eigenvalue of M_EOFA(m1, m2)
    (Hermitian positive definite), from the 4D field ``start``; returns
    (estimate, iterations' Rayleigh quotients)."""
    v = start * (1.0 / math.sqrt(solver.dot(start, start).real))
    history = []
    for _ in range(iters):
        w, _ = solver.apply_meofa(v, m1, m2, **opts)
        history.append(solver.dot(v, w).real / solver.dot(v, v).real)
        v = w * (1.0 / math.sqrt(solver.dot(w, w).real))
    return history[-1], history


def measure(solver, eta, m1, m2, approx, pole_tol=None, forecast=0, m_tol=1e-12, **opts):
    """One heatbath and its error: returns (phi, epsilon, stats)."""
    phi, st = solver.heatbath(eta, m1, m2, approx, pole_tol=pole_tol, forecast=forecast, **opts)
    mopts = dict(opts)
    mopts["tol"] = m_tol
    m_phi, _ = solver.apply_meofa(phi, m1, m2, **mopts)
    return phi, heatbath_error(solver, eta, phi, m_phi), st


def tune_pole_tolerances(solver, eta, m1, m2, approx, eps_tol, tol=1e-10, factor=10.0, max_tol=1e-3,
                         forecast=0, **opts):
    """The tuning scheme of Sec. V.B: start every solve at ``tol``; for each
    solve in order, multiply its tolerance by ``factor`` while the heatbath
    error epsilon stays <= eps_tol (and the tolerance <= max_tol).
    Returns (tolerances, epsilon of the tuned heatbath, trials)."""
    n = 2 * len(approx.beta)
    tols = [float(tol)] * n
    _, eps, _ = measure(solver, eta, m1, m2, approx, tols, forecast, tol=tol, **opts)
    if eps > eps_tol:
        raise ValueError(f"untuned heatbath error {eps:.3g} is already above {eps_tol:.3g}")
    trials = 1
    for j in range(n):
        while tols[j] * factor <= max_tol:
            trial = list(tols)
            trial[j] *= factor
            _, e, _ = measure(solver, eta, m1, m2, approx, trial, forecast, tol=tol, **opts)
            trials += 1
            if e > eps_tol:
                break
            tols, eps = trial, e
    return tols, eps, trials
