"""FP64 oracle of the EOFA action operator and of its heatbath (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module.  It composes the C oracle's H-form solves
(``Oracle.solve_h``), its App. A closed forms for k and Omega_pm, and numpy
projections; it shares nothing with the CUDA library.

4D fields have shape (T, Z, Y, X, 4, 3), 5D fields (T, Z, Y, X, Ls, 4, 3).
"""
from __future__ import annotations

import numpy as np

from . import Action, Oracle, gamma


def chiral_projector(chi: int) -> np.ndarray:
    """P_pm = (1 pm gamma_5) / 2 in the oracle's gamma basis (Sec. II)."""
    return 0.5 * (np.eye(4) + chi * gamma(4))


def omega_in(om: np.ndarray, chi: int, xi: np.ndarray) -> np.ndarray:
    """Omega_pm P_pm xi: the 5D field om[s] (P_pm xi)(x) (App. A, Omega_pm)."""
    pxi = np.einsum("ab,...bc->...ac", chiral_projector(chi), xi)
    return om[None, None, None, None, :, None, None] * pxi[..., None, :, :]


def omega_out(om: np.ndarray, chi: int, psi: np.ndarray) -> np.ndarray:
    """P_pm Omega_pm^dag psi: the 4D field P_pm sum_s om[s] psi(x, s) (om is real)."""
    v = np.einsum("s,...sbc->...bc", om, psi)
    return np.einsum("ab,...bc->...ac", chiral_projector(chi), v)


def _system(base: Action, U, m_h: float, beta: float, pm: int, m1: float, m2: float) -> Oracle:
    """H(m_h) + beta Delta_pm(m1, m2) P_pm on the lattice of ``base``."""
    return Oracle(base.replace(m1=m_h, m2=m1, m3=m2, beta=beta, pm=pm), U)


def meofa(base: Action, U, m1: float, m2: float, phi: np.ndarray, tol: float = 1e-13):
    """M_EOFA(m1, m2) phi, Eq. (eofa_action):

        phi - k P_- Om_-^dag H(m1)^-1 Om_- P_- phi
            + k P_+ Om_+^dag [H(m2) - Delta_+(m1, m2) P_+]^-1 Om_+ P_+ phi,

    k = k(m1, m2).  Returns (M phi, [stats of the two solves])."""
    o_minus = _system(base, U, m1, 0.0, -1, m1, m2)
    o_plus = _system(base, U, m2, -1.0, +1, m1, m2)
    k = o_minus.kcoef(m1, m2)
    om_m, om_p = o_minus.omega(-1), o_minus.omega(+1)
    x_m, st_m = o_minus.solve_h(omega_in(om_m, -1, phi), tol=tol)
    x_p, st_p = o_plus.solve_h(omega_in(om_p, +1, phi), tol=tol)
    out = phi - k * omega_out(om_m, -1, x_m) + k * omega_out(om_p, +1, x_p)
    return out, [st_m, st_p]


def heatbath(base: Action, U, m1: float, m2: float, alpha0: float, alpha, beta, eta: np.ndarray,
             tol: float = 1e-13):
    """phi = M_EOFA^(-1/2) eta through Eq. (eofa_heatbath): for each pole l,
    gamma_l = 1 / (1 + beta_l) and

        alpha_l gamma_l { eta
          + k gamma_l P_- Om_-^dag [H(m1) - gamma_l Delta_-(m1, m2) P_-]^-1 Om_- P_- eta
          - k gamma_l P_+ Om_+^dag [H(m2) - beta_l gamma_l Delta_+(m1, m2) P_+]^-1 Om_+ P_+ eta },

    plus alpha_0 eta.  Returns (phi, [stats of the 2 N_p solves, minus then
    plus per pole])."""
    o0 = _system(base, U, m1, 0.0, -1, m1, m2)
    k = o0.kcoef(m1, m2)
    om_m, om_p = o0.omega(-1), o0.omega(+1)
    src_m, src_p = omega_in(om_m, -1, eta), omega_in(om_p, +1, eta)
    phi = alpha0 * eta
    stats = []
    for al, bl in zip(alpha, beta):
        g = 1.0 / (1.0 + bl)
        x_m, st_m = _system(base, U, m1, -g, -1, m1, m2).solve_h(src_m, tol=tol)
        x_p, st_p = _system(base, U, m2, -bl * g, +1, m1, m2).solve_h(src_p, tol=tol)
        phi = phi + al * g * (eta + k * g * omega_out(om_m, -1, x_m) - k * g * omega_out(om_p, +1, x_p))
        stats += [st_m, st_p]
    return phi, stats


def heatbath_error(eta: np.ndarray, phi: np.ndarray, m_phi: np.ndarray) -> float:
    """epsilon = |eta^dag eta - phi^dag M_EOFA phi| / eta^dag eta, Eq. (heatbath_rel_err)."""
    ee = np.vdot(eta, eta).real
    return abs(ee - np.vdot(phi, m_phi).real) / ee
