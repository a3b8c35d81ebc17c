"""FP64 oracle of the EOFA pseudofermion force (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module; it shares nothing with the CUDA library.

Sec. III.C: with chi_1 = H(m1)^-1 Omega_- P_- phi and
chi_2 = [H(m2) - Delta_+(m1, m2) P_+]^-1 Omega_+ P_+ phi, the derivative of
S = phi^dag M_EOFA phi along U_mu(x) -> exp(s T^a) U_mu(x) is

    d^a S = k (g5 R5 chi_1)^dag (d^a D_W) chi_1 - k (g5 R5 chi_2)^dag (d^a D_W) chi_2,

Eq. (eofa_force), because the derivative of D_EOFA (and of H up to g5 R5) is
that of the Wilson operator on every s-slice.  The bilinear a^dag (d^a D_W) b
is written out from the oracle's D_W (forward hop (1 - gamma_mu) U_mu(x),
backward hop (1 + gamma_mu) U_mu(x-mu)^dag, weight -1/2, the time boundary
phase on links that cross t = T-1 -> 0) as in the first line of the paper's
bilinear identity.  T^a = i lambda_a / 2 (Tr T^a T^b = -delta^ab / 2).
"""
from __future__ import annotations

import numpy as np

from . import Oracle, gamma
from .action import _system, omega_in


def generators() -> np.ndarray:
    """T^a = i lambda_a / 2, a = 1..8 (Gell-Mann matrices written out)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return 0.5j * lam


def g5r5(chi: np.ndarray) -> np.ndarray:
    """gamma_5 R_5 chi: reflect s -> Ls-1-s, then gamma_5 on the spin index."""
    return np.einsum("ab,...sbc->...sac", gamma(4), chi[..., ::-1, :, :])


def _shift(f: np.ndarray, mu: int) -> np.ndarray:
    """f(x + mu) with periodic wrap (no boundary phase); mu 0..3 = x, y, z, t
    on the axes (T, Z, Y, X) = 3, 2, 1, 0."""
    return np.roll(f, -1, axis=3 - mu)


def bilinear(a: np.ndarray, b: np.ndarray, U: np.ndarray, t_bc: int) -> np.ndarray:
    """a^dag (d^a_{x,mu} D_W) b for every link and generator: array
    (T, Z, Y, X, 4, 8), complex (real when the total derivative is)."""
    T_ = generators()
    out = np.zeros(U.shape[:4] + (4, 8), dtype=np.complex128)
    for mu in range(4):
        Umu = U[..., mu, :, :]
        g = gamma(mu)
        one = np.eye(4)
        b_f, a_f = _shift(b, mu), _shift(a, mu)
        for A in range(8):
            # forward term a^dag(x) (1 - g) T^a U(x) b(x + mu)
            W = np.einsum("ij,...jk->...ik", T_[A], Umu)
            t1 = np.einsum("...ik,...sbk->...sbi", W, b_f)
            t1 = np.einsum("ab,...sbi->...sai", one - g, t1)
            f1 = np.einsum("...sai,...sai->...", a.conj(), t1)
            # backward term a^dag(x + mu) (1 + g) U(x)^dag T^a b(x)
            W2 = np.einsum("...ji,jk->...ik", Umu.conj(), T_[A])
            t2 = np.einsum("...ik,...sbk->...sbi", W2, b)
            t2 = np.einsum("ab,...sbi->...sai", one + g, t2)
            f2 = np.einsum("...sai,...sai->...", a_f.conj(), t2)
            val = -0.5 * (f1 - f2)
            if mu == 3:
                val[-1] *= t_bc  # links from t = T-1 to t = 0
            out[..., mu, A] = val
    return out


def eofa_force(base, U, m1: float, m2: float, phi: np.ndarray, tol: float = 1e-13):
    """d^a S for every link (x, mu) and generator a, Eq. (eofa_force):
    returns (dS (T, Z, Y, X, 4, 8) real, F (T, Z, Y, X, 4, 3, 3) =
    sum_a T^a d^a S, the largest |imaginary part| of dS, [stats])."""
    o_minus = _system(base, U, m1, 0.0, -1, m1, m2)
    o_plus = _system(base, U, m2, -1.0, +1, m1, m2)
    k = o_minus.kcoef(m1, m2)
    chi1, st1 = o_minus.solve_h(omega_in(o_minus.omega(-1), -1, phi), tol=tol)
    chi2, st2 = o_plus.solve_h(omega_in(o_minus.omega(+1), +1, phi), tol=tol)
    U = np.asarray(U)
    dS = k * bilinear(g5r5(chi1), chi1, U, base.t_bc) - k * bilinear(g5r5(chi2), chi2, U, base.t_bc)
    F = np.einsum("...a,aij->...ij", dS.real, generators())
    return dS.real, F, float(np.abs(dS.imag).max()), [st1, st2]


def action(base, U, m1: float, m2: float, phi: np.ndarray, tol: float = 1e-13) -> float:
    """S = phi^dag M_EOFA(m1, m2) phi, Eq. (eofa_action)."""
    from .action import meofa
    m_phi, _ = meofa(base, U, m1, m2, phi, tol=tol)
    return float(np.vdot(phi, m_phi).real)
