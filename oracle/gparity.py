"""FP64 oracle of the EOFA operators with G-parity boundary conditions
(test infrastructure; only tests/, __graft_entry__.smoke() and bench.py's
CPU leg may use it; it shares nothing with the CUDA library).

Sec. I: across a G-parity boundary the light doublet maps as
(u, d) -> (d-bar, -u-bar).  With the two-flavour field psi_1 = u,
psi_2 = C d-bar^T (C^T = -C), the boundary conditions in a G-parity
direction mu of extent L read

    psi_1(x + L mu^) = psi_2(x),      psi_2(x + L mu^) = -psi_1(x),

the gauge field obeys U(x + L mu^) = U(x)^*, and the charge-conjugate
flavour's Wilson operator carries the conjugate links: in the bulk
D_W^G = diag(D_W[U], D_W[U^*]).  The Wilson operator below is written from
these rules and the Wilson operator of Eq. (Ddwf) (forward hop
(1 - gamma_mu) U_mu(x) psi(x + mu), backward (1 + gamma_mu) U_mu(x - mu)^dag
psi(x - mu), weight -1/2, t_bc on hops across the t boundary).  Everything
in the fifth dimension is flavour-blind, so the EOFA operators are built
from the C oracle's s-space operators on the two flavours.

Fields: 5D (2, T, Z, Y, X, Ls, 4, 3), 4D (2, T, Z, Y, X, 4, 3).
"""
from __future__ import annotations

import numpy as np

from . import Oracle, gamma


def _axis(mu: int) -> int:
    """Array axis of direction mu (0..3 = x, y, z, t) in (f, T, Z, Y, X, ...)."""
    return 4 - mu


def _take(a: np.ndarray, axis: int, i: int) -> tuple:
    idx = [slice(None)] * a.ndim
    idx[axis] = i
    return tuple(idx)


def wilson(U: np.ndarray, psi: np.ndarray, M5: float, t_bc: int, gmask: int) -> np.ndarray:
    """D_W^G psi for psi of shape (2, T, Z, Y, X, n, 4, 3)."""
    Uf = np.stack([U, U.conj()])  # flavour 2 sees U^*
    out = (4.0 - M5) * psi
    one = np.eye(4)
    for mu in range(4):
        ax = _axis(mu)
        L = psi.shape[ax]
        g = gamma(mu)
        gp = (gmask >> mu) & 1
        sign = float(t_bc) if mu == 3 else 1.0
        # forward neighbour psi(x + mu), fixed up on the last slice
        fwd = np.roll(psi, -1, axis=ax)
        last, first = _take(psi, ax, L - 1), _take(psi, ax, 0)
        if gp:
            fwd[last] = np.stack([psi[1][_take(psi[1], ax - 1, 0)], -psi[0][_take(psi[0], ax - 1, 0)]])
        fwd[last] *= sign
        # backward neighbour psi(x - mu) and its link U(x - mu), fixed up on the first slice
        bwd = np.roll(psi, 1, axis=ax)
        Ul = Uf[:, :, :, :, :, mu]  # (2, T, Z, Y, X, 3, 3)
        Ub = np.roll(Ul, 1, axis=ax)
        if gp:
            # psi_1(x - L) = -psi_2(x), psi_2(x - L) = psi_1(x); U(x - L) = U(x)^*
            bwd[first] = np.stack([-psi[1][_take(psi[1], ax - 1, L - 1)], psi[0][_take(psi[0], ax - 1, L - 1)]])
            Ub[_take(Ub, ax, 0)] = np.stack([Ul[1][_take(Ul[1], ax - 1, L - 1)], Ul[0][_take(Ul[0], ax - 1, L - 1)]])
        bwd[first] *= sign
        t1 = np.einsum("...ij,...sbj->...sbi", Ul, fwd)
        t1 = np.einsum("ab,...sbi->...sai", one - g, t1)
        t2 = np.einsum("...ji,...sbj->...sbi", Ub.conj(), bwd)
        t2 = np.einsum("ab,...sbi->...sai", one + g, t2)
        out = out - 0.5 * (t1 + t2)
    return out


class GOracle:
    """(action, gauge field, G-parity directions); the s-space operators come
    from a C oracle on the flavour-stacked lattice X x Y x Z x 2T (they act
    site by site, so the stacking is only a container for both flavours)."""

    def __init__(self, action, U: np.ndarray, gmask: int):
        self.a = action
        self.U = np.ascontiguousarray(U, dtype=np.complex128)
        self.gmask = int(gmask)
        X, Y, Z, T = action.dims
        self.shape5 = (2, T, Z, Y, X, action.Ls, 4, 3)
        self.shape4 = (2, T, Z, Y, X, 4, 3)
        stacked = np.concatenate([self.U, self.U.conj()])
        self.s = Oracle(action.replace(dims=(X, Y, Z, 2 * T)), stacked)

    def _st(self, x):
        return np.ascontiguousarray(x).reshape(self.s.shape5)

    def _un(self, x):
        return x.reshape(self.shape5)

    def dw(self, x):
        return wilson(self.U, x, self.a.M5, self.a.t_bc, self.gmask)

    def ddwf(self, x, m):
        """Eq. (Ddwf): (b D_W + 1) x + (c D_W - 1) L(m) x."""
        Lx = self._un(self.s.L(self._st(x), m))
        return self.a.b * self.dw(x) + x + self.a.c * self.dw(Lx) - Lx

    def deofa(self, x, m):
        """D_EOFA(m) = D_DWF(m) D~(m)^-1 (Eq. eofa_dop)."""
        return self.ddwf(self._un(self.s.dtilde_inv(self._st(x), m)), m)

    def h(self, x, m):
        return self._un(self.s.g5r5(self._st(self.deofa(x, m))))

    def shift(self, x):
        """beta Delta_pm(m2, m3) P_pm x (site-local)."""
        a = self.a
        D = self.s.delta(a.m2, a.m3, a.pm)
        P = 0.5 * (np.eye(4) + a.pm * gamma(4))
        return a.beta * np.einsum("st,ab,...tbc->...sac", D, P, x)

    def hsys(self, x):
        """(H(m1) + beta Delta_pm(m2, m3) P_pm) x, Eq. (generic_eofa_system)."""
        return self.h(x, self.a.m1) + self.shift(x)

    def solve_h(self, phi, tol=1e-12, maxit=20000):
        """CG on the normal equations of the Hermitian system (plain numpy)."""
        A = self.hsys
        x = np.zeros_like(phi)
        r = A(phi)  # A^dag phi, A Hermitian
        p = r.copy()
        rr = np.vdot(r, r).real
        nb = np.linalg.norm(phi)
        for it in range(maxit):
            # the true residual, every 25 iterations
            if it % 25 == 0 and np.linalg.norm(phi - A(x)) <= tol * nb:
                return x, it
            Ap = A(A(p))
            al = rr / np.vdot(p, Ap).real
            x = x + al * p
            r = r - al * Ap
            rn = np.vdot(r, r).real
            p = r + (rn / rr) * p
            rr = rn
        return x, maxit


def action_g(base, U, gmask, m1, m2, phi, tol=1e-12):
    """S = phi^dag M_EOFA phi with G-parity (Eq. eofa_action), via two solves."""
    from .action import omega_in, omega_out

    def sys(mh, beta, pm):
        return GOracle(base.replace(m1=mh, m2=m1, m3=m2, beta=beta, pm=pm), U, gmask)
    om, op = sys(m1, 0.0, -1), sys(m2, -1.0, +1)
    k = om.s.kcoef(m1, m2)
    w_m, w_p = om.s.omega(-1), om.s.omega(+1)
    xm, _ = om.solve_h(omega_in(w_m, -1, phi), tol)
    xp, _ = op.solve_h(omega_in(w_p, +1, phi), tol)
    m_phi = phi - k * omega_out(w_m, -1, xm) + k * omega_out(w_p, +1, xp)
    return float(np.vdot(phi, m_phi).real), m_phi
