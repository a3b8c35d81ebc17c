"""Force norms of Sec. VI (Eqs. L2_force, Linf_force): the definition for
host arrays.  The library computes the same on the device from a force it
produced (``Solver.force_norms``, eofa_force_norms), without copying the
force to the host.

For F_mu(x) = sum_a T^a F^a_mu(x) with Tr T^a T^b = -delta^ab / 2, the norm
||F_mu(x)|| = [sum_a (F^a_mu(x))^2]^(1/2) equals sqrt(2) times the Frobenius
norm of the 3x3 matrix.  F_RMS = [sum_{x,mu} ||F_mu(x)||^2]^(1/2) / (4V) as
printed, and F_max = max_{x,mu} ||F_mu(x)||.
"""
from __future__ import annotations

import numpy as np


def link_norms(F) -> np.ndarray:
    """||F_mu(x)|| for every link of a (T, Z, Y, X, 4, 3, 3) force array
    (numpy or a torch tensor)."""
    if hasattr(F, "detach"):
        F = F.detach().cpu().numpy()
    return np.sqrt(2.0 * np.sum(np.abs(F) ** 2, axis=(-2, -1)))


def force_norms(F):
    """(F_RMS, F_max) of Eqs. (L2_force), (Linf_force)."""
    n = link_norms(F)
    return float(np.sqrt(np.sum(n ** 2)) / n.size), float(n.max())
