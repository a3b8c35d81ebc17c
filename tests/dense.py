"""Dense assembly helpers for the oracle pins (numpy, tiny lattices only)."""
import numpy as np


def assemble(op, n, shape):
    """Dense matrix of a linear map given as op(field) -> field."""
    M = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = op(e.reshape(shape)).reshape(-1)
    return M


def site_smatrix(Ap, Am, V, Ls, g5):
    """Dense 5D matrix of sum_x delta_xx' (Ap P+ + Am P-) (x) 1_colour."""
    Pp = 0.5 * (np.eye(4) + g5)
    Pm = 0.5 * (np.eye(4) - g5)
    blk = np.kron(Ap, np.kron(Pp, np.eye(3))) + np.kron(Am, np.kron(Pm, np.eye(3)))
    return np.kron(np.eye(V), blk)


def omega_matrix(om, V, Ls):
    """Dense 5D <- 4D map (Omega xi)(x, s) = om_s xi(x)."""
    blk = np.kron(om.reshape(Ls, 1), np.eye(12))
    return np.kron(np.eye(V), blk)


def chiral_proj5(chi, V, Ls, g5):
    P = 0.5 * (np.eye(4) + chi * g5)
    return np.kron(np.eye(V * Ls), np.kron(P, np.eye(3)))


def chiral_proj4(chi, V, g5):
    P = 0.5 * (np.eye(4) + chi * g5)
    return np.kron(np.eye(V), np.kron(P, np.eye(3)))
