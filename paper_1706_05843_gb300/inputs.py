"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds no arithmetic of the EOFA method itself: it only draws
gauge fields, gauge transformations and right-hand sides from a seeded
numpy ``PCG64`` stream.  Both sides of every parity check take their inputs
from here, so neither has to trust the other for its data.

Conventions (shared with ``include/eofa.h``):

* lattice extents ``dims = (X, Y, Z, T)``; 4D sites are stored
  lexicographically as ``[t][z][y][x]`` (x fastest);
* gauge field ``U[t][z][y][x][mu][row][col]`` complex128, ``mu = 0..3`` is
  x, y, z, t;
* 5D fermion field ``psi[t][z][y][x][s][spin][colour]`` complex128.

Gauge links follow the recipe used for the paper's stand-in ensembles: for
every link draw eight N(0,1) numbers ``h_a`` (in the order t, z, y, x, mu),
form the traceless Hermitian ``H = sum_a h_a lambda_a / 2`` from the
Gell-Mann matrices, exponentiate ``U = exp(i eps H)`` through an eigen-
decomposition and re-unitarise: Gram-Schmidt on rows one and two, row three
set to ``conj(r1 x r2)``.  The last step makes the field exactly (to
rounding) special unitary, so a two-row compressed copy reconstructs it.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann",
    "random_su3",
    "gauge_field",
    "unit_gauge",
    "gauge_transform",
    "gaussian_fermion",
    "gaussian_fermion_batch",
]


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3) complex128."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _reunitarise(u: np.ndarray) -> np.ndarray:
    """Gram-Schmidt rows 1-2, row 3 = conj(r1 x r2).  u: (..., 3, 3)."""
    r1 = u[..., 0, :]
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = u[..., 1, :]
    r2 = r2 - np.sum(np.conj(r1) * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    r3 = np.conj(np.cross(r1, r2))
    return np.stack([r1, r2, r3], axis=-2)


def _su3_from_draws(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i eps sum_a h_a lambda_a/2), re-unitarised.  h: (..., 8) float64."""
    lam = gell_mann()
    shape = h.shape[:-1]
    hflat = h.reshape(-1, 8)
    out = np.empty((hflat.shape[0], 3, 3), dtype=np.complex128)
    chunk = 1 << 18
    for lo in range(0, hflat.shape[0], chunk):
        hh = hflat[lo:lo + chunk]
        H = np.einsum("na,aij->nij", hh, lam) * 0.5
        w, V = np.linalg.eigh(H)
        ph = np.exp(1j * eps * w)
        U = np.einsum("nij,nj,nkj->nik", V, ph, np.conj(V))
        out[lo:lo + chunk] = _reunitarise(U)
    return out.reshape(shape + (3, 3))


def random_su3(n: int, eps: float, seed: int) -> np.ndarray:
    """n random SU(3) matrices exp(i eps H), H Gaussian in the algebra."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _su3_from_draws(rng.standard_normal((n, 8)), eps)


def gauge_field(dims, eps: float, seed: int) -> np.ndarray:
    """Random SU(3) gauge field U[t][z][y][x][mu][3][3] (complex128).

    dims = (X, Y, Z, T).  Draws are taken t-slice by t-slice, which is the
    same stream as one C-ordered draw of shape (T, Z, Y, X, 4, 8).
    """
    X, Y, Z, T = (int(d) for d in dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    U = np.empty((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    for t in range(T):
        h = rng.standard_normal((Z, Y, X, 4, 8))
        U[t] = _su3_from_draws(h, eps)
    return U


def unit_gauge(dims) -> np.ndarray:
    """Free field: every link the 3x3 identity."""
    X, Y, Z, T = (int(d) for d in dims)
    U = np.zeros((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def gauge_transform(dims, seed: int, eps: float = 1.0) -> np.ndarray:
    """Random site-local SU(3) matrices g[t][z][y][x][3][3]."""
    X, Y, Z, T = (int(d) for d in dims)
    return random_su3(X * Y * Z * T, eps, seed).reshape(T, Z, Y, X, 3, 3)


def gaussian_fermion(dims, Ls: int, seed: int) -> np.ndarray:
    """Complex Gaussian 5D field, real and imaginary parts N(0, 1).

    Shape (T, Z, Y, X, Ls, 4, 3) complex128.
    """
    X, Y, Z, T = (int(d) for d in dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((T, Z, Y, X, Ls, 4, 3, 2))
    return d[..., 0] + 1j * d[..., 1]


def heatbath_noise(dims, seed: int) -> np.ndarray:
    """The heatbath's 4D Gaussian eta: real and imaginary parts N(0, 1/2), so
    that P(eta) ~ exp(-eta^dag eta) (Sec. III.B).  Shape (T, Z, Y, X, 4, 3)."""
    X, Y, Z, T = (int(d) for d in dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((T, Z, Y, X, 4, 3, 2)) * np.sqrt(0.5)
    return d[..., 0] + 1j * d[..., 1]


def gaussian_fermion_batch(dims, Ls: int, seeds) -> np.ndarray:
    """Stack of ``gaussian_fermion`` fields, one per seed."""
    return np.stack([gaussian_fermion(dims, Ls, s) for s in seeds])
