"""Pins of the oracle's G-parity operators (Sec. I boundary conditions).

(a) G-parity in t alone is the single-flavour operator on a lattice of
    doubled time extent with links [U; U^*] and an antiperiodic seam: the
    C oracle's own operator checks the numpy G-parity Wilson operator and
    the composition of the EOFA system.
(b) Free field: a plane wave with psi_2 = c psi_1, c = +-i, and momenta
    (2 pi n + theta)/L, e^{i theta L} = c in G-parity directions, solves the
    boundary conditions and is an eigenvector with the momentum-space
    Wilson symbol, in any set of G-parity directions.
(c) Gauge covariance under transformations obeying the G-parity boundary
    condition Omega(x + L) = Omega(x)^* (flavour 2 transforms with Omega^*).
(d) H + beta Delta P stays Hermitian.
"""
import numpy as np
import pytest

from paper_1706_05843_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

ACT = dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.3, beta=-0.7, pm=-1)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def gfield(dims, Ls, seed):
    X, Y, Z, T = dims
    a = I.gaussian_fermion(dims, Ls, seed)
    b = I.gaussian_fermion(dims, Ls, seed + 1)
    return np.stack([a, b])


def test_t_gparity_is_doubled_time_lattice(oracle_mod):
    from oracle.gparity import GOracle
    O = oracle_mod
    dims, Ls = (4, 2, 2, 4), 4
    U = I.gauge_field(dims, 0.5, 5)
    g = GOracle(O.Action(dims=dims, Ls=Ls, t_bc=1, **ACT), U, gmask=8)
    X, Y, Z, T = dims
    ref = O.Oracle(O.Action(dims=(X, Y, Z, 2 * T), Ls=Ls, t_bc=-1, **ACT), np.concatenate([U, U.conj()]))
    psi = gfield(dims, Ls, 7)
    flat = psi.reshape(ref.shape5)
    assert rel(g.dw(psi).reshape(ref.shape5), ref.dw5(flat)) < 1e-14
    assert rel(g.hsys(psi).reshape(ref.shape5), ref.hsys(flat)) < 1e-14


@pytest.mark.parametrize("gmask,t_bc", [(1, -1), (3, -1), (6, 1), (9, -1), (15, 1)])
def test_free_field_twisted_plane_wave(oracle_mod, gmask, t_bc):
    from oracle.gparity import wilson
    O = oracle_mod
    dims = (4, 6, 4, 8)
    X, Y, Z, T = dims
    U = I.unit_gauge(dims)
    M5 = 1.8
    c = 1j
    rng = np.random.default_rng(3)
    chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    p = []
    for mu, L in enumerate(dims):
        theta = np.pi / 2 if (gmask >> mu) & 1 else 0.0  # e^{i theta} = c
        if mu == 3 and t_bc == -1:
            theta += np.pi
        p.append((2 * np.pi * (mu + 1) + theta) / L)
    t, z, y, x = np.meshgrid(range(T), range(Z), range(Y), range(X), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    psi1 = ph[..., None, None, None] * chi[None, None, None, None, None]
    psi = np.stack([psi1, c * psi1])  # (2, T, Z, Y, X, 1, 4, 3)
    out = wilson(U, psi, M5, t_bc, gmask)
    sym = (4 - M5) * np.eye(4, dtype=complex)
    for mu in range(4):
        sym += -np.cos(p[mu]) * np.eye(4) + 1j * np.sin(p[mu]) * O.gamma(mu)
    ref = np.einsum("ab,...sbc->...sac", sym, psi)
    assert rel(out, ref) < 1e-13


def test_gauge_covariance(oracle_mod):
    """D^G[U^Omega] (Omega psi) = Omega D^G[U] psi with Omega on flavour 1,
    Omega^* on flavour 2, and links across a G-parity boundary transformed
    with the conjugate Omega of the wrapped site."""
    from oracle.gparity import wilson
    dims = (4, 4, 2, 4)
    X, Y, Z, T = dims
    gmask, t_bc = 5, -1
    U = I.gauge_field(dims, 0.5, 9)
    Om = I.gauge_transform(dims, 11)
    Uo = np.empty_like(U)
    for mu in range(4):
        ax = 3 - mu
        L = dims[mu]
        On = np.roll(Om, -1, axis=ax)  # Omega(x + mu) on the wrapped lattice
        if (gmask >> mu) & 1:
            idx = [slice(None)] * 4
            idx[ax] = L - 1
            On[tuple(idx)] = On[tuple(idx)].conj()  # Omega(x + L) = Omega(x)^*
        Uo[..., mu, :, :] = Om @ U[..., mu, :, :] @ np.swapaxes(On.conj(), -1, -2)
    psi = gfield(dims, 2, 13)
    opsi = np.stack([np.einsum("...ij,...sbj->...sbi", Om, psi[0]),
                     np.einsum("...ij,...sbj->...sbi", Om.conj(), psi[1])])
    lhs = wilson(Uo, opsi, 1.8, t_bc, gmask)
    d = wilson(U, psi, 1.8, t_bc, gmask)
    rhs = np.stack([np.einsum("...ij,...sbj->...sbi", Om, d[0]),
                    np.einsum("...ij,...sbj->...sbi", Om.conj(), d[1])])
    assert rel(lhs, rhs) < 1e-13
    # a transformation that ignores the boundary condition breaks it
    Ubad = np.empty_like(U)
    for mu in range(4):
        On = np.roll(Om, -1, axis=3 - mu)
        Ubad[..., mu, :, :] = Om @ U[..., mu, :, :] @ np.swapaxes(On.conj(), -1, -2)
    assert rel(wilson(Ubad, opsi, 1.8, t_bc, gmask), rhs) > 1e-2


@pytest.mark.parametrize("gmask", [1, 10, 15])
def test_system_hermitian(oracle_mod, gmask):
    from oracle.gparity import GOracle
    O = oracle_mod
    dims, Ls = (4, 2, 4, 2), 4
    g = GOracle(O.Action(dims=dims, Ls=Ls, t_bc=-1, **ACT), I.gauge_field(dims, 0.5, 2), gmask)
    x, y = gfield(dims, Ls, 3), gfield(dims, Ls, 5)
    assert abs(np.vdot(y, g.hsys(x)) - np.vdot(g.hsys(y), x)) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)
    sol, it = g.solve_h(y, tol=1e-11)
    assert rel(g.hsys(sol), y) <= 1e-11


def test_stacked_force_fold(oracle_mod):
    """With G-parity in t the action depends on U through both halves of the
    stacked links [U; U^*]; the force on U is the stacked force on flavour
    1's copy plus the conjugate of that on flavour 2's copy (conj(T^a) is
    -T^a or T^a).  Checked against central differences of the stacked
    action under U -> exp(s T^a) U applied to both copies."""
    from scipy.linalg import expm
    from oracle import force as F
    O = oracle_mod
    dims, Ls = (4, 2, 2, 4), 4
    X, Y, Z, T = dims
    U = I.gauge_field(dims, 0.5, 6)
    sa = O.Action(dims=(X, Y, Z, 2 * T), Ls=Ls, M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, t_bc=-1)
    phi = np.stack([I.heatbath_noise(dims, 41), I.heatbath_noise(dims, 42)]).reshape((2 * T, Z, Y, X, 4, 3))
    _, Fs, _, _ = F.eofa_force(sa, np.concatenate([U, U.conj()]), 0.04, 1.0, phi)
    Fp = Fs[:T] + Fs[T:].conj()
    Tg = F.generators()
    h = 1e-4
    for (x, y, z, t), mu, gen in [((3, 1, 0, 3), 3, 2), ((1, 0, 1, 2), 0, 4)]:
        vals = []
        for sg in (+1, -1):
            Up = U.copy()
            Up[t, z, y, x, mu] = expm(sg * h * Tg[gen]) @ U[t, z, y, x, mu]
            vals.append(F.action(sa, np.concatenate([Up, Up.conj()]), 0.04, 1.0, phi))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = -2.0 * np.trace(Tg[gen] @ Fp[t, z, y, x, mu]).real
        assert abs(fd - an) < 1e-6 * (np.abs(Fp).max() + abs(an)), (fd, an)
