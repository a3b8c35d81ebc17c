"""Pins of the oracle's EOFA pseudofermion force (Sec. III.C, Eq. eofa_force).

The force is the derivative of S = phi^dag M_EOFA phi along
U_mu(x) -> exp(s T^a) U_mu(x); the oracle's closed form (two solves and the
spin-traced bilinear) is checked against central finite differences of S
itself, computed with the oracle's solves on perturbed gauge fields.  A
wrong sign, a swapped projector, a mis-shifted neighbour or a dropped
boundary phase each changes some derivative at O(1).
"""
import numpy as np
import pytest

from paper_1706_05843_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

M1, M2 = 0.04, 1.0


@pytest.fixture(scope="module")
def setup(oracle_mod):
    dims, Ls = (4, 4, 2, 4), 4
    a = oracle_mod.Action(dims=dims, Ls=Ls, M5=1.8, b=1.5, c=0.5, m1=M1, m2=M2, m3=M1, t_bc=-1)
    U = I.gauge_field(dims, 0.5, 3)
    phi = I.heatbath_noise(dims, 21)
    from oracle import force as F
    dS, Fm, imag, st = F.eofa_force(a, U, M1, M2, phi)
    return a, U, phi, dS, Fm, imag, st


def test_generators():
    from oracle.force import generators
    T = generators()
    for a in range(8):
        assert np.allclose(T[a], -T[a].conj().T)
        assert abs(np.trace(T[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) + 0.5 * (a == b)) < 1e-14
    # closed under commutation: [T1, T2] = -T3 (f_123 = 1 with T = i lambda/2)
    assert np.allclose(T[0] @ T[1] - T[1] @ T[0], -T[2])


def test_force_is_real_and_in_the_algebra(setup):
    a, U, phi, dS, Fm, imag, st = setup
    assert all(s.converged for s in st)
    # d^a S is real (H is Hermitian for every gauge field)
    assert imag < 1e-10 * np.abs(dS).max()
    assert np.abs(Fm + np.swapaxes(Fm, -1, -2).conj()).max() < 1e-14
    assert np.abs(np.trace(Fm, axis1=-2, axis2=-1)).max() < 1e-14


@pytest.mark.parametrize("site,mu,gen", [((0, 0, 0, 0), 0, 0), ((1, 2, 1, 3), 3, 7), ((3, 1, 0, 2), 1, 4),
                                         ((2, 3, 1, 1), 2, 2), ((0, 1, 0, 3), 3, 1), ((3, 0, 1, 0), 0, 5)])
def test_force_matches_finite_differences(oracle_mod, setup, site, mu, gen):
    """d/ds S(exp(s T^a) U_mu(x)) at s = 0 by central differences (h = 1e-4,
    truncation O(h^2)); sites given as (x, y, z, t), the t = 3 links cross
    the antiperiodic boundary."""
    from scipy.linalg import expm
    from oracle import force as F
    a, U, phi, dS, Fm, imag, st = setup
    x, y, z, t = site
    T = F.generators()[gen]
    h = 1e-4
    vals = []
    for sgn in (+1, -1):
        Up = U.copy()
        Up[t, z, y, x, mu] = expm(sgn * h * T) @ U[t, z, y, x, mu]
        vals.append(F.action(a, Up, M1, M2, phi))
    fd = (vals[0] - vals[1]) / (2 * h)
    an = dS[t, z, y, x, mu, gen]
    scale = np.abs(dS).max()
    assert abs(fd - an) < 1e-6 * scale + 1e-6 * abs(an), (fd, an, scale)


def test_force_norms(setup):
    """||F_mu(x)|| of Sec. VI from the matrix form equals the generator
    components' Euclidean norm; F_RMS and F_max as printed."""
    from paper_1706_05843_gb300.forces import force_norms, link_norms
    a, U, phi, dS, Fm, imag, st = setup
    ref = np.sqrt(np.sum(dS ** 2, axis=-1))
    assert np.allclose(link_norms(Fm), ref, rtol=1e-13)
    rms, mx = force_norms(Fm)
    assert abs(rms - np.sqrt(np.sum(ref ** 2)) / ref.size) < 1e-13 * rms
    assert mx == pytest.approx(ref.max(), rel=1e-13)
