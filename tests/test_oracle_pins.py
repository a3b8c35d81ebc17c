"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula: each compares the oracle
with an independent statement -- a closed form from a different passage, a
factorisation identity, a symmetry, a determinant identity, or a brute-force
dense computation -- so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import numpy as np
import pytest

from paper_1706_05843_gb300 import inputs as I
from tests.dense import (assemble, chiral_proj4, chiral_proj5, omega_matrix,
                         site_smatrix)

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

MOBIUS = dict(b=1.5, c=0.5)          # the Moebius point of the benchmark configs
MOBIUS2 = dict(b=1.4, c=0.8)         # b - c != 1: the closed forms are general
SHAMIR = dict(b=1.0, c=0.0)          # c = d = 1/2 in the paper's notation


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make(O, dims=(4, 4, 4, 4), Ls=8, eps=0.3, seed=1, **kw):
    a = O.Action(dims=dims, Ls=Ls, **kw)
    return O.Oracle(a, I.gauge_field(dims, eps, seed))


# --------------------------------------------------------------------------
# gamma basis (reading 9: chiral basis)
# --------------------------------------------------------------------------
def test_gamma_algebra(oracle_mod):
    O = oracle_mod
    g = [O.gamma(m) for m in range(5)]
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            anti = g[m] @ g[n] + g[n] @ g[m]
            assert np.allclose(anti, 2 * np.eye(4) * (m == n))
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]))
    for m in range(4):
        assert np.allclose(g[4] @ g[m] + g[m] @ g[4], 0)


# --------------------------------------------------------------------------
# D_W against the free-field momentum-space closed form (Eq. Ddwf)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (3, 1, 1, 2)])
@pytest.mark.parametrize("dag", [False, True])
def test_wilson_free_field_plane_wave(oracle_mod, n, dag):
    O = oracle_mod
    dims = (4, 4, 6, 4)
    a = O.Action(dims=dims, Ls=1, M5=1.8, t_bc=-1)
    o = O.Oracle(a, I.unit_gauge(dims))
    X, Y, Z, T = dims
    p = np.array([2 * np.pi * n[0] / X, 2 * np.pi * n[1] / Y,
                  2 * np.pi * n[2] / Z, (2 * n[3] + 1) * np.pi / T])
    rng = np.random.default_rng(3)
    eta = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y),
                             np.arange(X), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    psi = phase[..., None, None] * eta
    g = [O.gamma(m) for m in range(4)]
    sgn = -1.0 if dag else 1.0      # D_W^dag(p) = D_W(p)^dag flips the i sin term
    Dp = (4 - 1.8 - np.cos(p).sum()) * np.eye(4) + sgn * 1j * sum(
        g[m] * np.sin(p[m]) for m in range(4))
    expect = phase[..., None, None] * (Dp @ eta)
    got = o.dw4(psi, dag=dag)
    assert rel(got, expect) < 1e-13


def test_ddwf_free_field_momentum_space(oracle_mod):
    """5D check at unit links: D_DWF(p) = (b5 D_W(p)+1) + (c5 D_W(p)-1) L."""
    O = oracle_mod
    dims, Ls = (4, 4, 4, 4), 6
    a = O.Action(dims=dims, Ls=Ls, **MOBIUS)
    o = O.Oracle(a, I.unit_gauge(dims))
    p = np.array([np.pi / 2, 0, np.pi, 3 * np.pi / 4])
    t, z, y, x = np.meshgrid(*(np.arange(4),) * 4, indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    rng = np.random.default_rng(5)
    eta = rng.standard_normal((Ls, 4, 3)) + 1j * rng.standard_normal((Ls, 4, 3))
    psi = phase[..., None, None, None] * eta
    g = [O.gamma(m) for m in range(5)]
    Dw = (4 - 1.8 - np.cos(p).sum()) * np.eye(4) + 1j * sum(g[m] * np.sin(p[m]) for m in range(4))
    m = 0.04
    Lp, Lm = o.L_matrices(m)
    Pp, Pm = 0.5 * (np.eye(4) + g[4]), 0.5 * (np.eye(4) - g[4])
    L5 = np.kron(Lp, Pp) + np.kron(Lm, Pm)
    D5 = np.kron(np.eye(Ls), 1.5 * Dw + np.eye(4)) + np.kron(np.eye(Ls), 0.5 * Dw - np.eye(4)) @ L5
    expect = phase[..., None, None, None] * np.einsum("ab,bc->ac", D5, eta.reshape(Ls * 4, 3)).reshape(Ls, 4, 3)
    assert rel(o.ddwf(psi, m), expect) < 1e-13


# --------------------------------------------------------------------------
# gauge covariance: pins U vs U^dag and x+mu vs x-mu
# --------------------------------------------------------------------------
@pytest.mark.parametrize("pm", [1, -1])
def test_gauge_covariance(oracle_mod, pm):
    O = oracle_mod
    dims, Ls = (4, 4, 2, 4), 4
    a = O.Action(dims=dims, Ls=Ls, pm=pm, beta=0.7, **MOBIUS)
    U = I.gauge_field(dims, 0.7, 11)
    g = I.gauge_transform(dims, 12)
    X, Y, Z, T = dims
    Ug = np.empty_like(U)
    for mu, ax in enumerate([3, 2, 1, 0]):
        gs = np.roll(g, -1, axis=ax)        # g(x + mu)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gs, -1, -2))
    psi = I.gaussian_fermion(dims, Ls, 13)
    psig = np.einsum("tzyxab,tzyxsib->tzyxsia", g, psi)
    o, og = O.Oracle(a, U), O.Oracle(a, Ug)
    for name in ("k", "asys"):
        for dag in (False, True):
            lhs = getattr(og, name)(psig, dag=dag)
            rhs = np.einsum("tzyxab,tzyxsib->tzyxsia", g, getattr(o, name)(psi, dag=dag))
            assert rel(lhs, rhs) < 1e-13, (name, dag)


# --------------------------------------------------------------------------
# Eq. (eofa_dop): D_DWF = D_EOFA . D~  (App. A closed forms of M+-)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("coef", [MOBIUS, MOBIUS2, SHAMIR])
@pytest.mark.parametrize("m", [0.04, 0.3, 1.0])
def test_factorisation(oracle_mod, coef, m):
    o = make(oracle_mod, Ls=8, **coef)
    psi = I.gaussian_fermion(o.a.dims, o.a.Ls, 21)
    for dag in (False, True):
        if not dag:
            lhs, rhs = o.ddwf(psi, m), o.deofa(o.dtilde(psi, m), m)
        else:   # (D_EOFA D~)^dag = D~^dag D_EOFA^dag
            lhs, rhs = o.ddwf(psi, m, dag=True), o.dtilde(o.deofa(psi, m, dag=True), m, dag=True)
        assert rel(lhs, rhs) < 1e-13


@pytest.mark.parametrize("coef", [MOBIUS, MOBIUS2, SHAMIR])
def test_mpm_closed_form_vs_numeric(oracle_mod, coef):
    """M+- = (1 - L+-)(b5 + c5 L+-)^-1, the matrices implied by Eq. (eofa_dop)."""
    o = make(oracle_mod, dims=(2, 2, 2, 2), Ls=10, **coef)
    b5, c5 = coef["b"], coef["c"]
    for m in (0.04, 0.5, 1.0):
        Lp, Lm = o.L_matrices(m)
        Mp, Mm = o.mpm(m)
        E = np.eye(10)
        assert np.allclose(Mp, (E - Lp) @ np.linalg.inv(b5 * E + c5 * Lp), atol=1e-14)
        assert np.allclose(Mm, (E - Lm) @ np.linalg.inv(b5 * E + c5 * Lm), atol=1e-14)


def test_shamir_limit(oracle_mod):
    """c = d = 1/2: App. A Moebius forms reduce to the Shamir ones.

    The Shamir M+- of App. A carry the m corner at (Ls-1, 0) for M+ and
    (0, Ls-1) for M-; the corner that agrees with L+- of Eq. (Ddwf), with
    Eq. (Ddwf_ooee) and with the Moebius forms at c = d is the transpose:
    (0, Ls-1) for M+ and (Ls-1, 0) for M-.  This test pins that reading.
    """
    Ls, m = 8, 0.1
    o = make(oracle_mod, dims=(2, 2, 2, 2), Ls=Ls, **SHAMIR)
    Mp, Mm = o.mpm(m)
    E = np.eye(Ls)
    sub = np.eye(Ls, k=-1)          # delta_{s, s'+1}
    Mp_expect = E - sub
    Mp_expect[0, Ls - 1] = m
    Mm_expect = E - sub.T
    Mm_expect[Ls - 1, 0] = m
    assert np.allclose(Mp, Mp_expect, atol=1e-15)
    assert np.allclose(Mm, Mm_expect, atol=1e-15)
    m1, m2 = 0.04, 0.6
    assert abs(o.kcoef(m1, m2) - (m2 - m1)) < 1e-15
    Dp = np.zeros((Ls, Ls)); Dp[Ls - 1, Ls - 1] = m2 - m1
    Dm = np.zeros((Ls, Ls)); Dm[0, 0] = m2 - m1
    assert np.allclose(o.delta(m1, m2, 1), Dp, atol=1e-15)
    assert np.allclose(o.delta(m1, m2, -1), Dm, atol=1e-15)
    assert np.allclose(o.omega(1), np.eye(Ls)[Ls - 1])
    assert np.allclose(o.omega(-1), np.eye(Ls)[0])
    psi = I.gaussian_fermion(o.a.dims, Ls, 3)
    assert rel(o.dtilde(psi, m), psi) < 1e-15


def test_shamir_shift_operators(oracle_mod):
    """App. B (Shamir): beta g5 R5 Delta_+-(m2,m3) P+- is a single corner
    entry +-beta (m3 - m2) P+- at (s, s') = (0, Ls-1) resp. (Ls-1, 0)."""
    Ls, dims = 6, (2, 2, 2, 2)
    for pm in (1, -1):
        a = oracle_mod.Action(dims=dims, Ls=Ls, beta=0.7, pm=pm, m1=0.04, m2=0.3,
                              m3=0.05, **SHAMIR)
        U = I.gauge_field(dims, 0.3, 1)
        o = oracle_mod.Oracle(a, U)
        o0 = oracle_mod.Oracle(a.replace(beta=0.0), U)
        psi = I.gaussian_fermion(dims, Ls, 4)
        shift = o.asys(psi) - o0.asys(psi)
        g5 = oracle_mod.gamma(4)
        P = 0.5 * (np.eye(4) + pm * g5)
        expect = np.zeros_like(psi)
        src, dst = (Ls - 1, 0) if pm > 0 else (0, Ls - 1)
        expect[..., dst, :, :] = pm * 0.7 * (0.05 - 0.3) * np.einsum("ab,...bc->...ac", P, psi[..., src, :, :])
        assert rel(shift, expect) < 1e-14


# --------------------------------------------------------------------------
# other App. A identities
# --------------------------------------------------------------------------
@pytest.mark.parametrize("coef", [MOBIUS, MOBIUS2, SHAMIR])
def test_delta_equals_k_omega_omega(oracle_mod, coef):
    o = make(oracle_mod, dims=(2, 2, 2, 2), Ls=12, **coef)
    for mA, mB in [(0.04, 1.0), (0.0362, 0.5), (0.3, 0.1)]:
        k = o.kcoef(mA, mB)
        for pm in (1, -1):
            om = o.omega(pm)
            assert np.allclose(o.delta(mA, mB, pm), k * np.outer(om, om), rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("coef", [MOBIUS, MOBIUS2])
def test_dtilde_inverse_closed_form(oracle_mod, coef):
    o = make(oracle_mod, Ls=8, **coef)
    psi = I.gaussian_fermion(o.a.dims, 8, 8)
    for m in (0.04, 1.0):
        assert rel(o.dtilde_inv(o.dtilde(psi, m), m), psi) < 1e-14
        assert rel(o.dtilde(o.dtilde_inv(psi, m), m), psi) < 1e-14


@pytest.mark.parametrize("coef", [MOBIUS, MOBIUS2, SHAMIR])
def test_dtilde_determinant(oracle_mod, coef):
    """Eq. (dtilde_det): det D~ = ((c+d)^Ls + m (c-d)^Ls)^(12 V)."""
    dims, Ls, m = (2, 2, 2, 2), 4, 0.3
    o = make(oracle_mod, dims=dims, Ls=Ls, **coef)
    V = 16
    n = V * Ls * 12
    D = assemble(lambda v: o.dtilde(v, m), n, o.shape5)
    sign, logdet = np.linalg.slogdet(D)
    N = coef["b"] ** Ls + m * coef["c"] ** Ls
    assert abs(logdet - 12 * V * np.log(abs(N))) < 1e-10
    assert abs(sign - np.sign(N) ** (12 * V)) < 1e-10


# --------------------------------------------------------------------------
# hermiticity (Sec. II) and dense determinant identities
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def dense24(oracle_mod):
    """Dense matrices on a 2^4 x Ls=4 lattice with random SU(3) links."""
    O = oracle_mod
    dims, Ls = (2, 2, 2, 2), 4
    m1, m2 = 0.04, 1.0
    a = O.Action(dims=dims, Ls=Ls, m1=m1, m2=m2, m3=m1, **MOBIUS)
    o = O.Oracle(a, I.gauge_field(dims, 0.5, 1))
    n = 16 * Ls * 12
    d = dict(o=o, n=n, V=16, Ls=Ls, m1=m1, m2=m2)
    d["H1"] = assemble(lambda v: o.h(v, m1), n, o.shape5)
    d["H2"] = assemble(lambda v: o.h(v, m2), n, o.shape5)
    d["E1"] = assemble(lambda v: o.deofa(v, m1), n, o.shape5)
    d["E2"] = assemble(lambda v: o.deofa(v, m2), n, o.shape5)
    d["W1"] = assemble(lambda v: o.ddwf(v, m1), n, o.shape5)
    d["W2"] = assemble(lambda v: o.ddwf(v, m2), n, o.shape5)
    return d


def test_h_hermitian(dense24):
    for key in ("H1", "H2"):
        H = dense24[key]
        assert np.abs(H - H.conj().T).max() < 1e-14


def test_g5r5_ddwf_not_hermitian(dense24, oracle_mod):
    """Sanity: for Moebius (alpha != 1) g5 R5 D_DWF is not Hermitian (Sec. II)."""
    o = dense24["o"]
    G = assemble(o.g5r5, dense24["n"], o.shape5)
    A = G @ dense24["W1"]
    assert np.abs(A - A.conj().T).max() > 1e-2


def test_hsys_hermitian(oracle_mod, dense24):
    o = dense24["o"]
    for pm in (1, -1):
        for beta in (-1.0, 0.7):
            oo = oracle_mod.Oracle(o.a.replace(pm=pm, beta=beta, m2=1.0, m3=0.3), o.U)
            A = assemble(oo.hsys, dense24["n"], o.shape5)
            assert np.abs(A - A.conj().T).max() < 1e-14


def test_det_ratio_dwf_vs_eofa(dense24):
    """Eq. (eofa_action_test)."""
    d = dense24
    ld = lambda M: np.linalg.slogdet(M)
    sW1, lW1 = ld(d["W1"]); sW2, lW2 = ld(d["W2"])
    sE1, lE1 = ld(d["E1"]); sE2, lE2 = ld(d["E2"])
    N1 = 1.5 ** 4 + d["m1"] * 0.5 ** 4
    N2 = 1.5 ** 4 + d["m2"] * 0.5 ** 4
    lhs = lW1 - lW2
    rhs = 12 * d["V"] * np.log(N1 / N2) + lE1 - lE2
    assert abs(lhs - rhs) < 1e-9
    assert abs(sW1 / sW2 - sE1 / sE2) < 1e-9


def dense_meofa(O, d):
    """Dense M_EOFA(m1, m2) of Eq. (eofa_action) from dense H(m1), H(m2)."""
    o, V, Ls = d["o"], d["V"], d["Ls"]
    m1, m2 = d["m1"], d["m2"]
    g5 = O.gamma(4)
    k = o.kcoef(m1, m2)
    Omp = omega_matrix(o.omega(1), V, Ls)
    Omm = omega_matrix(o.omega(-1), V, Ls)
    Pp4, Pm4 = chiral_proj4(1, V, g5), chiral_proj4(-1, V, g5)
    Dp = site_smatrix(o.delta(m1, m2, 1), np.zeros((Ls, Ls)), V, Ls, g5)
    Hm = np.linalg.inv(d["H1"])
    Hp = np.linalg.inv(d["H2"] - Dp)
    return (np.eye(12 * V) - k * Pm4 @ Omm.T @ Hm @ Omm @ Pm4
            + k * Pp4 @ Omp.T @ Hp @ Omp @ Pp4)


def test_det_ratio_equals_m_eofa(oracle_mod, dense24):
    """Eqs. (EOFA_factorization), (eofa_action), (eofa_pi):
    det D_EOFA(m1) / det D_EOFA(m2) = 1 / det M_EOFA, and M_EOFA is
    Hermitian positive definite (its spectrum is not asserted to start at 1:
    the paper's '1.0' is rounded and random fields give ~0.99)."""
    d = dense24
    M = dense_meofa(oracle_mod, d)
    assert np.abs(M - M.conj().T).max() < 1e-12
    ev = np.linalg.eigvalsh(0.5 * (M + M.conj().T))
    assert ev.min() > 0.5
    _, lE1 = np.linalg.slogdet(d["E1"])
    _, lE2 = np.linalg.slogdet(d["E2"])
    sM, lM = np.linalg.slogdet(M)
    assert abs((lE1 - lE2) + lM) < 1e-9
    assert abs(sM - 1) < 1e-9


# --------------------------------------------------------------------------
# M_EOFA application and heatbath (Eqs. eofa_action, eofa_heatbath)
# --------------------------------------------------------------------------
def test_meofa_apply_matches_dense(oracle_mod, dense24):
    """The oracle's M_EOFA phi (two H-form solves and the Omega projections)
    equals the dense M_EOFA built from inverted dense H matrices."""
    from oracle import action as A
    d = dense24
    o = d["o"]
    M = dense_meofa(oracle_mod, d)
    eta = I.heatbath_noise(o.a.dims, 5)
    out, st = A.meofa(o.a, o.U, d["m1"], d["m2"], eta)
    assert all(s.converged for s in st)
    assert rel(out.reshape(-1), M @ eta.reshape(-1)) < 1e-10


@pytest.mark.parametrize("coef", [MOBIUS2, SHAMIR], ids=["b1.4_c0.8", "shamir"])
def test_m_eofa_other_kernels(oracle_mod, coef):
    """For b - c != 1 and for Shamir (c = d = 1/2) the App. A closed forms of
    k and Omega_pm still give det D_EOFA(m1) / det D_EOFA(m2) = 1 / det M_EOFA
    with M_EOFA Hermitian positive definite, and the oracle's two-solve
    M_EOFA phi equals the dense one."""
    from oracle import action as A
    O = oracle_mod
    dims, Ls, m1, m2 = (2, 2, 2, 2), 4, 0.04, 1.0
    o = O.Oracle(O.Action(dims=dims, Ls=Ls, m1=m1, m2=m2, m3=m1, **coef), I.gauge_field(dims, 0.5, 2))
    n = 16 * Ls * 12
    d = dict(o=o, n=n, V=16, Ls=Ls, m1=m1, m2=m2)
    d["H1"] = assemble(lambda v: o.h(v, m1), n, o.shape5)
    d["H2"] = assemble(lambda v: o.h(v, m2), n, o.shape5)
    M = dense_meofa(O, d)
    assert np.abs(M - M.conj().T).max() < 1e-12
    assert np.linalg.eigvalsh(0.5 * (M + M.conj().T)).min() > 0.5
    _, lE1 = np.linalg.slogdet(assemble(lambda v: o.deofa(v, m1), n, o.shape5))
    _, lE2 = np.linalg.slogdet(assemble(lambda v: o.deofa(v, m2), n, o.shape5))
    sM, lM = np.linalg.slogdet(M)
    assert abs((lE1 - lE2) + lM) < 1e-9
    assert abs(sM - 1) < 1e-9
    eta = I.heatbath_noise(dims, 8)
    out, _ = A.meofa(o.a, o.U, m1, m2, eta)
    assert rel(out.reshape(-1), M @ eta.reshape(-1)) < 1e-10


def test_heatbath_woodbury_identity(oracle_mod, dense24):
    """Eq. (eofa_heatbath) is the Woodbury rewrite of
    alpha_0 + sum_l alpha_l (M_EOFA + beta_l)^-1: the two agree for any
    coefficients, not only those of a good approximation to x^(-1/2)."""
    from oracle import action as A
    d = dense24
    o = d["o"]
    M = dense_meofa(oracle_mod, d)
    eta = I.heatbath_noise(o.a.dims, 6)
    a0, al, bl = 0.3, [0.7, 0.2, 1.3], [0.05, 0.9, 4.0]
    phi, st = A.heatbath(o.a, o.U, d["m1"], d["m2"], a0, al, bl, eta)
    assert len(st) == 6 and all(s.converged for s in st)
    n = M.shape[0]
    ref = a0 * eta.reshape(-1)
    for a, b in zip(al, bl):
        ref = ref + a * np.linalg.solve(M + b * np.eye(n), eta.reshape(-1))
    assert rel(phi.reshape(-1), ref) < 1e-10


def test_heatbath_error_falls_with_poles(oracle_mod, dense24):
    """epsilon of Eq. (heatbath_rel_err) falls with the number of poles, and
    with enough poles phi is M_EOFA^(-1/2) eta to double precision (Sec. III.B,
    Fig. 2 left: a modest pole count reaches double precision)."""
    from oracle import action as A
    from paper_1706_05843_gb300 import rational
    d = dense24
    o = d["o"]
    M = dense_meofa(oracle_mod, d)
    Mh = 0.5 * (M + M.conj().T)
    w, Q = np.linalg.eigh(Mh)
    eta = I.heatbath_noise(o.a.dims, 7)
    e = eta.reshape(-1)
    exact = Q @ ((Q.conj().T @ e) / np.sqrt(w))
    eps = []
    for n in (2, 4, 10):
        r = rational.inv_sqrt(n, 0.95 * w[0], 1.05 * w[-1])
        phi, _ = A.heatbath(o.a, o.U, d["m1"], d["m2"], r.alpha0, r.alpha, r.beta, eta)
        mphi, _ = A.meofa(o.a, o.U, d["m1"], d["m2"], phi)
        eps.append(A.heatbath_error(eta, phi, mphi))
        # |phi - M^-1/2 eta| <= err |M^-1/2 eta| up to the solver tolerance
        assert rel(phi.reshape(-1), exact) <= 1.01 * r.err + 1e-11
    assert eps[0] > eps[1] > eps[2]
    assert eps[2] < 1e-12


# --------------------------------------------------------------------------
# Cayley form (App. B, Eq. precond_mobius_eofa_system and delta_rank_one)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("coef", [MOBIUS, MOBIUS2, SHAMIR])
@pytest.mark.parametrize("pm", [1, -1])
@pytest.mark.parametrize("beta", [-1.0, 0.0, 0.7])
def test_cayley_identity(oracle_mod, coef, pm, beta):
    """K = (D_EOFA(m1) + beta g5 R5 Delta_pm(m2,m3) P_pm) D~(m1)."""
    o = make(oracle_mod, dims=(4, 2, 2, 4), Ls=8, pm=pm, beta=beta, m2=1.0, m3=0.2, **coef)
    psi = I.gaussian_fermion(o.a.dims, 8, 31)
    assert rel(o.k(psi), o.asys(o.dtilde(psi, o.a.m1))) < 1e-13
    # adjoint of the same identity
    assert rel(o.k(psi, dag=True), o.dtilde(o.asys(psi, dag=True), o.a.m1, dag=True)) < 1e-13


@pytest.mark.parametrize("coef", [MOBIUS, MOBIUS2])
def test_rank_one_shift(oracle_mod, coef):
    """R5 Delta_pm(m2,m3) D~_pm(m1) = u_pm (x) v_pm (App. B)."""
    Ls = 8
    for pm in (1, -1):
        o = make(oracle_mod, dims=(2, 2, 2, 2), Ls=Ls, pm=pm, m1=0.04, m2=1.0, m3=0.3, **coef)
        Lp, Lm = o.L_matrices(0.04)
        Dt = coef["b"] * np.eye(Ls) + coef["c"] * (Lp if pm > 0 else Lm)
        R5 = np.eye(Ls)[::-1]
        lhs = R5 @ o.delta(1.0, 0.3, pm) @ Dt
        u, k = o.uv()
        v = np.zeros(Ls); v[Ls - 1 if pm > 0 else 0] = k
        assert np.abs(lhs - np.outer(u, v)).max() < 1e-14 * np.abs(lhs).max()


def test_beta_zero_reduces_to_dwf(oracle_mod):
    o = make(oracle_mod, beta=0.0, **MOBIUS)
    psi = I.gaussian_fermion(o.a.dims, o.a.Ls, 2)
    assert rel(o.k(psi), o.ddwf(psi, o.a.m1)) < 1e-15
    assert rel(o.asys(psi), o.deofa(psi, o.a.m1)) < 1e-15


def test_equal_shift_masses_remove_the_shift(oracle_mod):
    """k(m2, m3) of App. A carries the factor (m3 - m2): with m3 = m2 the
    shift vanishes for any beta and the system is H(m1) alone; with m3 != m2
    it does not (the check is not vacuous)."""
    psi = I.gaussian_fermion((4, 4, 4, 4), 8, 3)
    for pm in (1, -1):
        o1 = make(oracle_mod, beta=-1.0, pm=pm, m1=0.04, m2=0.5, m3=0.5, **MOBIUS)
        o0 = make(oracle_mod, beta=0.0, pm=pm, m1=0.04, m2=0.5, m3=0.5, **MOBIUS)
        assert rel(o1.hsys(psi), o0.hsys(psi)) < 1e-15
        assert rel(o1.k(psi), o0.k(psi)) < 1e-15
        o2 = make(oracle_mod, beta=-1.0, pm=pm, m1=0.04, m2=0.5, m3=0.6, **MOBIUS)
        assert rel(o2.hsys(psi), o0.hsys(psi)) > 1e-6


@pytest.mark.parametrize("name", ["k", "asys", "ddwf", "deofa", "dw5", "dtilde", "L"])
def test_adjoints(oracle_mod, name):
    o = make(oracle_mod, dims=(4, 2, 2, 4), Ls=6, beta=0.7, m3=0.3, **MOBIUS2)
    x = I.gaussian_fermion(o.a.dims, 6, 41)
    y = I.gaussian_fermion(o.a.dims, 6, 42)
    f = getattr(o, name)
    extra = () if name in ("k", "asys", "dw5") else (0.2,)
    Ax = f(x, *extra, dag=False)
    Ady = f(y, *extra, dag=True)
    lhs, rhs = np.vdot(y, Ax), np.vdot(Ady, x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# --------------------------------------------------------------------------
# solver: dense brute force, true vs recursive residual, H-form vs K-form
# --------------------------------------------------------------------------
@pytest.mark.parametrize("pm", [1, -1])
@pytest.mark.parametrize("beta", [-1.0, 0.0])
def test_solve_h_dense(oracle_mod, pm, beta):
    O = oracle_mod
    dims, Ls = (2, 2, 2, 2), 4
    a = O.Action(dims=dims, Ls=Ls, pm=pm, beta=beta, **MOBIUS)
    o = O.Oracle(a, I.gauge_field(dims, 0.5, 1))
    n = 16 * Ls * 12
    A = assemble(o.hsys, n, o.shape5)
    phi = I.gaussian_fermion(dims, Ls, 1001)
    exact = np.linalg.solve(A, phi.reshape(-1)).reshape(o.shape5)
    psi, st = o.solve_h(phi, tol=1e-12)
    assert st.converged
    assert st.true_res < 1e-11
    assert abs(st.true_res - st.recur_res) < 1e-11
    assert rel(psi, exact) < 1e-9


def test_solve_k_relates_to_h(oracle_mod):
    """H-form solution = D~(m1) . K-form solution of K psi' = g5 R5 phi."""
    o = make(oracle_mod, dims=(4, 4, 2, 4), Ls=6, eps=0.3, **MOBIUS)
    phi = I.gaussian_fermion(o.a.dims, 6, 1001)
    psi, st = o.solve_h(phi, tol=1e-12)
    psip, st2 = o.solve_k(o.g5r5(phi), tol=1e-12)
    assert st.converged and st2.converged
    assert rel(psi, o.dtilde(psip, o.a.m1)) < 1e-9
    assert rel(o.hsys(psi), phi) < 1e-11
    assert rel(o.k(psip), o.g5r5(phi)) < 1e-11


def test_solve_free_field_closed_form(oracle_mod):
    """Unit links, one plane wave: the K-form solve equals the inverse of the
    momentum-space 4Ls x 4Ls matrix of K (colour identity)."""
    O = oracle_mod
    dims, Ls = (4, 4, 4, 4), 4
    a = O.Action(dims=dims, Ls=Ls, beta=-1.0, **MOBIUS)
    o = O.Oracle(a, I.unit_gauge(dims))
    p = np.array([np.pi / 2, np.pi, 0, np.pi / 4])
    t, z, y, x = np.meshgrid(*(np.arange(4),) * 4, indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    rng = np.random.default_rng(9)
    eta = rng.standard_normal((Ls, 4, 3)) + 1j * rng.standard_normal((Ls, 4, 3))
    b = phase[..., None, None, None] * eta
    # momentum-space K: apply the oracle to the 4Ls basis plane waves
    Kp = np.zeros((Ls * 4, Ls * 4), dtype=complex)
    for j in range(Ls * 4):
        e = np.zeros((Ls, 4, 3), dtype=complex)
        e[j // 4, j % 4, 0] = 1
        out = o.k(phase[..., None, None, None] * e)
        Kp[:, j] = (out[0, 0, 0, 0] / phase[0, 0, 0, 0])[:, :, 0].reshape(-1)
    sol = np.linalg.solve(Kp, eta.transpose(2, 0, 1).reshape(3, Ls * 4).T).T.reshape(3, Ls, 4).transpose(1, 2, 0)
    psip, st = o.solve_k(b, tol=1e-13)
    assert st.converged
    assert rel(psip, phase[..., None, None, None] * sol) < 1e-10


@pytest.mark.parametrize("coef", [MOBIUS, SHAMIR])
@pytest.mark.parametrize("pm", [1, -1])
def test_k_at_sites_matches_full_lattice(oracle_mod, coef, pm):
    """The site-by-site evaluation (used at full benchmark sizes) agrees with
    the full-lattice operator: Eq. (Ddwf) regrouped as D_W chi + psi - L psi."""
    o = make(oracle_mod, dims=(4, 4, 2, 6), Ls=8, pm=pm, beta=0.7, m3=0.3, **coef)
    psi = I.gaussian_fermion(o.a.dims, 8, 51)
    full = o.k(psi).reshape(-1, 8, 4, 3)
    sites = np.array([0, 1, 5, 17, 63, 100, 191])
    assert rel(o.k_sites(psi, sites), full[sites]) < 1e-14
