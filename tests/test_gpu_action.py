"""GPU parity of the EOFA action calls: switching a context's system,
M_EOFA phi (Eq. eofa_action) and the heatbath M_EOFA^(-1/2) eta
(Eq. eofa_heatbath), through the C ABI against the FP64 CPU oracle.

The heatbath is compared with the oracle's for arbitrary coefficients (the
Woodbury form holds for any alpha, beta), and with coefficients that
approximate x^(-1/2) on an interval holding the spectrum of M_EOFA its
error epsilon (Eq. heatbath_rel_err) is judged with the oracle's M_EOFA.
"""
import numpy as np
import pytest

from paper_1706_05843_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MOB = dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, t_bc=-1)
M1, M2 = 0.04, 1.0
# (dims, Ls, eps, action overrides)
CASES = [((4, 4, 4, 4), 8, 0.3, {}),
         ((2, 2, 2, 6), 4, 0.5, dict(beta=0.7, pm=-1, m3=0.3)),
         ((2, 4, 2, 4), 16, 0.5, dict(b=1.4, c=0.8))]
IDS = [f"{'x'.join(map(str, d))}_Ls{l}" for d, l, _, _ in CASES]
# the spectrum of M_EOFA on these fields lies in about [1.0, 8.7]
SPECTRUM = (0.5, 20.0)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_05843_gb300 import build
    build.build()
    import oracle
    oracle.build()
    from paper_1706_05843_gb300 import binding as B
    B.lib()
    return torch, B, oracle


def setup(env, case, seed=1):
    torch, B, O = env
    dims, Ls, eps, kw = case
    act = dict(MOB)
    act.update(kw)
    U = I.gauge_field(dims, eps, seed)
    a = O.Action(dims=dims, Ls=Ls, **act)
    return torch, B.Solver(U, dims, Ls, **act), a, U


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_set_system_matches_fresh_context(env, case):
    """After eofa_set_system the context applies and solves the new system
    (the oracle built for it judges), and switching back restores the old."""
    torch, s, a, U = setup(env, case)
    O = env[2]
    psi = I.gaussian_fermion(a.dims, a.Ls, 77)
    x = torch.from_numpy(psi).cuda()
    new = dict(m1=0.3, m2=0.04, m3=0.6, beta=-0.4, pm=-a.pm)
    s.set_system(**new)
    o_new = O.Oracle(a.replace(**new), U)
    assert rel(s.apply_h(x).cpu().numpy(), o_new.hsys(psi)) < 1e-12
    sol, st = s.solve(x, tol=1e-10, inner="f32")
    assert rel(o_new.hsys(sol.cpu().numpy()), psi) <= 1e-10, st.as_dict()
    s.set_system(a.m1, a.m2, a.m3, a.beta, a.pm)
    o_old = O.Oracle(a, U)
    assert rel(s.apply_h(x).cpu().numpy(), o_old.hsys(psi)) < 1e-12
    sol, st = s.solve(x, tol=1e-10, inner="f32")
    assert rel(o_old.hsys(sol.cpu().numpy()), psi) <= 1e-10, st.as_dict()
    s.close()


def test_set_system_rejects_singular(env):
    torch, s, a, U = setup(env, CASES[0])
    from paper_1706_05843_gb300 import binding as B
    with pytest.raises(B.EofaError) as e:
        s.set_system(0.04, 1.0, 0.04, -1.0, 2)
    assert e.value.status == 1
    # N(m) = b5^Ls + m c5^Ls = 0 at m = -(b5/c5)^Ls
    with pytest.raises(B.EofaError) as e:
        s.set_system(-(1.5 / 0.5) ** 8, 1.0, 0.04, -1.0, 1)
    assert e.value.status == 3
    # the context still solves its own system
    O = env[2]
    psi = I.gaussian_fermion(a.dims, a.Ls, 78)
    assert rel(s.apply_h(torch.from_numpy(psi).cuda()).cpu().numpy(), O.Oracle(a, U).hsys(psi)) < 1e-12
    s.close()


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_meofa_parity(env, case, inner):
    torch, s, a, U = setup(env, case)
    from oracle import action as A
    eta = I.heatbath_noise(a.dims, 11)
    out, st = s.apply_meofa(torch.from_numpy(eta).cuda(), M1, M2, tol=1e-11, inner=inner)
    ref, _ = A.meofa(a, U, M1, M2, eta)
    assert all(x.status == 0 and x.true_res <= 1e-11 for x in st), [x.as_dict() for x in st]
    assert rel(out.cpu().numpy(), ref) < 1e-9
    # the context's own system is back
    psi = I.gaussian_fermion(a.dims, a.Ls, 79)
    O = env[2]
    assert rel(s.apply_h(torch.from_numpy(psi).cuda()).cpu().numpy(), O.Oracle(a, U).hsys(psi)) < 1e-12
    s.close()


class Coef:
    def __init__(self, alpha0, alpha, beta):
        self.alpha0, self.alpha, self.beta = alpha0, list(alpha), list(beta)


ARBITRARY = Coef(0.3, [0.7, 0.2, 1.3], [0.05, 0.9, 4.0])


@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
@pytest.mark.parametrize("inner,forecast", [("f64", 0), ("f32", 0), ("f32", 2)])
def test_heatbath_parity(env, case, inner, forecast):
    """Eq. (eofa_heatbath) on the GPU equals the oracle's for the same
    coefficients, with and without the chronological guess."""
    torch, s, a, U = setup(env, case)
    from oracle import action as A
    eta = I.heatbath_noise(a.dims, 12)
    phi, st = s.heatbath(torch.from_numpy(eta).cuda(), M1, M2, ARBITRARY, forecast=forecast, tol=1e-11,
                         inner=inner)
    ref, _ = A.heatbath(a, U, M1, M2, ARBITRARY.alpha0, ARBITRARY.alpha, ARBITRARY.beta, eta)
    assert len(st) == 6 and all(x.status == 0 and x.true_res <= 1e-11 for x in st)
    assert rel(phi.cpu().numpy(), ref) < 1e-9
    s.close()


@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_heatbath_error(env, case):
    """epsilon = |eta^dag eta - phi^dag M phi| / eta^dag eta, with M_EOFA phi
    from the oracle, reaches the solver's accuracy with 10 poles (Sec. III.B),
    and is far larger with 3 (Fig. 2 left: it falls with the pole count)."""
    torch, s, a, U = setup(env, case)
    from oracle import action as A
    from paper_1706_05843_gb300 import rational
    eta = I.heatbath_noise(a.dims, 13)
    e = torch.from_numpy(eta).cuda()
    eps = {}
    for n in (3, 10):
        r = rational.inv_sqrt(n, *SPECTRUM)
        phi, st = s.heatbath(e, M1, M2, r, tol=1e-12, inner="f32")
        phi = phi.cpu().numpy()
        mphi, _ = A.meofa(a, U, M1, M2, phi)
        eps[n] = A.heatbath_error(eta, phi, mphi)
        # the GPU's own M_EOFA gives the same epsilon
        mg, _ = s.apply_meofa(torch.from_numpy(phi).cuda(), M1, M2, tol=1e-12, inner="f32")
        assert abs(A.heatbath_error(eta, phi, mg.cpu().numpy()) - eps[n]) < 1e-10
        # and the library's device inner products give it too
        from paper_1706_05843_gb300 import heatbath as H
        assert abs(H.heatbath_error(s, e, torch.from_numpy(phi).cuda(), mg) - eps[n]) < 1e-10
    assert eps[10] < 1e-10
    assert eps[3] > 1e3 * eps[10]
    s.close()


def test_heatbath_forecast_and_pole_tolerances(env):
    """The chronological guess (Sec. V.B) leaves phi unchanged to the solver
    tolerance and cuts the iterations of the later poles; loosened per-pole
    tolerances are obeyed and cut iterations further."""
    case = CASES[0]
    torch, s, a, U = setup(env, case)
    from paper_1706_05843_gb300 import rational
    r = rational.inv_sqrt(8, *SPECTRUM)
    e = torch.from_numpy(I.heatbath_noise(a.dims, 14)).cuda()
    phi0, st0 = s.heatbath(e, M1, M2, r, forecast=0, tol=1e-10, inner="f32")
    phi4, st4 = s.heatbath(e, M1, M2, r, forecast=4, tol=1e-10, inner="f32")
    assert rel(phi4.cpu().numpy(), phi0.cpu().numpy()) < 1e-8
    it0 = [x.inner_iters for x in st0]
    it4 = [x.inner_iters for x in st4]
    print("iterations without / with forecasting:", it0, it4)
    # the later poles: measured 364 against 754 iterations on this field
    assert sum(it4[8:]) < 0.7 * sum(it0[8:])
    tols = [1e-10] * 4 + [1e-6] * (len(it0) - 4)
    phit, stt = s.heatbath(e, M1, M2, r, pole_tol=tols, forecast=0, tol=1e-10, inner="f32")
    assert all(x.true_res <= t for x, t in zip(stt, tols))
    assert sum(x.inner_iters for x in stt) < sum(it0)
    s.close()


def test_heatbath_arguments(env):
    torch, s, a, U = setup(env, CASES[0])
    from paper_1706_05843_gb300 import binding as B
    e = torch.from_numpy(I.heatbath_noise(a.dims, 15)).cuda()
    phi = torch.empty_like(e)
    opts = B.make_opts(tol=1e-10)
    for kw in (dict(beta=[-1.0]), dict(beta=[float("nan")])):
        with pytest.raises(B.EofaError) as ex:
            B.eofa_heatbath(s.ctx, M1, M2, 0.1, [1.0], kw["beta"], e, phi, opts)
        assert ex.value.status == 1
    with pytest.raises(B.EofaError) as ex:
        B.eofa_heatbath(s.ctx, M1, M2, 0.1, [1.0], [0.5], e, phi, opts, forecast=9)
    assert ex.value.status == 1
    with pytest.raises(B.EofaError) as ex:
        B.eofa_heatbath(s.ctx, M1, M2, 0.1, [1.0], [0.5], e, e, opts)
    assert ex.value.status == 1
    # no poles: phi = alpha_0 eta
    B.eofa_heatbath(s.ctx, M1, M2, 0.25, [], [], e, phi, opts)
    assert rel(phi.cpu().numpy(), 0.25 * e.cpu().numpy()) < 1e-15
    s.close()


def test_largest_eigenvalue_matches_oracle(env):
    """Power iteration through the library's M_EOFA gives the oracle's
    Rayleigh quotients, which rise monotonically (M_EOFA is Hermitian
    positive definite)."""
    torch, s, a, U = setup(env, CASES[1])
    from oracle import action as A
    from paper_1706_05843_gb300 import heatbath as H
    v0 = I.heatbath_noise(a.dims, 3)
    lam, hist = H.largest_eigenvalue(s, M1, M2, torch.from_numpy(v0).cuda(), iters=8, tol=1e-12, inner="f32")
    v = v0 / np.linalg.norm(v0)
    ref = []
    for _ in range(8):
        w, _ = A.meofa(a, U, M1, M2, v)
        ref.append(np.vdot(v, w).real / np.vdot(v, v).real)
        v = w / np.linalg.norm(w)
    assert np.allclose(hist, ref, rtol=1e-9)
    assert all(x <= y * (1 + 1e-12) for x, y in zip(hist, hist[1:]))
    s.close()


def test_pole_tolerance_tuning(env):
    """The per-solve tolerance tuning of Sec. V.B keeps epsilon below its
    target while relaxing tolerances and cutting the iteration count."""
    torch, s, a, U = setup(env, CASES[0])
    from paper_1706_05843_gb300 import heatbath as H
    from paper_1706_05843_gb300 import rational
    r = rational.poles_for(1e-11, *SPECTRUM)
    e = torch.from_numpy(I.heatbath_noise(a.dims, 16)).cuda()
    _, eps0, st0 = H.measure(s, e, M1, M2, r, tol=1e-10, inner="f32")
    tols, eps, trials = H.tune_pole_tolerances(s, e, M1, M2, r, eps_tol=1e-9, tol=1e-10, factor=100.0,
                                               max_tol=1e-4, inner="f32")
    _, eps1, st1 = H.measure(s, e, M1, M2, r, pole_tol=tols, tol=1e-10, inner="f32")
    it0, it1 = sum(x.inner_iters for x in st0), sum(x.inner_iters for x in st1)
    print(f"untuned eps {eps0:.3g} {it0} iterations; tuned eps {eps1:.3g} {it1} iterations; "
          f"{trials} trials; tolerances {tols}")
    assert eps0 <= 1e-9 and eps1 <= 1e-9
    assert max(tols) > 1e-10
    assert it1 < it0
    s.close()


FORCE_CASES = [((4, 4, 2, 4), 4, 0.5, {}), CASES[0], CASES[2]]
FORCE_IDS = ["4x4x2x4_Ls4", IDS[0], IDS[2]]


@pytest.mark.parametrize("case", FORCE_CASES, ids=FORCE_IDS)
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_force_parity(env, case, inner):
    """The EOFA force (Eq. eofa_force) per link against the oracle's, whose
    closed form is pinned to finite differences of the action."""
    torch, s, a, U = setup(env, case)
    from oracle import force as F
    phi = I.heatbath_noise(a.dims, 21)
    f, st = s.force(torch.from_numpy(phi).cuda(), M1, M2, tol=1e-12, inner=inner)
    assert all(x.status == 0 for x in st)
    dS, Fo, imag, _ = F.eofa_force(a, U, M1, M2, phi)
    f = f.cpu().numpy()
    assert rel(f, Fo) < 1e-9
    # anti-Hermitian and traceless
    assert np.abs(f + np.swapaxes(f, -1, -2).conj()).max() < 1e-14 * np.abs(f).max() + 1e-300
    assert np.abs(np.trace(f, axis1=-2, axis2=-1)).max() < 1e-13 * np.abs(f).max()
    # d^a S = -2 Tr(T^a F) recovers the oracle's derivatives
    dS_gpu = -2.0 * np.einsum("aij,...ji->...a", F.generators(), f).real
    assert np.abs(dS_gpu - dS).max() < 1e-9 * np.abs(dS).max()
    s.close()
