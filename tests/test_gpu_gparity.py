"""GPU parity with G-parity boundary conditions (Sec. I): the library's
G-parity context (two flavours stacked along t, conjugate links on flavour
2, flavour-changing boundary hops) against the oracle's flavour-doubled
operators written directly from the boundary conditions."""
import numpy as np
import pytest

from paper_1706_05843_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MOB = dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, beta=-1.0, pm=1, t_bc=-1)
M1, M2 = 0.04, 1.0
# (dims, Ls, eps, G-parity directions, action overrides)
CASES = [((4, 4, 2, 4), 4, 0.5, 1, {}),
         ((4, 4, 4, 4), 8, 0.3, 3, dict(beta=0.7, pm=-1, m3=0.3)),
         ((2, 4, 2, 4), 16, 0.5, 8, dict(b=1.4, c=0.8, t_bc=1)),
         ((4, 2, 4, 6), 12, 0.5, 15, {})]
IDS = [f"{'x'.join(map(str, d))}_Ls{l}_g{g}" for d, l, _, g, _ in CASES]


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
    from oracle.gparity import GOracle
    dims, Ls, eps, gm, kw = case
    act = dict(MOB)
    act.update(kw)
    U = I.gauge_field(dims, eps, seed)
    a = O.Action(dims=dims, Ls=Ls, **act)
    return torch, B.Solver(U, dims, Ls, gparity=gm, **act), GOracle(a, U, gm), a, U


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def two_flavour(dims, Ls, seed):
    return np.stack([I.gaussian_fermion(dims, Ls, seed), I.gaussian_fermion(dims, Ls, seed + 1)])


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_gparity_apply_parity(env, case):
    torch, s, g, a, U = setup(env, case)
    psi = two_flavour(a.dims, a.Ls, 77)
    out = s.apply_h(torch.from_numpy(psi).cuda()).cpu().numpy()
    assert out.shape == psi.shape
    assert rel(out, g.hsys(psi)) < 1e-12
    s.close()


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_gparity_solve(env, case, inner):
    torch, s, g, a, U = setup(env, case)
    phi = two_flavour(a.dims, a.Ls, 1001)
    psi, st = s.solve(torch.from_numpy(phi).cuda(), tol=1e-10, inner=inner)
    assert rel(g.hsys(psi.cpu().numpy()), phi) <= 1e-10, st.as_dict()
    s.close()


def stacked(a, U):
    """The C oracle of the flavour-stacked lattice X x Y x Z x 2T, links
    [U; U^*], antiperiodic seam: G-parity in t with t_bc = +1 (the
    equivalence is pinned on the CPU)."""
    X, Y, Z, T = a.dims
    return a.replace(dims=(X, Y, Z, 2 * T), t_bc=-1), np.concatenate([U, U.conj()])


def test_gparity_meofa_and_force_t(env):
    """M_EOFA phi and the force on the physical links for G-parity in t,
    against the oracle on the stacked lattice (force folded: flavour 1's
    link plus the conjugate of flavour 2's)."""
    from oracle import action as A
    from oracle import force as F
    torch, s, g, a, U = setup(env, CASES[2])
    X, Y, Z, T = a.dims
    sa, sU = stacked(a, U)
    phi = np.stack([I.heatbath_noise(a.dims, 21), I.heatbath_noise(a.dims, 22)])
    e = torch.from_numpy(phi).cuda()
    out, st = s.apply_meofa(e, M1, M2, tol=1e-12, inner="f32")
    ref, _ = A.meofa(sa, sU, M1, M2, phi.reshape((2 * T, Z, Y, X, 4, 3)))
    assert rel(out.cpu().numpy().reshape(ref.shape), ref) < 1e-9
    f, st = s.force(e, M1, M2, tol=1e-12, inner="f32")
    _, Fs, _, _ = F.eofa_force(sa, sU, M1, M2, phi.reshape((2 * T, Z, Y, X, 4, 3)))
    assert rel(f.cpu().numpy(), Fs[:T] + Fs[T:].conj()) < 1e-9
    s.close()


def test_gparity_force_matches_action_differences(env):
    """G-parity in x and z: the library's force on the physical links equals
    central differences of the library's own S = phi^dag M_EOFA phi under
    U_mu(x) -> exp(s T^a) U_mu(x), on a G-parity boundary link, an interior
    link and a time-boundary link."""
    from scipy.linalg import expm
    from oracle import force as F
    torch, B, O = env
    dims, Ls, gm = (4, 2, 4, 4), 4, 5
    act = dict(MOB)
    U = I.gauge_field(dims, 0.5, 4)
    phi = np.stack([I.heatbath_noise(dims, 31), I.heatbath_noise(dims, 32)])
    e = torch.from_numpy(phi).cuda()

    def S(Uc):
        s = B.Solver(Uc, dims, Ls, gparity=gm, **act)
        m, _ = s.apply_meofa(e, M1, M2, tol=1e-13, inner="f64")
        s.close()
        return float(torch.vdot(e.flatten(), m.flatten()).real)

    s = B.Solver(U, dims, Ls, gparity=gm, **act)
    f, _ = s.force(e, M1, M2, tol=1e-13, inner="f64")
    f = f.cpu().numpy()
    s.close()
    assert np.abs(f + np.swapaxes(f, -1, -2).conj()).max() < 1e-13 * np.abs(f).max()
    Tg = F.generators()
    h = 5e-4
    for (x, y, z, t), mu, gen in [((3, 1, 0, 2), 0, 3), ((1, 0, 3, 1), 2, 6), ((2, 1, 1, 0), 1, 1),
                                  ((0, 0, 2, 3), 3, 0)]:
        vals = []
        for sg in (+1, -1):
            Up = U.copy()
            Up[t, z, y, x, mu] = expm(sg * h * Tg[gen]) @ U[t, z, y, x, mu]
            vals.append(S(Up))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = -2.0 * np.trace(Tg[gen] @ f[t, z, y, x, mu]).real
        assert abs(fd - an) < 1e-5 * (np.abs(f).max() + abs(an)), (fd, an)
