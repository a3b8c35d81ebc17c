"""GPU parity at the benchmark sizes, in the launch configuration bench.py
times, judged by the FP64 oracle on the whole lattice.

* 16^3x32 Ls=16 (links exp(i 0.5 H)) and 24^3x64 Ls=12 (exp(i 0.7 H),
  m1 = m3 = 0.0362): K and K^dag applied by the GPU equal the oracle's on
  every site to 1e-12.
* Every solve form is judged by the oracle's own full-lattice operator:
  ||phi - (H + beta Delta P) psi|| / ||phi|| <= 1e-10 for the H form (the
  stopping tolerance of the defect-correction scheme, Sec. V.A) and
  ||b - K psi'|| / ||b|| <= 1e-10 for the K form (App. B), at 16^3x32 Ls=16
  with FP64, FP32, FP16 and BF16 inner storage and at 24^3x64 Ls=12 with FP32, FP16
  and BF16 inner storage for each of its four right-hand sides; the GPU's own
  true residual agrees with the oracle's.
* The batched workload (16 right-hand sides, 8 on 16^4 Ls=16 and 8 on
  12^3x24 Ls=12, one eofa_solve_batched call): every system judged the same
  way by the oracle of its own lattice.
* The FP64-inner solution of the benchmark solve agrees element by element
  with the oracle's solution of the same system at the 48 sites stored in
  tests/golden (written by tests/golden/oracle_solution_sample.py).
"""
import os

import numpy as np
import pytest

from paper_1706_05843_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ACT = dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, beta=-1.0, pm=1, t_bc=-1)
CFG2 = ((16, 16, 16, 32), 16, 0.5, {})
CFG3 = ((24, 24, 24, 64), 12, 0.7, dict(m1=0.0362, m3=0.0362))
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_psi_16x16x16x32_Ls16.npz")
TOL = 1e-10


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


_CACHE = {}


def workload(env, case):
    """(gauge, oracle, solver) of a benchmark lattice, built once per module."""
    torch, B, O = env
    dims, Ls, eps, kw = case
    key = (dims, Ls)
    if key not in _CACHE:
        act = dict(ACT, **kw)
        U = I.gauge_field(dims, eps, 1)
        _CACHE.clear()   # one large lattice resident at a time
        _CACHE[key] = (U, O.Oracle(O.Action(dims=dims, Ls=Ls, **act), U), B.Solver(U, dims, Ls, **act))
    return _CACHE[key]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def check_apply(env, case):
    torch = env[0]
    _, o, s = workload(env, case)
    psi = I.gaussian_fermion(case[0], case[1], 77)
    x = torch.from_numpy(psi).cuda()
    assert rel(s.apply(x).cpu().numpy(), o.k(psi)) < 1e-12
    assert rel(s.apply(x, dag=True).cpu().numpy(), o.k(psi, dag=True)) < 1e-12


def test_fullsize_apply_whole_lattice_16c32(env):
    check_apply(env, CFG2)


@pytest.mark.parametrize("inner", ["f64", "f32", "f16", "bf16"])
def test_fullsize_h_solve_judged_by_oracle(env, inner):
    """The benchmark solve (H form, 16^3x32 Ls=16, rhs seed 1001)."""
    torch = env[0]
    _, o, s = workload(env, CFG2)
    phi = I.gaussian_fermion(CFG2[0], CFG2[1], 1001)
    psi, st = s.solve(torch.from_numpy(phi).cuda(), tol=TOL, inner=inner)
    res = rel(o.hsys(psi.cpu().numpy()), phi)
    print(f"16^3x32 Ls=16 {inner}: oracle residual {res:.4e}, GPU true residual {st.true_res:.4e}, "
          f"{st.outer_iters} outer / {st.inner_iters} inner iterations")
    assert st.status == 0
    assert res <= TOL, res
    assert abs(res - st.true_res) <= 1e-12


def test_fullsize_k_solve_judged_by_oracle(env):
    torch = env[0]
    _, o, s = workload(env, CFG2)
    b = o.g5r5(I.gaussian_fermion(CFG2[0], CFG2[1], 1001))
    psip, st = s.solve(torch.from_numpy(b).cuda(), tol=TOL, inner="f32", rhs_form=1)
    res = rel(o.k(psip.cpu().numpy()), b)
    assert st.status == 0 and res <= TOL, res


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="stored oracle solution not written")
def test_fullsize_solution_matches_stored_oracle_solution(env):
    """psi from the FP64-inner solve against the oracle's psi (solved to
    1e-12) at the stored sites.  Both have relative residual <= 1e-10, so
    their difference is A^-1 times a residual of that size; the bound below
    allows a condition number of 1e3."""
    torch = env[0]
    _, o, s = workload(env, CFG2)
    g = np.load(GOLDEN)
    assert float(g["residual"]) <= 1e-12
    phi = I.gaussian_fermion(CFG2[0], CFG2[1], 1001)
    for inner in ("f64", "f32"):
        psi, st = s.solve(torch.from_numpy(phi).cuda(), tol=TOL, inner=inner)
        got = psi.cpu().numpy().reshape(-1, CFG2[1], 4, 3)[g["sites"]]
        err = rel(got, g["psi"])
        print(f"{inner}: |psi - psi_oracle| / |psi_oracle| at the stored sites = {err:.3e}")
        assert err <= 1e-7, (inner, err)


def test_fullsize_apply_whole_lattice_24c64(env):
    check_apply(env, CFG3)


@pytest.mark.parametrize("inner", ["f16", "bf16", "f32"])
def test_fullsize_24c64_solves_judged_by_oracle(env, inner):
    """24^3x64 Ls=12, m = 0.0362, the four right-hand sides of the workload."""
    torch = env[0]
    _, o, s = workload(env, CFG3)
    for k in range(4):
        phi = I.gaussian_fermion(CFG3[0], CFG3[1], 1001 + k)
        psi, st = s.solve(torch.from_numpy(phi).cuda(), tol=TOL, inner=inner)
        res = rel(o.hsys(psi.cpu().numpy()), phi)
        print(f"24^3x64 Ls=12 {inner} rhs {k}: oracle residual {res:.4e}, {st.inner_iters} inner iterations")
        assert st.status == 0 and res <= TOL, (k, res)
        assert abs(res - st.true_res) <= 1e-12


def test_batched_uneven_workload_judged_by_oracle(env):
    """The batched workload: 16 right-hand sides over 16^4 Ls=16 (gauge seed
    1) and 12^3x24 Ls=12 (gauge seed 2), links exp(i 0.5 H), FP32 inner, in
    one eofa_solve_batched call."""
    torch, B, O = env
    _CACHE.clear()
    groups = [((16, 16, 16, 16), 16, 1), ((12, 12, 12, 24), 12, 2)]
    solvers, oracles, phis = [], [], []
    k = 0
    for dims, Ls, gseed in groups:
        U = I.gauge_field(dims, 0.5, gseed)
        o = O.Oracle(O.Action(dims=dims, Ls=Ls, **ACT), U)
        Ud = torch.from_numpy(U).cuda()
        for _ in range(8):
            solvers.append(B.Solver(Ud, dims, Ls, **ACT))
            oracles.append(o)
            phis.append(I.gaussian_fermion(dims, Ls, 1001 + k))
            k += 1
    rhs = [torch.from_numpy(p).cuda() for p in phis]
    sols = [torch.empty_like(r) for r in rhs]
    st = B.eofa_solve_batched([s.ctx for s in solvers], rhs, sols, B.make_opts(tol=TOL, inner="f32"))
    for i, (o, phi, x, t) in enumerate(zip(oracles, phis, sols, st)):
        res = rel(o.hsys(x.cpu().numpy()), phi)
        assert t.status == 0 and res <= TOL, (i, res, t.as_dict())
        assert abs(res - t.true_res) <= 1e-12
    for s in solvers:
        s.close()


def test_fullsize_force_and_heatbath_properties(env):
    """At 16^3x32 Ls=16 the force must be the derivative of the library's own
    action S = phi^dag M_EOFA phi: central differences along
    U_mu(x) -> exp(s T^a) U_mu(x) on the link and generator with the largest
    force component; and a heatbath with Zolotarev coefficients on an
    interval holding the spectrum gives epsilon <= 1e-9 (Eq. heatbath_rel_err),
    properties that hold at any size."""
    from scipy.linalg import expm
    from oracle.force import generators
    from paper_1706_05843_gb300 import heatbath as H
    from paper_1706_05843_gb300 import rational
    torch, B, O = env
    _CACHE.clear()
    dims, Ls, eps = (16, 16, 16, 32), 16, 0.5
    U = I.gauge_field(dims, eps, 1)
    phi = torch.from_numpy(I.heatbath_noise(dims, 31)).cuda()
    m1, m2 = ACT["m1"], ACT["m2"]
    s = B.Solver(U, dims, Ls, **ACT)
    f, _ = s.force(phi, m1, m2, tol=1e-13, inner="f32")
    f = f.cpu().numpy()
    Tg = generators()
    comp = -2.0 * np.einsum("aij,...ji->...a", Tg, f).real    # d^a S per link
    idx = np.unravel_index(np.argmax(np.abs(comp)), comp.shape)
    t, z, y, x, mu, gen = (int(i) for i in idx)
    h = 1e-3
    vals = []
    for sg in (+1, -1):
        Up = U.copy()
        Up[t, z, y, x, mu] = expm(sg * h * Tg[gen]) @ U[t, z, y, x, mu]
        sp = B.Solver(Up, dims, Ls, **ACT)
        m, _ = sp.apply_meofa(phi, m1, m2, tol=1e-13, inner="f32")
        vals.append(float(torch.vdot(phi.flatten(), m.flatten()).real))
        sp.close()
    fd = (vals[0] - vals[1]) / (2 * h)
    an = comp[idx]
    assert abs(fd - an) < 2e-3 * abs(an), (fd, an, idx)
    # heatbath error on [0.5, 30] (the spectrum ends near 21.8 here)
    r = rational.poles_for(1e-11, 0.5, 30.0)
    eta = phi
    out, st = s.heatbath(eta, m1, m2, r, forecast=4, tol=1e-11, inner="f32")
    mo, _ = s.apply_meofa(out, m1, m2, tol=1e-12, inner="f32")
    assert H.heatbath_error(s, eta, out, mo) < 1e-9
    s.close()
