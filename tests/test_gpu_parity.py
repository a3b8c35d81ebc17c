"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Operator application (K, K^dag, H + beta Delta P) must agree element by
element to 1e-12 relative (FP64).  Every solve is judged by the oracle's own
operator: ||phi - (H + beta Delta P) psi_gpu|| / ||phi|| <= 1e-10 (H form) or
||b - K psi'_gpu|| / ||b|| <= 1e-10 (K form), and the solution is compared
with the oracle's to the accuracy that residual implies.
"""
import numpy as np
import pytest

from paper_1706_05843_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MOB = dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, t_bc=-1)

# (dims, Ls, eps, action overrides): config-1 point, chiralities, beta values,
# Shamir and b - c != 1, every compiled Ls, and ragged tiles (the number of
# sites per parity is not a multiple of the CTA tile).
CASES = [
    ((4, 4, 4, 4), 8, 0.3, dict(beta=-1.0, pm=1)),
    ((4, 4, 4, 4), 8, 0.3, dict(beta=0.0, pm=1)),
    ((4, 4, 4, 4), 8, 0.3, dict(beta=0.7, pm=-1, m3=0.3)),
    ((4, 4, 4, 4), 8, 0.3, dict(beta=-1.0, pm=-1, m2=0.6, m3=0.1)),
    ((6, 2, 2, 2), 8, 0.5, dict(beta=-1.0, pm=1)),
    ((2, 2, 2, 6), 4, 0.5, dict(beta=0.7, pm=1)),
    ((4, 2, 6, 2), 12, 0.7, dict(beta=-1.0, pm=-1, m1=0.0362, m3=0.0362)),
    ((2, 4, 2, 4), 16, 0.5, dict(beta=-1.0, pm=1)),
    ((4, 4, 2, 2), 8, 0.5, dict(beta=-1.0, pm=1, b=1.0, c=0.0)),
    ((4, 2, 4, 2), 8, 0.5, dict(beta=0.7, pm=-1, b=1.4, c=0.8, m3=0.2)),
]
IDS = [f"{'x'.join(map(str, d))}_Ls{l}_{i}" for i, (d, l, _, _) in enumerate(CASES)]


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
    o = O.Oracle(O.Action(dims=dims, Ls=Ls, **act), U)
    s = B.Solver(U, dims, Ls, **act)
    return torch, s, o


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_apply_parity(env, case):
    torch, s, o = setup(env, case)
    psi = I.gaussian_fermion(case[0], case[1], 77)
    x = torch.from_numpy(psi).cuda()
    assert rel(s.apply(x).cpu().numpy(), o.k(psi)) < 1e-12
    assert rel(s.apply(x, dag=True).cpu().numpy(), o.k(psi, dag=True)) < 1e-12
    assert rel(s.apply_h(x).cpu().numpy(), o.hsys(psi)) < 1e-12
    s.close()


@pytest.mark.parametrize("case", CASES[:4] + CASES[5:8], ids=IDS[:4] + IDS[5:8])
@pytest.mark.parametrize("inner", ["f64", "f32", "f16", "bf16"])
def test_solve_h_parity(env, case, inner):
    torch, s, o = setup(env, case)
    phi = I.gaussian_fermion(case[0], case[1], 1001)
    psi, st = s.solve(torch.from_numpy(phi).cuda(), tol=1e-10, inner=inner)
    psi = psi.cpu().numpy()
    res = rel(o.hsys(psi), phi)
    assert res <= 1e-10, (res, st.as_dict())
    assert st.true_res <= 1e-10
    assert abs(st.true_res - res) < 1e-11
    ref, ost = o.solve_h(phi, tol=1e-12)
    # |psi - psi_ref| / |psi_ref| is bounded by cond * residual; the
    # fields here are small and well conditioned
    assert rel(psi, ref) < 1e-6
    s.close()


@pytest.mark.parametrize("case", CASES[:1] + CASES[2:3] + CASES[8:], ids=IDS[:1] + IDS[2:3] + IDS[8:])
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_solve_k_parity(env, case, inner):
    torch, s, o = setup(env, case)
    b = I.gaussian_fermion(case[0], case[1], 1002)
    psip, st = s.solve(torch.from_numpy(b).cuda(), tol=1e-10, inner=inner, rhs_form=1)
    psip = psip.cpu().numpy()
    assert rel(o.k(psip), b) <= 1e-10
    s.close()


def test_solve_with_guess_and_zero_rhs(env):
    torch, s, o = setup(env, CASES[0])
    phi = I.gaussian_fermion(CASES[0][0], CASES[0][1], 1001)
    x = torch.from_numpy(phi).cuda()
    psi, st = s.solve(x, tol=1e-10, inner="f64")
    # restart from the converged answer: no inner iteration is needed
    psi2, st2 = s.solve(x, tol=1e-10, inner="f64", out=psi.clone(), use_guess=True)
    assert st2.inner_iters == 0
    assert rel(o.hsys(psi2.cpu().numpy()), phi) <= 1e-10
    z = torch.zeros_like(x)
    psi0, st0 = s.solve(z, tol=1e-10)
    assert float(psi0.abs().max()) == 0.0
    s.close()


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[5], CASES[6]], ids=[IDS[0], IDS[2], IDS[5], IDS[6]])
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_solve_dense_scheme(env, case, inner):
    """The dense even-odd scheme (no Cayley form, dense Ls x Ls site block,
    App. B) solves the same EOFA system: the oracle's operator judges the
    answer, which agrees with the Cayley-form solve."""
    torch, s, o = setup(env, case)
    phi = I.gaussian_fermion(case[0], case[1], 1001)
    x = torch.from_numpy(phi).cuda()
    psi_d, st_d = s.solve(x, tol=1e-10, inner=inner, method=1)
    psi_c, st_c = s.solve(x, tol=1e-10, inner=inner)
    assert st_d.status == 0 and st_d.inner_iters > 0
    assert rel(o.hsys(psi_d.cpu().numpy()), phi) <= 1e-10, st_d.as_dict()
    assert rel(psi_d.cpu().numpy(), psi_c.cpu().numpy()) < 1e-8
    print(f"{case[0]} Ls={case[1]} {inner}: dense {st_d.inner_iters} iterations, Cayley {st_c.inner_iters}")
    s.close()


def test_dense_scheme_rejects_16bit(env):
    torch, s, o = setup(env, CASES[0])
    from paper_1706_05843_gb300 import binding as B
    x = torch.from_numpy(I.gaussian_fermion(CASES[0][0], CASES[0][1], 1001)).cuda()
    with pytest.raises(B.EofaError) as ei:
        s.solve(x, tol=1e-10, inner="f16", method=1)
    assert ei.value.status == 2
    s.close()


def test_hop_timing_stats(env):
    """Both timing modes report hop launches, time and algorithmic bytes: the
    graph path a sample of four launches per inner solve, kernel timing every
    inner-solver hop launch; the solutions agree."""
    torch, s, o = setup(env, CASES[0])
    phi = torch.from_numpy(I.gaussian_fermion(CASES[0][0], CASES[0][1], 1001)).cuda()
    from paper_1706_05843_gb300 import binding as B
    psi_g, st_g = s.solve(phi, tol=1e-10, inner="f32")
    psi_t, st_t = s.solve(phi, tol=1e-10, inner="f32", kernel_timing=True)
    per = B.lib().eofa_hop_bytes(s.ctx, 1, 0) + B.lib().eofa_hop_bytes(s.ctx, 1, 1)
    assert st_g.hop_launches == 4 * st_g.outer_iters and st_g.hop_ms > 0
    assert abs(st_g.hop_bytes - per * 2 * st_g.outer_iters) <= 1e-6 * st_g.hop_bytes
    assert st_t.hop_launches >= 4 * st_t.inner_iters and st_t.hop_ms > 0
    assert rel(psi_g.cpu().numpy(), psi_t.cpu().numpy()) < 1e-8
    s.close()


def test_not_converged_status(env):
    torch, s, o = setup(env, CASES[0])
    from paper_1706_05843_gb300 import binding as B
    phi = I.gaussian_fermion(CASES[0][0], CASES[0][1], 1001)
    psi, st = s.solve(torch.from_numpy(phi).cuda(), tol=1e-10, inner="f64", max_iter=5, check=False)
    assert st.status == 4
    assert st.inner_iters <= 16 + 5
    s.close()


def test_non_su3_gauge_rejected(env):
    torch, B, O = env
    dims = (4, 4, 4, 4)
    U = I.gauge_field(dims, 0.3, 1)
    U[0, 0, 0, 0, 0] *= 1.01
    with pytest.raises(B.EofaError) as e:
        B.Solver(U, dims, 8, **MOB)
    assert e.value.status == 1


BATCH = [((4, 4, 4, 4), 8, 0.5, dict(beta=-1.0, pm=1)),
         ((2, 2, 2, 6), 4, 0.5, dict(beta=0.7, pm=-1, m3=0.3)),
         ((4, 2, 6, 2), 12, 0.7, dict(beta=-1.0, pm=1, m1=0.0362, m3=0.0362)),
         ((2, 4, 2, 4), 16, 0.5, dict(beta=-1.0, pm=-1))]


@pytest.mark.parametrize("inner", ["f32", "f16", "f64"])
def test_solve_batched_uneven_lattices(env, inner):
    """One batched call over systems of different lattices and Ls; every
    solution is judged by the oracle's operator and matches the one-by-one
    solve."""
    torch, B, O = env
    solvers, oracles, rhs = [], [], []
    for i, case in enumerate(BATCH):
        torch_, s, o = setup(env, case, seed=10 + i)
        solvers.append(s)
        oracles.append(o)
        rhs.append(torch.from_numpy(I.gaussian_fermion(case[0], case[1], 2000 + i)).cuda())
    sols = [torch.empty_like(r) for r in rhs]
    opts = B.make_opts(tol=1e-10, inner=inner)
    stats = B.eofa_solve_batched([s.ctx for s in solvers], rhs, sols, opts)
    for i, (s, o) in enumerate(zip(solvers, oracles)):
        phi = rhs[i].cpu().numpy()
        psi = sols[i].cpu().numpy()
        assert rel(o.hsys(psi), phi) <= 1e-10, (i, stats[i].as_dict())
        assert stats[i].status == 0
        one, st1 = s.solve(rhs[i], tol=1e-10, inner=inner)
        assert rel(psi, one.cpu().numpy()) < 1e-8
    for s in solvers:
        s.close()


def test_equal_shift_masses_collapse_to_the_plain_system(env):
    """m3 = m2 zeroes k(m2, m3): the library's H + beta Delta P with beta = -1
    equals its beta = 0 operator, the oracle's H(m1), and its solve is judged
    by the plain system (the Sherman-Morrison factors degenerate to 1)."""
    torch, B, O = env
    dims, Ls = (4, 4, 4, 4), 8
    U = I.gauge_field(dims, 0.3, 1)
    act = dict(MOB, beta=-1.0, pm=1, m2=0.5, m3=0.5)
    s1 = B.Solver(U, dims, Ls, **act)
    s0 = B.Solver(U, dims, Ls, **dict(act, beta=0.0))
    o0 = O.Oracle(O.Action(dims=dims, Ls=Ls, **dict(act, beta=0.0)), U)
    psi = I.gaussian_fermion(dims, Ls, 7)
    x = torch.from_numpy(psi).cuda()
    h1 = s1.apply_h(x).cpu().numpy()
    assert rel(h1, s0.apply_h(x).cpu().numpy()) < 1e-14
    assert rel(h1, o0.hsys(psi)) < 1e-12
    phi = I.gaussian_fermion(dims, Ls, 1001)
    for s in (s1, s0):
        out, st = s.solve(torch.from_numpy(phi).cuda(), tol=1e-10, inner="f32")
        assert rel(o0.hsys(out.cpu().numpy()), phi) <= 1e-10
    s1.close()
    s0.close()


def test_solve_batched_rejects_duplicate_context(env):
    torch, B, O = env
    torch_, s, o = setup(env, CASES[0])
    r = torch.from_numpy(I.gaussian_fermion(CASES[0][0], CASES[0][1], 1)).cuda()
    with pytest.raises(B.EofaError) as e:
        B.eofa_solve_batched([s.ctx, s.ctx], [r, r.clone()], [torch.empty_like(r), torch.empty_like(r)],
                             B.make_opts(tol=1e-10))
    assert e.value.status == 1
    s.close()
