"""GPU tests of the batched solve, whose FP64 defect correction runs on the
device: one graph launch per call holds every system's first residual,
inner CGNR chunks, outer steps (correction, FP64 residual, decision) and
inner restarts.

* The device loop takes the decisions of the host-driven one (same inner
  targets, caps and order of checks) on the same deterministic kernels, so
  each system's outer steps and inner iterations equal those of its
  one-by-one solve, and the solutions agree to rounding.  Every solution is
  judged by the oracle's operator.
* The graph is kept for later calls on the same contexts: a repeated call
  gives bit-identical solutions; after eofa_set_system the kept graph is
  dropped and the batch solves the new system (judged by a new oracle).
* Edge cases: a zero right-hand side (solution exactly zero, no outer step)
  beside systems that start from an initial guess, the iteration cap
  (EOFA_ERR_NOT_CONVERGED with the best solution written), and a deadline
  (EOFA_ERR_TIMEOUT from the device decision), after which the same
  contexts solve to 1e-10; a G-parity context (twice the 5D volume, two
  flavours) in one batch with ordinary ones.
"""
import numpy as np
import pytest

from paper_1706_05843_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MOB = dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, t_bc=-1)
BATCH = [((4, 4, 4, 4), 8, 0.5, dict(beta=-1.0, pm=1)),
         ((2, 2, 2, 6), 4, 0.5, dict(beta=0.7, pm=-1, m3=0.3)),
         ((4, 2, 6, 2), 12, 0.7, dict(beta=-1.0, pm=1, m1=0.0362, m3=0.0362)),
         ((2, 4, 2, 4), 16, 0.5, dict(beta=-1.0, pm=-1))]
NOT_CONVERGED, TIMEOUT = 4, 6
CHUNK = 16  # CG iterations per chunk of the device loop


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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_batch(env, cases=BATCH, seed0=10):
    torch, B, O = env
    solvers, oracles, rhs = [], [], []
    for i, (dims, Ls, eps, kw) in enumerate(cases):
        act = dict(MOB)
        act.update(kw)
        U = I.gauge_field(dims, eps, seed0 + i)
        oracles.append(O.Oracle(O.Action(dims=dims, Ls=Ls, **act), U))
        solvers.append(B.Solver(U, dims, Ls, **act))
        rhs.append(torch.from_numpy(I.gaussian_fermion(dims, Ls, 2000 + i)).cuda())
    return solvers, oracles, rhs


def close(solvers):
    for s in solvers:
        s.close()


@pytest.mark.parametrize("inner", ["f32", "f64", "bf16"])
def test_batched_equals_one_by_one(env, inner):
    torch, B, O = env
    solvers, oracles, rhs = make_batch(env)
    sols = [torch.empty_like(r) for r in rhs]
    st = B.eofa_solve_batched([s.ctx for s in solvers], rhs, sols, B.make_opts(tol=1e-10, inner=inner))
    for i, (s, o) in enumerate(zip(solvers, oracles)):
        psi = sols[i].cpu().numpy()
        assert st[i].status == 0
        assert rel(o.hsys(psi), rhs[i].cpu().numpy()) <= 1e-10, st[i].as_dict()
        one, st1 = s.solve(rhs[i], tol=1e-10, inner=inner)
        print(f"system {i}: batched {st[i].outer_iters} outer / {st[i].inner_iters} inner, "
              f"one by one {st1.outer_iters} / {st1.inner_iters}; launches {st[i].kernel_launches}")
        assert (st[i].outer_iters, st[i].inner_iters) == (st1.outer_iters, st1.inner_iters)
        assert rel(psi, one.cpu().numpy()) < 1e-12
        assert st[i].kernel_launches > 0
    close(solvers)


def test_solve_batched_helper_checks_sizes(env):
    """binding.solve_batched: the same solutions as the C-named call, and a
    right-hand side of another lattice is refused before the library."""
    torch, B, O = env
    solvers, oracles, rhs = make_batch(env)
    sols, st = B.solve_batched(solvers, rhs, tol=1e-10, inner="f32")
    ref = [torch.empty_like(r) for r in rhs]
    B.eofa_solve_batched([s.ctx for s in solvers], rhs, ref, B.make_opts(tol=1e-10, inner="f32"))
    for i in range(len(rhs)):
        assert st[i].status == 0 and torch.equal(sols[i], ref[i])
    with pytest.raises(ValueError):
        B.solve_batched(solvers, [rhs[1], rhs[0]] + rhs[2:], tol=1e-10, inner="f32")
    close(solvers)


def test_batched_kept_graph_repeat_and_set_system(env):
    torch, B, O = env
    solvers, oracles, rhs = make_batch(env)
    ctxs = [s.ctx for s in solvers]
    opts = B.make_opts(tol=1e-10, inner="f32")
    a = [torch.empty_like(r) for r in rhs]
    b = [torch.empty_like(r) for r in rhs]
    sa = B.eofa_solve_batched(ctxs, rhs, a, opts)
    sb = B.eofa_solve_batched(ctxs, rhs, b, opts)  # the kept graph
    for i in range(len(rhs)):
        assert torch.equal(a[i], b[i])
        assert sa[i].inner_iters == sb[i].inner_iters
    # a new operator on system 1: the kept graph goes, the new system is solved
    dims, Ls, eps, kw = BATCH[1]
    new = dict(m1=0.1, m2=0.8, m3=0.2, beta=0.5, pm=1)
    solvers[1].set_system(new["m1"], new["m2"], new["m3"], new["beta"], new["pm"])
    act = dict(MOB)
    act.update(kw)
    act.update(new)
    o1 = O.Oracle(O.Action(dims=dims, Ls=Ls, **act), I.gauge_field(dims, eps, 11))
    st = B.eofa_solve_batched(ctxs, rhs, a, opts)
    assert all(x.status == 0 for x in st)
    assert rel(o1.hsys(a[1].cpu().numpy()), rhs[1].cpu().numpy()) <= 1e-10
    for i in (0, 2, 3):
        assert rel(oracles[i].hsys(a[i].cpu().numpy()), rhs[i].cpu().numpy()) <= 1e-10
    close(solvers)


def test_batched_zero_rhs_and_initial_guess(env):
    torch, B, O = env
    solvers, oracles, rhs = make_batch(env)
    rhs[0] = torch.zeros_like(rhs[0])
    exact, _ = solvers[1].solve(rhs[1], tol=1e-10, inner="f32")
    sols = [torch.full_like(rhs[0], 3.0), exact.clone(), torch.zeros_like(rhs[2]),
            torch.from_numpy(I.gaussian_fermion(BATCH[3][0], BATCH[3][1], 77)).cuda()]
    st = B.eofa_solve_batched([s.ctx for s in solvers], rhs, sols,
                              B.make_opts(tol=1e-10, inner="f32", use_guess=True))
    assert st[0].status == 0 and st[0].outer_iters == 0 and st[0].inner_iters == 0
    assert torch.count_nonzero(sols[0]).item() == 0
    for i in (1, 2, 3):
        assert st[i].status == 0
        assert rel(oracles[i].hsys(sols[i].cpu().numpy()), rhs[i].cpu().numpy()) <= 1e-10
    # started from its own solution, system 1 needs at most one short correction
    one, st1 = solvers[2].solve(rhs[2], tol=1e-10, inner="f32")
    assert st[1].outer_iters <= 1
    print("guess at the solution:", st[1].as_dict(), "zero guess:", st[2].as_dict(), "no guess:", st1.as_dict())
    assert st[2].inner_iters == st1.inner_iters  # a zero guess is the unguessed start
    close(solvers)


def test_batched_iteration_cap(env):
    torch, B, O = env
    solvers, oracles, rhs = make_batch(env)
    sols = [torch.empty_like(r) for r in rhs]
    st = B.eofa_solve_batched([s.ctx for s in solvers], rhs, sols,
                              B.make_opts(tol=1e-10, inner="f32", max_iter=20), check=False)
    assert B.lib().eofa_last_error(solvers[0].ctx).decode() == "iteration cap"
    for i in range(len(rhs)):
        assert st[i].status == NOT_CONVERGED
        assert 20 <= st[i].inner_iters < 20 + CHUNK
        psi = sols[i].cpu().numpy()
        assert np.isfinite(psi).all()
        r = rel(oracles[i].hsys(psi), rhs[i].cpu().numpy())
        assert r < 1.0 and abs(r - st[i].true_res) <= 1e-12 + 1e-6 * r
    close(solvers)


def test_batched_deadline(env):
    torch, B, O = env
    cases = [((8, 8, 8, 8), 8, 0.5, dict(beta=-1.0, pm=1)), ((8, 8, 8, 8), 8, 0.5, dict(beta=0.7, pm=-1))]
    solvers, oracles, rhs = make_batch(env, cases)
    ctxs = [s.ctx for s in solvers]
    sols = [torch.empty_like(r) for r in rhs]
    full = B.eofa_solve_batched(ctxs, rhs, sols, B.make_opts(tol=1e-10, inner="f32"))
    st = B.eofa_solve_batched(ctxs, rhs, sols, B.make_opts(tol=1e-10, inner="f32", timeout_ms=2), check=False)
    for i in range(len(rhs)):
        print(f"system {i}: full {full[i].inner_iters} iterations, with a 2 ms deadline {st[i].as_dict()}")
        assert st[i].status == TIMEOUT
        assert st[i].inner_iters < full[i].inner_iters
        assert np.isfinite(sols[i].cpu().numpy()).all()
    st = B.eofa_solve_batched(ctxs, rhs, sols, B.make_opts(tol=1e-10, inner="f32"))
    for i in range(len(rhs)):
        assert st[i].status == 0
        assert rel(oracles[i].hsys(sols[i].cpu().numpy()), rhs[i].cpu().numpy()) <= 1e-10
    close(solvers)


def test_batched_with_gparity_context(env):
    """A G-parity context (two flavours stacked along t, flavour-changing
    boundary hops) in one batch with an ordinary one; each judged by its own
    oracle and equal to its one-by-one solve."""
    torch, B, O = env
    from oracle.gparity import GOracle
    dims, Ls, gm = (4, 4, 2, 4), 8, 3
    act = dict(MOB, beta=-1.0, pm=1)
    U = I.gauge_field(dims, 0.5, 21)
    sg = B.Solver(U, dims, Ls, gparity=gm, **act)
    og = GOracle(O.Action(dims=dims, Ls=Ls, **act), U, gm)
    phig = np.stack([I.gaussian_fermion(dims, Ls, 3000), I.gaussian_fermion(dims, Ls, 3001)])
    solvers, oracles, rhs = make_batch(env, BATCH[:2])
    solvers.insert(0, sg)
    rhs.insert(0, torch.from_numpy(phig).cuda())
    sols = [torch.empty_like(r) for r in rhs]
    st = B.eofa_solve_batched([s.ctx for s in solvers], rhs, sols, B.make_opts(tol=1e-10, inner="f32"))
    assert all(x.status == 0 for x in st)
    assert rel(og.hsys(sols[0].cpu().numpy()), phig) <= 1e-10
    for i in (1, 2):
        assert rel(oracles[i - 1].hsys(sols[i].cpu().numpy()), rhs[i].cpu().numpy()) <= 1e-10
    one, st1 = sg.solve(rhs[0], tol=1e-10, inner="f32")
    assert (st[0].outer_iters, st[0].inner_iters) == (st1.outer_iters, st1.inner_iters)
    assert rel(sols[0].cpu().numpy(), one.cpu().numpy()) < 1e-12
    close(solvers)


def test_batched_non_finite_rhs(env):
    """A NaN in one system's right-hand side stops the call with
    EOFA_ERR_NONFINITE at the source-norm check, before the device loop; the
    same contexts then solve a clean batch to 1e-10."""
    torch, B, O = env
    solvers, oracles, rhs = make_batch(env)
    ctxs = [s.ctx for s in solvers]
    bad = [r.clone() for r in rhs]
    bad[2].view(-1)[17] = float("nan")
    sols = [torch.empty_like(r) for r in rhs]
    with pytest.raises(B.EofaError) as e:
        B.eofa_solve_batched(ctxs, bad, sols, B.make_opts(tol=1e-10, inner="f32"))
    assert e.value.status == 5
    assert "system 2" in str(e.value)
    st = B.eofa_solve_batched(ctxs, rhs, sols, B.make_opts(tol=1e-10, inner="f32"))
    for i in range(len(rhs)):
        assert st[i].status == 0
        assert rel(oracles[i].hsys(sols[i].cpu().numpy()), rhs[i].cpu().numpy()) <= 1e-10
    close(solvers)


def test_batched_more_systems_than_one_graph(env):
    """34 systems: the call runs them as graphs of at most 32; all are judged
    by the oracle, and a failure in the second graph is reported on the
    first context with its system index."""
    torch, B, O = env
    dims, Ls = (2, 2, 2, 6), 4
    act = dict(MOB, beta=-1.0, pm=1)
    U = I.gauge_field(dims, 0.5, 5)
    o = O.Oracle(O.Action(dims=dims, Ls=Ls, **act), U)
    solvers = [B.Solver(U, dims, Ls, **act) for _ in range(34)]
    ctxs = [s.ctx for s in solvers]
    rhs = [torch.from_numpy(I.gaussian_fermion(dims, Ls, 4000 + i)).cuda() for i in range(34)]
    sols = [torch.empty_like(r) for r in rhs]
    st = B.eofa_solve_batched(ctxs, rhs, sols, B.make_opts(tol=1e-10, inner="f32"))
    for i in range(34):
        assert st[i].status == 0
        assert rel(o.hsys(sols[i].cpu().numpy()), rhs[i].cpu().numpy()) <= 1e-10
    bad = [r.clone() for r in rhs]
    bad[33].view(-1)[3] = float("inf")
    with pytest.raises(B.EofaError) as e:
        B.eofa_solve_batched(ctxs, bad, sols, B.make_opts(tol=1e-10, inner="f32"))
    assert e.value.status == 5 and "system 33" in str(e.value)
    close(solvers)
