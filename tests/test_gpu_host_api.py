"""GPU tests of the host-buffer solve, the device diagnostics and the FMA
throughput probe.

eofa_solve_host takes a host right-hand side and writes the solution to host
memory inside the call (page-locked buffers read in place and filled by the
copy engine while the true residual is computed, pageable ones staged, in
every mix); the answer must be the device solve's (the solver is
deterministic, so bit for bit) and is judged by the oracle.  A zero
right-hand side gives an exactly zero solution; a non-finite one leaves sol
untouched.  eofa_dot must
equal numpy's FP64 inner product (and repeat bit for bit), eofa_force_norms
the Sec. VI definition evaluated on the host.  The FMA probe must report a
positive throughput with FP32 above FP64.
"""
import numpy as np
import pytest

from paper_1706_05843_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ACT = dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, beta=-1.0, pm=1, t_bc=-1)


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


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_solve_host_matches_device_solve(env, inner):
    torch, B, O = env
    dims, Ls = (4, 4, 4, 4), 8
    U = I.gauge_field(dims, 0.3, 1)
    s = B.Solver(U, dims, Ls, **ACT)
    o = O.Oracle(O.Action(dims=dims, Ls=Ls, **ACT), U)
    phi = I.gaussian_fermion(dims, Ls, 1001)
    dev, st_d = s.solve(torch.from_numpy(phi).cuda(), tol=1e-10, inner=inner)
    host_rhs = torch.from_numpy(phi).pin_memory()
    host_sol = torch.empty_like(host_rhs).pin_memory()
    _, st_h = s.solve_host(host_rhs, host_sol, tol=1e-10, inner=inner)
    assert st_h.status == 0 and st_h.inner_iters == st_d.inner_iters
    assert np.array_equal(host_sol.numpy(), dev.cpu().numpy())
    assert np.linalg.norm(phi - o.hsys(host_sol.numpy())) / np.linalg.norm(phi) <= 1e-10
    # pageable buffers (the staging path) give the same answer
    out_p = np.empty_like(phi)
    _, st_p = s.solve_host(phi, out_p, tol=1e-10, inner=inner)
    assert st_p.status == 0 and np.array_equal(out_p, host_sol.numpy())
    # pageable numpy buffers and the initial guess: restarting from the
    # converged answer needs no inner iteration
    out = host_sol.numpy().copy()
    _, st_g = s.solve_host(phi, out, tol=1e-10, inner=inner, use_guess=True)
    assert st_g.status == 0 and st_g.inner_iters == 0
    # the same restart from page-locked buffers (the guess read in place)
    _, st_gp = s.solve_host(host_rhs, host_sol, tol=1e-10, inner=inner, use_guess=True)
    assert st_gp.status == 0 and st_gp.inner_iters == 0
    # mixed: page-locked rhs with a pageable sol, and the reverse
    out_m = np.empty_like(phi)
    s.solve_host(host_rhs, out_m, tol=1e-10, inner=inner)
    sol_m = torch.zeros_like(host_rhs).pin_memory()
    s.solve_host(phi, sol_m, tol=1e-10, inner=inner)
    assert np.array_equal(out_m, dev.cpu().numpy()) and np.array_equal(sol_m.numpy(), dev.cpu().numpy())
    s.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_solve_host_zero_and_nonfinite_rhs(env, pinned):
    torch, B, O = env
    dims, Ls = (4, 4, 4, 4), 8
    s = B.Solver(I.gauge_field(dims, 0.3, 1), dims, Ls, **ACT)

    def buf(a):
        t = torch.from_numpy(a)
        return t.pin_memory() if pinned else t

    zero = buf(np.zeros((4, 4, 4, 4, Ls, 4, 3), dtype=np.complex128))
    out = buf(np.full((4, 4, 4, 4, Ls, 4, 3), 7.0 + 1j))
    _, st = s.solve_host(zero, out, tol=1e-10, inner="f32")
    assert st.status == 0 and st.inner_iters == 0
    assert torch.count_nonzero(out).item() == 0
    bad = I.gaussian_fermion(dims, Ls, 5)
    bad.reshape(-1)[123] = np.nan
    out = buf(np.full((4, 4, 4, 4, Ls, 4, 3), 7.0 + 1j))
    _, st = s.solve_host(buf(bad), out, tol=1e-10, inner="f32", check=False)
    assert st.status == 5  # EOFA_ERR_NONFINITE
    assert bool((out.numpy() == 7.0 + 1j).all())  # untouched
    s.close()


def test_solve_host_rejects_device_arguments(env):
    torch, B, O = env
    dims, Ls = (4, 4, 4, 4), 8
    s = B.Solver(I.gauge_field(dims, 0.3, 1), dims, Ls, **ACT)
    x = torch.zeros((4, 4, 4, 4, Ls, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(TypeError):
        s.solve_host(x, x.cpu())
    s.close()


def test_measure_fma(env):
    torch, B, O = env
    f64 = B.eofa_measure_fma("f64", reps=3)
    f32 = B.eofa_measure_fma("f32", reps=3)
    print(f"FMA throughput: FP64 {f64:.2f} TFLOP/s, FP32 {f32:.2f} TFLOP/s")
    assert 0.0 < f64 < f32


def test_dot_matches_numpy(env):
    torch, B, O = env
    dims, Ls = (4, 4, 4, 4), 8
    s = B.Solver(I.gauge_field(dims, 0.3, 1), dims, Ls, **ACT)
    a = I.gaussian_fermion(dims, Ls, 21)
    b = I.gaussian_fermion(dims, Ls, 22)
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    ref = np.vdot(a.ravel(), b.ravel())
    got = s.dot(da, db)
    assert abs(got - ref) <= 1e-13 * abs(ref)
    assert s.dot(da, db) == got                       # fixed summation order
    assert abs(s.dot(da, da).real - np.vdot(a.ravel(), a.ravel()).real) <= 1e-13 * np.vdot(a.ravel(), a.ravel()).real
    s.close()


def test_force_norms_match_definition(env):
    torch, B, O = env
    from paper_1706_05843_gb300 import forces
    dims, Ls = (4, 4, 4, 4), 8
    s = B.Solver(I.gauge_field(dims, 0.3, 1), dims, Ls, **ACT)
    phi = torch.from_numpy(I.heatbath_noise(dims, 31)).cuda()
    f, _ = s.force(phi, ACT["m1"], ACT["m2"], tol=1e-10, inner="f32")
    rms, mx = s.force_norms(f)
    hrms, hmx = forces.force_norms(f.cpu().numpy())
    assert rms == pytest.approx(hrms, rel=1e-13)
    assert mx == pytest.approx(hmx, rel=1e-13)
    s.close()


def test_tile_sweep_reports_the_tuner(env):
    """eofa_tile_time gives the autotuner's per-variant launch times (the
    dslash sweep over tile shapes); the variant it chose is the fastest."""
    torch, B, O = env
    dims, Ls = (4, 4, 4, 4), 8
    s = B.Solver(I.gauge_field(dims, 0.3, 1), dims, Ls, **ACT)
    lib = B.lib()
    assert lib.eofa_tile_time(s.ctx, 1, 0, 0) == 0.0          # no FP32 solve yet
    s.solve(torch.from_numpy(I.gaussian_fermion(dims, Ls, 1001)).cuda(), tol=1e-10, inner="f32")
    for prec, nvar in [(1, 4), (0, 2)]:                         # FP32 inner, FP64 outer kinds
        for k in range(4):
            t = [lib.eofa_tile_time(s.ctx, prec, k, v) for v in range(4)]
            timed = [x for x in t if x > 0]
            assert 2 <= len(timed) <= nvar, (prec, k, t)
            assert t[lib.eofa_tile_variant(s.ctx, prec, k)] == min(timed)
    assert lib.eofa_tile_time(s.ctx, 1, 0, 4) == -1.0
    assert lib.eofa_tile_time(s.ctx, 0, 0, 2) == 0.0             # FP64 has two variants
    s.close()


def test_solver_rejects_fields_of_another_size(env):
    """The C ABI takes plain pointers; the Solver checks every field's size
    before a call, so a field of another lattice never reaches a kernel."""
    torch, B, O = env
    dims, Ls = (4, 4, 4, 4), 8
    U = I.gauge_field(dims, 0.3, 1)
    with pytest.raises(ValueError):
        B.Solver(U[:2], dims, Ls, **ACT)
    s = B.Solver(U, dims, Ls, **ACT)
    small = torch.zeros((2, 2, 2, 2, Ls, 4, 3), dtype=torch.complex128, device="cuda")
    for call in (lambda: s.apply(small), lambda: s.apply_h(small), lambda: s.solve(small),
                 lambda: s.solve_host(small.cpu().numpy(), small.cpu().numpy()),
                 lambda: s.force_norms(small), lambda: s.heatbath(small, 0.04, 1.0, None)):
        with pytest.raises(ValueError):
            call()
    phi = torch.from_numpy(I.gaussian_fermion(dims, Ls, 1001)).cuda()
    with pytest.raises(ValueError):
        s.solve(phi, out=small)
    _, st = s.solve(phi, tol=1e-10, inner="f32")      # the context is unharmed
    assert st.status == 0
    s.close()
