"""GPU tests of the solver's failure paths, in forms that cannot fault or
hang the GPU: every wait in the device-driven CG loop is bounded, so a
deadline that runs out ends the loop through its condition kernel and the
solve returns a status.

* timeout: the benchmark workload (16^3x32, Ls=16, FP32 inner) with a
  deadline far below the solve time.  With 40 ms the deadline falls inside
  the first inner solve, so the device-side check (%globaltimer in the loop's
  condition kernel) is the one that stops it: the solve returns
  EOFA_ERR_TIMEOUT after a number of inner iterations between one CG chunk
  and the full count.  With 1 ms the host check before the inner loop may
  fire first; either way the status is EOFA_ERR_TIMEOUT.
* non-finite right-hand side: one NaN in phi gives EOFA_ERR_NONFINITE (the
  norm of the source is checked before any iteration), and an Inf in the
  middle of the field does too.
* after each failure the same context solves a valid system to 1e-10.
"""
import numpy as np
import pytest

from paper_1706_05843_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ACT = dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, beta=-1.0, pm=1, t_bc=-1)
TIMEOUT, NONFINITE = 6, 5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_05843_gb300 import build
    build.build()
    from paper_1706_05843_gb300 import binding as B
    B.lib()
    return torch, B


@pytest.fixture(scope="module")
def bench_solver(env):
    torch, B = env
    dims, Ls = (16, 16, 16, 32), 16
    U = I.gauge_field(dims, 0.5, 1)
    s = B.Solver(U, dims, Ls, **ACT)
    rhs = torch.from_numpy(I.gaussian_fermion(dims, Ls, 1001)).cuda()
    _, st = s.solve(rhs, tol=1e-10, inner="f32")   # tunes and captures the CG graph
    full = st.inner_iters
    yield torch, B, s, rhs, full
    s.close()


def test_device_deadline_stops_the_loop(bench_solver):
    torch, B, s, rhs, full = bench_solver
    _, st = s.solve(rhs, tol=1e-10, inner="f32", timeout_ms=40, check=False)
    assert st.status == TIMEOUT
    # stopped inside the device loop: at least the first CG chunk ran, far
    # fewer than the full solve's iterations
    assert 16 <= st.inner_iters < full
    assert B.lib().eofa_last_error(s.ctx).decode().startswith("solve exceeded")
    _, st = s.solve(rhs, tol=1e-10, inner="f32")
    assert st.status == 0 and st.true_res <= 1e-10


def test_tiny_timeout(bench_solver):
    torch, B, s, rhs, full = bench_solver
    _, st = s.solve(rhs, tol=1e-10, inner="f32", timeout_ms=1, check=False)
    assert st.status == TIMEOUT
    assert st.inner_iters < full


@pytest.mark.parametrize("bad", ["nan", "inf"])
def test_non_finite_rhs(env, bad):
    torch, B = env
    dims, Ls = (4, 4, 4, 4), 8
    U = I.gauge_field(dims, 0.3, 1)
    s = B.Solver(U, dims, Ls, **ACT)
    phi = I.gaussian_fermion(dims, Ls, 1001)
    x = phi.copy()
    if bad == "nan":
        x[0, 0, 0, 0, 0, 0, 0] = np.nan
    else:
        x[2, 1, 3, 1, 5, 2, 1] = complex(np.inf, 0.0)
    _, st = s.solve(torch.from_numpy(x).cuda(), tol=1e-10, inner="f32", check=False)
    assert st.status == NONFINITE
    with pytest.raises(B.EofaError) as e:
        s.solve(torch.from_numpy(x).cuda(), tol=1e-10, inner="f32")
    assert e.value.status == NONFINITE
    _, st = s.solve(torch.from_numpy(phi).cuda(), tol=1e-10, inner="f32")
    assert st.status == 0 and st.true_res <= 1e-10
    s.close()
