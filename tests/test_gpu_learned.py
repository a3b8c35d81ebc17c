"""GPU tests of the learned preconditioner through the C ABI.

The BF16 tensor-core network (forward and both backward passes) is compared
with the FP64 numpy oracle evaluated on the same BF16-rounded inputs and
weights; the remaining difference comes from BF16 storage of the two hidden
activations and from the order of FP32 accumulation (measured ~0.5%, bound
2%).  Training must reduce its loss, and a solve preconditioned by the
trained network must reach the true residual 1e-10 judged by the solver
oracle; the test prints what the trained network gains over the untrained
one and over the method without it.
"""
import numpy as np
import pytest

from oracle import net as N
from paper_1706_05843_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_05843_gb300 import build
    build.build()
    from paper_1706_05843_gb300 import binding as B
    B.lib()
    import oracle
    oracle.build()
    return torch, B, oracle


def init_weights(seed, scale=None):
    """He-style initial weights (the random draw belongs to the caller)."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in zip(N.CIN, N.COUT):
        s = scale if scale is not None else np.sqrt(2.0 / (81 * ci))
        parts.append(rng.standard_normal(81 * co * ci) * s)
    return np.concatenate(parts).astype(np.float32)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dims,S", [((4, 4, 4, 4), 3), ((6, 2, 4, 2), 2)])
def test_net_forward_matches_oracle(env, dims, S):
    torch, B, O = env
    X, Y, Z, T = dims
    w = init_weights(1)
    x = np.random.default_rng(2).standard_normal((S, T, Z, Y, X, 24))
    xb, wb = N.bf16_round(x), N.bf16_round(w)
    ref = N.forward(xb, wb)
    xt = torch.from_numpy(xb.astype(np.float32)).cuda()
    out = torch.empty_like(xt)
    B.eofa_net_forward(wb.astype(np.float32), dims, xt, out)
    assert rel(out.cpu().numpy(), ref) < 2e-2


def test_net_backward_matches_oracle(env):
    torch, B, O = env
    dims, S = (4, 4, 2, 4), 2
    X, Y, Z, T = dims
    w = N.bf16_round(init_weights(3))
    x = N.bf16_round(np.random.default_rng(4).standard_normal((S, T, Z, Y, X, 24)))
    g = N.bf16_round(np.random.default_rng(5).standard_normal((S, T, Z, Y, X, 24)))
    dw_ref, dx_ref = N.backward(x, w, g)
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    gt = torch.from_numpy(g.astype(np.float32)).cuda()
    din = torch.empty_like(xt)
    dw = B.eofa_net_backward(w.astype(np.float32), dims, xt, gt, din)
    off = 0
    for ci, co in zip(N.CIN, N.COUT):
        n = 81 * ci * co
        assert rel(dw[off:off + n], dw_ref[off:off + n]) < 3e-2
        off += n
    assert rel(din.cpu().numpy(), dx_ref) < 3e-2


def test_train_and_preconditioned_solve(env):
    torch, B, O = env
    dims, Ls = (4, 4, 4, 4), 8
    act = dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, beta=-1.0, pm=1, t_bc=-1)
    U = I.gauge_field(dims, 0.5, 1)
    s = B.Solver(U, dims, Ls, **act)
    srcs = [torch.from_numpy(I.gaussian_fermion(dims, Ls, 3000 + i)).cuda() for i in range(6)]
    w0 = init_weights(7)
    opts = B.make_train_opts(pairs=48, snapshot_every=4, epochs=6, batch=4, lr=2e-3, solve_tol=1e-6)
    w, st = B.eofa_train_preconditioner(s.ctx, srcs, w0, opts)
    assert st.pairs == 48 and st.steps == 72
    assert st.loss_last < st.loss_first
    o = O.Oracle(O.Action(dims=dims, Ls=Ls, **act), U)
    phi = I.gaussian_fermion(dims, Ls, 1001)
    x = torch.from_numpy(phi).cuda()
    iters = {}
    for name, weights in [("trained", w), ("untrained", w0)]:
        B.eofa_set_preconditioner(s.ctx, weights)
        psi, sst = s.solve(x, tol=1e-10, inner="f32", precond=1)
        assert rel(o.hsys(psi.cpu().numpy()), phi) <= 1e-10
        iters[name] = (sst.inner_iters, sst.precond_iters, sst.precond_fallbacks, sst.seconds)
        assert sst.precond_iters >= 1
    psi, sst = s.solve(x, tol=1e-10, inner="f32")
    iters["cgnr"] = (sst.inner_iters, sst.seconds)
    print("inner iterations / seconds:", iters, "training:", st.as_dict())
    s.close()
