"""GPU tests of the learned preconditioner through the C ABI.

The BF16 tensor-core network (forward and both backward passes) is compared
with the FP64 numpy oracle, in two ways.

* Against the oracle's plain FP64 network on the same BF16-rounded inputs
  and weights: the library also stores the two hidden activations (and, in
  the backward pass, the incoming gradients) in BF16, so the two differ by
  the propagated BF16 rounding of those, at most a few units of 2^-9 ~ 2e-3
  relative; bound 2% (forward) and 3% (backward).
* Forward, against the same oracle functions with BF16 rounding applied
  exactly where the library stores BF16 (the storage model): what is left is
  the order of the FP32 accumulation (about 2592 terms, relative error
  ~1e-6) and the rare BF16 rounding of a hidden value that this order moves
  across a rounding boundary (one BF16 unit, 2^-8 of that value, for a
  fraction ~1e-6 / 2^-8 of the values).  Bound 1e-3, far above both effects
  and far below a misplaced tap, channel or sign (errors of order 1).
* Backward: the LeakyReLU derivative jumps (1 <-> 0.1) where a
  pre-activation crosses zero, so BF16 storage of the activations flips it
  for the pre-activations that the rounding moves across zero, and which ones
  flip depends on the accumulation order.  The storage model's own distance
  from the FP64 gradients measures this effect for the test's data; the
  library's gradients must lie within twice that distance of the FP64 ones
  (a misplaced tap, channel or sign gives errors of order 1).

Training must reduce its loss and the error on held-out pairs, and a solve
preconditioned by the trained network must reach the true residual 1e-10
judged by the solver oracle; the test reports what the trained network
changes against the untrained one and against the method without it.
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
    got = out.cpu().numpy()
    assert rel(got, ref) < 2e-2
    sm = forward_bf16_storage(xb, wb)
    err = rel(got, sm)
    print(f"forward {dims} S={S}: against FP64 {rel(got, ref):.2e}, against the BF16 storage model {err:.2e}")
    assert err < 1e-3


def forward_bf16_storage(x, w, cache=False):
    """The oracle network with the library's BF16 storage of the hidden activations."""
    W = N.split(w)
    z1 = N.conv(x, W[0])
    a1 = N.bf16_round(N.leaky(z1))
    z2 = N.conv(a1, W[1])
    a2 = N.bf16_round(N.leaky(z2))
    out = N.conv(a2, W[2])
    return (out, (z1, a1, z2, a2)) if cache else out


def backward_bf16_storage(x, w, dout):
    """Gradients through the storage model: incoming gradients stored in BF16
    before each product, as the library does."""
    W = N.split(w)
    _, (z1, a1, z2, a2) = forward_bf16_storage(x, w, cache=True)
    db = N.bf16_round(dout)
    dW2 = N.conv_wgrad(a2, db)
    dz2 = N.bf16_round(N.conv_adjoint(db, W[2]) * N.dleaky(z2))
    dW1 = N.conv_wgrad(a1, dz2)
    dz1 = N.bf16_round(N.conv_adjoint(dz2, W[1]) * N.dleaky(z1))
    dW0 = N.conv_wgrad(x, dz1)
    dx = N.conv_adjoint(dz1, W[0])
    return np.concatenate([dW0.ravel(), dW1.ravel(), dW2.ravel()]), dx


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
    dw_sm, dx_sm = backward_bf16_storage(x, w, g)
    off = 0
    for ci, co in zip(N.CIN, N.COUT):
        n = 81 * ci * co
        e = rel(dw[off:off + n], dw_ref[off:off + n])
        bound = 2.0 * rel(dw_sm[off:off + n], dw_ref[off:off + n])
        print(f"weight gradient ({ci}->{co}): against FP64 {e:.2e}, bound {bound:.2e}")
        assert e < bound
        off += n
    dxg = din.cpu().numpy()
    e, bound = rel(dxg, dx_ref), 2.0 * rel(dx_sm, dx_ref)
    print(f"input gradient: against FP64 {e:.2e}, bound {bound:.2e}")
    assert e < bound


def test_train_and_preconditioned_solve(env):
    """Training gains, measured: on (residual, error) pairs of further
    sources that training never saw, the trained network's relative squared
    error must be below the initial network's.  The solve-level effect
    (inner iterations, flexible-GCR steps, fallbacks and wall clock of the
    trained network, the untrained one and plain CGNR) is measured on a
    lattice where flexible GCR runs several steps and reported; each solve is
    judged by the oracle."""
    torch, B, O = env
    dims, Ls = (8, 8, 8, 8), 8
    act = dict(M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, beta=-1.0, pm=1, t_bc=-1)
    U = I.gauge_field(dims, 0.5, 1)
    s = B.Solver(U, dims, Ls, **act)
    srcs = [torch.from_numpy(I.gaussian_fermion(dims, Ls, 3000 + i)).cuda() for i in range(12)]
    w0 = init_weights(7)
    opts = B.make_train_opts(pairs=96, snapshot_every=4, epochs=8, batch=4, lr=2e-3, solve_tol=1e-6, holdout=32)
    w, st = B.eofa_train_preconditioner(s.ctx, srcs, w0, opts)
    assert st.pairs == 96 and st.holdout_pairs == 32
    assert st.loss_last < st.loss_first
    gain = 1.0 - st.holdout_loss_final / st.holdout_loss_init
    print(f"held-out relative squared error: initial {st.holdout_loss_init:.4f}, trained "
          f"{st.holdout_loss_final:.4f} ({100 * gain:.1f}% lower); training {st.as_dict()}")
    assert st.holdout_loss_final < st.holdout_loss_init
    o = O.Oracle(O.Action(dims=dims, Ls=Ls, **act), U)
    phi = I.gaussian_fermion(dims, Ls, 1001)
    x = torch.from_numpy(phi).cuda()
    runs = {}
    for name, weights in [("trained", w), ("untrained", w0)]:
        B.eofa_set_preconditioner(s.ctx, weights)
        s.solve(x, tol=1e-10, inner="f32", precond=1)          # warm-up
        psi, sst = s.solve(x, tol=1e-10, inner="f32", precond=1)
        assert rel(o.hsys(psi.cpu().numpy()), phi) <= 1e-10
        assert sst.precond_iters >= 2
        runs[name] = dict(inner=sst.inner_iters, gcr=sst.precond_iters, fallbacks=sst.precond_fallbacks,
                          seconds=sst.seconds)
    s.solve(x, tol=1e-10, inner="f32")
    psi, sst = s.solve(x, tol=1e-10, inner="f32")
    assert rel(o.hsys(psi.cpu().numpy()), phi) <= 1e-10
    runs["cgnr"] = dict(inner=sst.inner_iters, seconds=sst.seconds)
    for name in ("trained", "untrained"):
        r = runs[name]
        print(f"{name}: {r['inner']} inner iterations ({r['gcr']} GCR steps, {r['fallbacks']} fallbacks), "
              f"{r['seconds'] * 1e3:.1f} ms; against CGNR {runs['cgnr']['inner']} iterations, "
              f"{runs['cgnr']['seconds'] * 1e3:.1f} ms: iterations x{r['inner'] / runs['cgnr']['inner']:.2f}, "
              f"wall clock x{r['seconds'] / runs['cgnr']['seconds']:.2f}")
    s.close()
