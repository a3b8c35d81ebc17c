"""GPU test of eofa_apply_noalloc, the entry point for callers that cannot
call cudaMalloc (a framework that owns all device memory through its own
pool, or a loop that cannot afford cudaMalloc's implicit synchronisation).

It must give the same K in as eofa_apply, on two calls in a row (the static
work space keeps the previous call's contents, so the second call checks
that nothing stale leaks through), agree with the FP64 CPU oracle's K,
reject lattices larger than its static work space under either limit,
reject non-SU(3) links and then work again on the next valid call (the
check flag is cleared every call), and refuse a capturing stream.  The file
is named to be collected last.
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
    from paper_1706_05843_gb300 import binding as B
    B.lib()
    return torch, B


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("dims,Ls,kw", [((4, 4, 4, 4), 8, {}),
                                        ((8, 8, 8, 8), 8, dict(pm=-1, beta=0.7, m3=0.3)),
                                        ((6, 2, 2, 2), 12, {})])
def test_noalloc_matches_apply_twice(env, dims, Ls, kw):
    torch, B = env
    act = dict(ACT)
    act.update(kw)
    U = torch.from_numpy(I.gauge_field(dims, 0.5, 3)).cuda()
    s = B.Solver(U, dims, Ls, **act)
    p = B.make_params(dims, Ls, **act)
    for seed in (11, 12):
        x = torch.from_numpy(I.gaussian_fermion(dims, Ls, seed)).cuda()
        ref = s.apply(x)
        out = torch.full_like(x, float("nan"))
        B.eofa_apply_noalloc(p, U, x, out)
        torch.cuda.synchronize()
        assert rel(out, ref) <= 1e-12
    s.close()


def test_noalloc_rejects_large_lattice(env):
    torch, B = env
    dims, Ls = (8, 8, 8, 16), 8          # 8192 sites > 4096
    p = B.make_params(dims, Ls, **ACT)
    U = torch.zeros((16, 8, 8, 8, 4, 3, 3), dtype=torch.complex128, device="cuda")
    x = torch.zeros((16, 8, 8, 8, Ls, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.EofaError) as e:
        B.eofa_apply_noalloc(p, U, x, torch.empty_like(x))
    assert e.value.status == 2


def test_noalloc_rejects_too_many_5d_sites(env):
    torch, B = env
    dims, Ls = (8, 8, 8, 8), 16          # 4096 4D sites, but 65536 > 32768 5D sites
    p = B.make_params(dims, Ls, **ACT)
    U = torch.zeros((8, 8, 8, 8, 4, 3, 3), dtype=torch.complex128, device="cuda")
    x = torch.zeros((8, 8, 8, 8, Ls, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.EofaError) as e:
        B.eofa_apply_noalloc(p, U, x, torch.empty_like(x))
    assert e.value.status == 2


def test_noalloc_matches_oracle(env, oracle_mod):
    torch, B = env
    dims, Ls = (4, 4, 4, 4), 8
    Un = I.gauge_field(dims, 0.3, 1)
    phi = I.gaussian_fermion(dims, Ls, 1001)
    o = oracle_mod.Oracle(oracle_mod.Action(dims=dims, Ls=Ls, **ACT), Un)
    ref = o.k(phi)
    p = B.make_params(dims, Ls, **ACT)
    out = torch.empty((4, 4, 4, 4, Ls, 4, 3), dtype=torch.complex128, device="cuda")
    B.eofa_apply_noalloc(p, torch.from_numpy(Un).cuda(), torch.from_numpy(phi).cuda(), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12


def test_noalloc_rejects_non_su3_then_recovers(env):
    torch, B = env
    dims, Ls = (4, 4, 4, 4), 8
    p = B.make_params(dims, Ls, **ACT)
    U = torch.from_numpy(I.gauge_field(dims, 0.5, 3)).cuda()
    x = torch.from_numpy(I.gaussian_fermion(dims, Ls, 11)).cuda()
    bad = U.clone()
    bad[1, 2, 3, 0, 2] *= 1.01           # one link no longer unitary
    with pytest.raises(B.EofaError) as e:
        B.eofa_apply_noalloc(p, bad, x, torch.empty_like(x))
    assert e.value.status == 1
    s = B.Solver(U, dims, Ls, **ACT)
    ref = s.apply(x)
    out = torch.full_like(x, float("nan"))
    B.eofa_apply_noalloc(p, U, x, out)   # the flag left set by the rejected call is cleared
    torch.cuda.synchronize()
    assert rel(out, ref) <= 1e-12
    s.close()


def test_noalloc_refuses_capturing_stream(env):
    torch, B = env
    dims, Ls = (4, 4, 4, 4), 8
    p = B.make_params(dims, Ls, **ACT)
    U = torch.from_numpy(I.gauge_field(dims, 0.5, 3)).cuda()
    x = torch.from_numpy(I.gaussian_fermion(dims, Ls, 11)).cuda()
    out = torch.empty_like(x)
    B.eofa_apply_noalloc(p, U, x, out)   # first call on the device: before any capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    status = []
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            status.append(B.lib().eofa_apply_noalloc(B.C.byref(p), B._dptr(U), B._dptr(x), B._dptr(out),
                                                     B._stream(st)))
    assert status == [2]
