"""ctypes binding of libeofa.so (include/eofa.h): argument marshalling only.

Every step of the solve runs inside the CUDA library.  Device memory and
streams come from PyTorch (complex128 CUDA tensors, torch streams).  If the
library is missing this module raises: there is no CPU fallback.

The functions keep the C names (``eofa_create``, ``eofa_apply``, ...); the
``Solver`` class is a small convenience wrapper over them.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libeofa.so")

F64, F32, F16, BF16 = 0, 1, 2, 3
PREC = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16}

STATUS = {0: "EOFA_OK", 1: "EOFA_ERR_ARG", 2: "EOFA_ERR_UNSUPPORTED", 3: "EOFA_ERR_SINGULAR",
          4: "EOFA_ERR_NOT_CONVERGED", 5: "EOFA_ERR_NONFINITE", 6: "EOFA_ERR_TIMEOUT",
          7: "EOFA_ERR_CUDA", 8: "EOFA_ERR_OOM"}


class EofaError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class eofa_params(C.Structure):
    _fields_ = [("dims", C.c_int * 4), ("Ls", C.c_int), ("M5", C.c_double), ("b", C.c_double),
                ("c", C.c_double), ("m1", C.c_double), ("m2", C.c_double), ("m3", C.c_double),
                ("beta", C.c_double), ("pm", C.c_int), ("t_bc", C.c_int)]


class eofa_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("inner", C.c_int),
                ("inner_tol", C.c_double), ("max_outer", C.c_int), ("precond", C.c_int),
                ("use_guess", C.c_int), ("rhs_form", C.c_int), ("kernel_timing", C.c_int),
                ("method", C.c_int), ("timeout_ms", C.c_long)]


class eofa_solve_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iters", C.c_int), ("inner_iters", C.c_int),
                ("hop_launches", C.c_int), ("true_res", C.c_double), ("recur_res", C.c_double),
                ("seconds", C.c_double), ("hop_ms", C.c_double), ("hop_bytes", C.c_double),
                ("kernel_launches", C.c_long), ("precond_iters", C.c_int), ("precond_fallbacks", C.c_int),
                ("precond_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


NET_WEIGHTS = 207360


class eofa_train_opts(C.Structure):
    _fields_ = [("pairs", C.c_int), ("snapshot_every", C.c_int), ("epochs", C.c_int), ("batch", C.c_int),
                ("lr", C.c_double), ("solve_tol", C.c_double), ("holdout", C.c_int)]


class eofa_train_stats(C.Structure):
    _fields_ = [("pairs", C.c_int), ("steps", C.c_int), ("solves", C.c_int), ("loss_first", C.c_double),
                ("loss_last", C.c_double), ("seconds", C.c_double), ("holdout_pairs", C.c_int),
                ("holdout_loss_init", C.c_double), ("holdout_loss_final", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# name -> (argtypes, restype); must match include/eofa.h
_vp = C.c_void_p
_fp = C.POINTER(C.c_float)
_dp = C.POINTER(C.c_double)
SIGNATURES = {
    "eofa_create": ([C.POINTER(eofa_params), _vp, _vp, C.POINTER(_vp)], C.c_int),
    "eofa_create_gparity": ([C.POINTER(eofa_params), _vp, C.c_int, _vp, C.POINTER(_vp)], C.c_int),
    "eofa_apply": ([_vp, _vp, _vp, _vp], C.c_int),
    "eofa_apply_dag": ([_vp, _vp, _vp, _vp], C.c_int),
    "eofa_apply_h": ([_vp, _vp, _vp, _vp], C.c_int),
    "eofa_solve": ([_vp, _vp, _vp, C.POINTER(eofa_solve_opts), C.POINTER(eofa_solve_stats), _vp], C.c_int),
    "eofa_apply_batched": ([C.POINTER(_vp), C.c_int, C.POINTER(_vp), C.POINTER(_vp), C.c_int, _vp], C.c_int),
    "eofa_solve_batched": ([C.POINTER(_vp), C.c_int, C.POINTER(_vp), C.POINTER(_vp),
                            C.POINTER(eofa_solve_opts), C.POINTER(eofa_solve_stats), _vp], C.c_int),
    "eofa_solve_host": ([_vp, _dp, _dp, C.POINTER(eofa_solve_opts), C.POINTER(eofa_solve_stats), _vp], C.c_int),
    "eofa_measure_fma": ([C.c_int, C.c_int, _dp, _vp], C.c_int),
    "eofa_dot": ([_vp, _vp, _vp, C.c_long, _dp, _dp, _vp], C.c_int),
    "eofa_force_norms": ([_vp, _vp, _dp, _dp, _vp], C.c_int),
    "eofa_destroy": ([_vp], None),
    "eofa_apply_noalloc": ([C.POINTER(eofa_params), _vp, _vp, _vp, _vp], C.c_int),
    "eofa_net_forward": ([_fp, C.POINTER(C.c_int), C.c_int, _vp, _vp, _vp], C.c_int),
    "eofa_net_backward": ([_fp, C.POINTER(C.c_int), C.c_int, _vp, _vp, _fp, _vp, _vp], C.c_int),
    "eofa_train_preconditioner": ([_vp, C.POINTER(_vp), C.c_int, _fp, C.POINTER(eofa_train_opts), _fp,
                                   C.POINTER(eofa_train_stats), _vp], C.c_int),
    "eofa_set_preconditioner": ([_vp, _fp], C.c_int),
    "eofa_status_string": ([C.c_int], C.c_char_p),
    "eofa_last_error": ([_vp], C.c_char_p),
    "eofa_hop_bytes": ([_vp, C.c_int, C.c_int], C.c_double),
    "eofa_tile_sites": ([_vp, C.c_int, C.c_int], C.c_int),
    "eofa_tile_variant": ([_vp, C.c_int, C.c_int], C.c_int),
    "eofa_tile_time": ([_vp, C.c_int, C.c_int, C.c_int], C.c_double),
    "eofa_set_system": ([_vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int], C.c_int),
    "eofa_apply_meofa": ([_vp, C.c_double, C.c_double, _vp, _vp, C.POINTER(eofa_solve_opts),
                          C.POINTER(eofa_solve_stats), _vp], C.c_int),
    "eofa_force": ([_vp, C.c_double, C.c_double, _vp, _vp, C.POINTER(eofa_solve_opts),
                    C.POINTER(eofa_solve_stats), _vp], C.c_int),
    "eofa_heatbath": ([_vp, C.c_double, C.c_double, C.c_int, _dp, _dp, _dp, C.c_int, _vp, _vp,
                       C.POINTER(eofa_solve_opts), C.POINTER(eofa_solve_stats), _vp], C.c_int),
}

_lib = None


def lib():
    """Load libeofa.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1706_05843_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _dptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()):
        raise TypeError("fields must be contiguous complex128 CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _need(a, n, what):
    """The library takes plain pointers: a field of another size would be
    read or written past its end, so the Solver checks sizes first."""
    size = a.size if isinstance(a, np.ndarray) else a.numel()
    if size != n:
        raise ValueError(f"{what}: {size} complex elements, the context needs {n}")


def _check(ctx, status):
    if status != 0:
        msg = lib().eofa_last_error(ctx).decode() if ctx else ""
        raise EofaError(status, msg)


def make_params(dims, Ls, M5=1.8, b=1.5, c=0.5, m1=0.04, m2=1.0, m3=0.04, beta=-1.0, pm=1, t_bc=-1):
    p = eofa_params()
    for i in range(4):
        p.dims[i] = int(dims[i])
    p.Ls, p.M5, p.b, p.c = int(Ls), float(M5), float(b), float(c)
    p.m1, p.m2, p.m3, p.beta = float(m1), float(m2), float(m3), float(beta)
    p.pm, p.t_bc = int(pm), int(t_bc)
    return p


def make_opts(tol=1e-10, inner="f64", inner_tol=0.0, max_iter=0, max_outer=0, use_guess=False,
              rhs_form=0, kernel_timing=False, timeout_ms=0, precond=0, method=0):
    o = eofa_solve_opts()
    o.tol, o.inner, o.inner_tol = float(tol), PREC[inner] if isinstance(inner, str) else int(inner), float(inner_tol)
    o.max_iter, o.max_outer, o.precond = int(max_iter), int(max_outer), int(precond)
    o.use_guess, o.rhs_form, o.kernel_timing = int(use_guess), int(rhs_form), int(kernel_timing)
    o.timeout_ms, o.method = int(timeout_ms), int(method)
    return o


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------
def eofa_create(params, gauge, stream=None):
    ctx = C.c_void_p()
    _check(None, lib().eofa_create(C.byref(params), _dptr(gauge), _stream(stream), C.byref(ctx)))
    return ctx


def eofa_create_gparity(params, gauge, gparity_dirs, stream=None):
    ctx = C.c_void_p()
    _check(None, lib().eofa_create_gparity(C.byref(params), _dptr(gauge), int(gparity_dirs), _stream(stream),
                                           C.byref(ctx)))
    return ctx


def eofa_apply(ctx, inp, out, stream=None):
    _check(ctx, lib().eofa_apply(ctx, _dptr(inp), _dptr(out), _stream(stream)))


def eofa_apply_dag(ctx, inp, out, stream=None):
    _check(ctx, lib().eofa_apply_dag(ctx, _dptr(inp), _dptr(out), _stream(stream)))


def eofa_apply_h(ctx, inp, out, stream=None):
    _check(ctx, lib().eofa_apply_h(ctx, _dptr(inp), _dptr(out), _stream(stream)))


def eofa_solve(ctx, rhs, sol, opts, stream=None, check=True):
    st = eofa_solve_stats()
    s = lib().eofa_solve(ctx, _dptr(rhs), _dptr(sol), C.byref(opts), C.byref(st), _stream(stream))
    if check:
        _check(ctx, s)
    return st


def _hptr(a):
    """Host complex128 field (numpy array or CPU torch tensor, contiguous)."""
    if isinstance(a, np.ndarray):
        if not (a.dtype == np.complex128 and a.flags["C_CONTIGUOUS"]):
            raise TypeError("host fields must be contiguous complex128 arrays")
        return a.ctypes.data_as(_dp)
    import torch
    if not (isinstance(a, torch.Tensor) and not a.is_cuda and a.dtype == torch.complex128 and a.is_contiguous()):
        raise TypeError("host fields must be contiguous complex128 CPU tensors or numpy arrays")
    return C.cast(C.c_void_p(a.data_ptr()), _dp)


def eofa_solve_host(ctx, rhs, sol, opts, stream=None, check=True):
    """eofa_solve with host rhs and sol (copies inside the call)."""
    st = eofa_solve_stats()
    s = lib().eofa_solve_host(ctx, _hptr(rhs), _hptr(sol), C.byref(opts), C.byref(st), _stream(stream))
    if check:
        _check(ctx, s)
    return st


def eofa_measure_fma(prec, reps=5, stream=None):
    """Measured FMA throughput of the current device in TFLOP/s."""
    out = C.c_double(0.0)
    _check(None, lib().eofa_measure_fma(PREC[prec] if isinstance(prec, str) else int(prec), int(reps), C.byref(out),
                                        _stream(stream)))
    return out.value


def eofa_dot(ctx, a, b, stream=None):
    """<a, b> of two complex128 CUDA tensors of equal size, on the device (FP64)."""
    if a.numel() != b.numel():
        raise ValueError("eofa_dot needs fields of equal size")
    re, im = C.c_double(0.0), C.c_double(0.0)
    _check(ctx, lib().eofa_dot(ctx, _dptr(a), _dptr(b), int(a.numel()), C.byref(re), C.byref(im), _stream(stream)))
    return complex(re.value, im.value)


def eofa_force_norms(ctx, force, stream=None):
    """(F_RMS, F_max) of a force from eofa_force, on the device."""
    rms, mx = C.c_double(0.0), C.c_double(0.0)
    _check(ctx, lib().eofa_force_norms(ctx, _dptr(force), C.byref(rms), C.byref(mx), _stream(stream)))
    return rms.value, mx.value


def eofa_set_system(ctx, m1, m2, m3, beta, pm):
    _check(ctx, lib().eofa_set_system(ctx, float(m1), float(m2), float(m3), float(beta), int(pm)))


def eofa_apply_meofa(ctx, m1, m2, phi, out, opts, stream=None, check=True):
    st = (eofa_solve_stats * 2)()
    s = lib().eofa_apply_meofa(ctx, float(m1), float(m2), _dptr(phi), _dptr(out), C.byref(opts), st,
                               _stream(stream))
    if check:
        _check(ctx, s)
    return list(st)


def eofa_force(ctx, m1, m2, phi, force, opts, stream=None, check=True):
    st = (eofa_solve_stats * 2)()
    s = lib().eofa_force(ctx, float(m1), float(m2), _dptr(phi), _dptr(force), C.byref(opts), st, _stream(stream))
    if check:
        _check(ctx, s)
    return list(st)


def _doubles(v):
    a = np.ascontiguousarray(v, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def eofa_heatbath(ctx, m1, m2, alpha0, alpha, beta, eta, phi, opts, pole_tol=None, forecast=0, stream=None,
                  check=True):
    np_ = len(beta)
    if len(alpha) != np_:
        raise ValueError("alpha and beta need one entry per pole")
    a, ap = _doubles([alpha0, *alpha])
    b, bp = _doubles(beta if np_ else [0.0])
    t, tp = (None, None) if pole_tol is None else _doubles(pole_tol)
    if t is not None and len(t) != 2 * np_:
        raise ValueError("pole_tol needs two entries per pole")
    st = (eofa_solve_stats * max(1, 2 * np_))()
    s = lib().eofa_heatbath(ctx, float(m1), float(m2), np_, ap, bp, tp, int(forecast), _dptr(eta), _dptr(phi),
                            C.byref(opts), st, _stream(stream))
    if check:
        _check(ctx, s)
    return list(st)[:2 * np_]


def eofa_apply_batched(ctxs, ins, outs, dag=False, stream=None):
    n = len(ctxs)
    ca = (C.c_void_p * n)(*[c.value for c in ctxs])
    ia = (C.c_void_p * n)(*[_dptr(t).value for t in ins])
    oa = (C.c_void_p * n)(*[_dptr(t).value for t in outs])
    _check(None, lib().eofa_apply_batched(ca, n, ia, oa, int(dag), _stream(stream)))


def eofa_solve_batched(ctxs, rhss, sols, opts, stream=None, check=True):
    n = len(ctxs)
    ca = (C.c_void_p * n)(*[c.value for c in ctxs])
    ra = (C.c_void_p * n)(*[_dptr(t).value for t in rhss])
    sa = (C.c_void_p * n)(*[_dptr(t).value for t in sols])
    st = (eofa_solve_stats * n)()
    s = lib().eofa_solve_batched(ca, n, ra, sa, C.byref(opts), st, _stream(stream))
    if check:
        _check(ctxs[0] if n else None, s)  # errors are reported on the first context
    return list(st)


def eofa_apply_noalloc(params, gauge, inp, out, stream=None):
    """out = K inp without any device allocation (no context; small lattices)."""
    V = int(np.prod([int(x) for x in params.dims]))
    _need(gauge, V * 4 * 9, "gauge field")
    _need(inp, V * int(params.Ls) * 12, "input field")
    _need(out, V * int(params.Ls) * 12, "output field")
    _check(None, lib().eofa_apply_noalloc(C.byref(params), _dptr(gauge), _dptr(inp), _dptr(out),
                                          _stream(stream)))


def _f32ptr(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(_fp)


def _weights(w):
    """The network's weights as host float32: the library copies exactly
    NET_WEIGHTS of them."""
    a, p = _f32ptr(w)
    if a.size != NET_WEIGHTS:
        raise ValueError(f"weights: {a.size} values, the network has {NET_WEIGHTS}")
    return a, p


def _net_rows(dims, *fields):
    """Every network field holds (slices, T, Z, Y, X, 24) float32 values."""
    n = int(fields[0].shape[0]) * int(np.prod([int(x) for x in dims])) * 24
    for f in fields:
        size = None if f is None else (f.size if isinstance(f, np.ndarray) else f.numel())
        if size is not None and size != n:
            raise ValueError(f"network field: {size} values, the lattice and slice count need {n}")


def _f32dev(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("network fields must be contiguous float32 CUDA tensors")
    return C.c_void_p(t.data_ptr())


def eofa_net_forward(weights, dims, inp, out, stream=None):
    """out = net(inp); inp, out: float32 CUDA tensors (S, T, Z, Y, X, 24)."""
    w, wp = _weights(weights)
    _net_rows(dims, inp, out)
    d = (C.c_int * 4)(*[int(x) for x in dims])
    _check(None, lib().eofa_net_forward(wp, d, int(inp.shape[0]), _f32dev(inp), _f32dev(out), _stream(stream)))


def eofa_net_backward(weights, dims, inp, dout, din=None, stream=None):
    """dL/dW (numpy float32, NET_WEIGHTS) and, if din is given, dL/d(inp) into din."""
    w, wp = _weights(weights)
    _net_rows(dims, inp, dout, din)
    d = (C.c_int * 4)(*[int(x) for x in dims])
    dw = np.zeros(NET_WEIGHTS, dtype=np.float32)
    _check(None, lib().eofa_net_backward(wp, d, int(inp.shape[0]), _f32dev(inp), _f32dev(dout),
                                         dw.ctypes.data_as(_fp), _f32dev(din) if din is not None else None,
                                         _stream(stream)))
    return dw


def make_train_opts(pairs=2000, snapshot_every=8, epochs=3, batch=8, lr=1e-3, solve_tol=1e-6, holdout=0):
    o = eofa_train_opts()
    o.pairs, o.snapshot_every, o.epochs, o.batch = int(pairs), int(snapshot_every), int(epochs), int(batch)
    o.lr, o.solve_tol, o.holdout = float(lr), float(solve_tol), int(holdout)
    return o


def eofa_train_preconditioner(ctx, sources, init_weights, opts, stream=None):
    """Train on the context's lattice; returns (weights numpy float32, stats)."""
    n = len(sources)
    sa = (C.c_void_p * n)(*[_dptr(t).value for t in sources])
    w, wp = _weights(init_weights)
    out = np.zeros(NET_WEIGHTS, dtype=np.float32)
    st = eofa_train_stats()
    _check(ctx, lib().eofa_train_preconditioner(ctx, sa, n, wp, C.byref(opts), out.ctypes.data_as(_fp),
                                                C.byref(st), _stream(stream)))
    return out, st


def eofa_set_preconditioner(ctx, weights):
    w, wp = _weights(weights)
    _check(ctx, lib().eofa_set_preconditioner(ctx, wp))


def eofa_destroy(ctx):
    if ctx is not None and ctx.value:
        lib().eofa_destroy(ctx)


def eofa_status_string(s):
    return lib().eofa_status_string(int(s)).decode()


def eofa_hop_bytes(ctx, prec, with_local):
    return float(lib().eofa_hop_bytes(ctx, int(prec), int(with_local)))


def solve_batched(solvers, rhs, out=None, stream=None, check=True, **opts):
    """eofa_solve_batched over Solver objects (one right-hand side each),
    with every field's size checked against its solver; returns (solutions,
    per-system stats)."""
    if len(rhs) != len(solvers) or (out is not None and len(out) != len(solvers)):
        raise ValueError("one right-hand side (and solution) per solver")
    sols = [s._new() for s in solvers] if out is None else list(out)
    for s, r, x in zip(solvers, rhs, sols):
        _need(r, s._n5, "right-hand side")
        _need(x, s._n5, "solution")
    st = eofa_solve_batched([s.ctx for s in solvers], rhs, sols, make_opts(**opts), stream, check=check)
    return sols, st


class Solver:
    """Context owner: Solver(gauge, dims, Ls, **action) then apply / solve.
    gparity: 0, or the bit mask of G-parity directions (bit 0 = x .. bit 3 =
    t); fields then carry a leading flavour axis of 2."""

    def __init__(self, gauge, dims, Ls, stream=None, gparity=0, **action):
        import torch
        if isinstance(gauge, np.ndarray):
            gauge = torch.from_numpy(np.ascontiguousarray(gauge)).cuda()
        self.params = make_params(dims, Ls, **action)
        self.dims, self.Ls, self.gparity = tuple(dims), int(Ls), int(gparity)
        self.ctx = None
        X, Y, Z, T = self.dims
        _need(gauge, X * Y * Z * T * 4 * 9, "gauge field")
        if self.gparity:
            self.ctx = eofa_create_gparity(self.params, gauge, self.gparity, stream)
        else:
            self.ctx = eofa_create(self.params, gauge, stream)

    @property
    def _flavours(self):
        return (2,) if self.gparity else ()

    @property
    def shape5(self):
        X, Y, Z, T = self.dims
        return self._flavours + (T, Z, Y, X, self.Ls, 4, 3)

    def _new(self):
        import torch
        return torch.empty(self.shape5, dtype=torch.complex128, device="cuda")

    @property
    def _n5(self):
        return int(np.prod(self.shape5))

    @property
    def _n4(self):
        return int(np.prod(self.shape4))

    def apply(self, x, dag=False, stream=None):
        _need(x, self._n5, "input field")
        out = self._new()
        (eofa_apply_dag if dag else eofa_apply)(self.ctx, x, out, stream)
        return out

    def apply_h(self, x, stream=None):
        _need(x, self._n5, "input field")
        out = self._new()
        eofa_apply_h(self.ctx, x, out, stream)
        return out

    def solve(self, rhs, stream=None, out=None, check=True, **opts):
        _need(rhs, self._n5, "right-hand side")
        sol = self._new() if out is None else out
        _need(sol, self._n5, "solution")
        st = eofa_solve(self.ctx, rhs, sol, make_opts(**opts), stream, check=check)
        return sol, st

    def solve_host(self, rhs, out, stream=None, check=True, **opts):
        """Solve with host rhs and host out (numpy complex128 or CPU tensors)."""
        _need(rhs, self._n5, "right-hand side")
        _need(out, self._n5, "solution")
        st = eofa_solve_host(self.ctx, rhs, out, make_opts(**opts), stream, check=check)
        return out, st

    def hop_bytes(self, prec, with_local):
        return eofa_hop_bytes(self.ctx, prec, with_local)

    @property
    def shape4(self):
        X, Y, Z, T = self.dims
        return self._flavours + (T, Z, Y, X, 4, 3)

    def set_system(self, m1, m2, m3, beta, pm):
        eofa_set_system(self.ctx, m1, m2, m3, beta, pm)

    def apply_meofa(self, phi, m1, m2, stream=None, check=True, **opts):
        """M_EOFA(m1, m2) phi for a 4D field; returns (out, [minus, plus] stats)."""
        import torch
        _need(phi, self._n4, "4D field")
        out = torch.empty(self.shape4, dtype=torch.complex128, device="cuda")
        st = eofa_apply_meofa(self.ctx, m1, m2, phi, out, make_opts(**opts), stream, check)
        return out, st

    def force(self, phi, m1, m2, stream=None, check=True, **opts):
        """EOFA pseudofermion force sum_a T^a d^a S per link, shape
        (T, Z, Y, X, 4, 3, 3); returns (force, [chi_1, chi_2] stats)."""
        import torch
        _need(phi, self._n4, "4D field")
        X, Y, Z, T = self.dims
        f = torch.empty((T, Z, Y, X, 4, 3, 3), dtype=torch.complex128, device="cuda")
        st = eofa_force(self.ctx, m1, m2, phi, f, make_opts(**opts), stream, check)
        return f, st

    def dot(self, a, b, stream=None):
        """<a, b> on the device (complex)."""
        return eofa_dot(self.ctx, a, b, stream)

    def force_norms(self, force, stream=None):
        """(F_RMS, F_max) of a force from Solver.force (Sec. VI)."""
        X, Y, Z, T = self.dims
        _need(force, X * Y * Z * T * 4 * 9, "force")
        return eofa_force_norms(self.ctx, force, stream)

    def heatbath(self, eta, m1, m2, approx, pole_tol=None, forecast=0, stream=None, check=True, **opts):
        """M_EOFA(m1, m2)^(-1/2) eta with the rational approximation ``approx``
        (alpha0, alpha, beta attributes, e.g. rational.InvSqrt); returns
        (phi, stats of the 2 N_p solves)."""
        import torch
        _need(eta, self._n4, "4D field")
        phi = torch.empty(self.shape4, dtype=torch.complex128, device="cuda")
        st = eofa_heatbath(self.ctx, m1, m2, approx.alpha0, approx.alpha, approx.beta, eta, phi,
                           make_opts(**opts), pole_tol, forecast, stream, check)
        return phi, st

    def train_preconditioner(self, sources, init_weights, opts, stream=None):
        """eofa_train_preconditioner on this context's lattice, with the
        sources' sizes checked; returns (weights, stats)."""
        for t in sources:
            _need(t, self._n5, "training source")
        return eofa_train_preconditioner(self.ctx, sources, init_weights, opts, stream)

    def set_preconditioner(self, weights):
        eofa_set_preconditioner(self.ctx, weights)

    def close(self):
        if self.ctx is not None:
            eofa_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if self.ctx is not None:
                self.close()
        except Exception:
            pass
