"""FP64 CPU oracle for the EOFA Dirac-equation solve (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``eofa_oracle.c`` (plain C,
compiled with gcc and OpenMP) through ctypes and shares nothing with the CUDA
library.  Every function cites the passage of arXiv:1706.05843 it follows in
the C source.

Fields are numpy complex128 arrays in the layouts of
``paper_1706_05843_gb300.inputs``: gauge ``(T, Z, Y, X, 4, 3, 3)``, 5D fields
``(T, Z, Y, X, Ls, 4, 3)``, 4D fields ``(T, Z, Y, X, 4, 3)``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eofa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    """Mirror of ``oracle_params`` in eofa_oracle.c."""
    _fields_ = [
        ("dims", C.c_int * 4),
        ("Ls", C.c_int),
        ("M5", C.c_double),
        ("b", C.c_double),
        ("c", C.c_double),
        ("m1", C.c_double),
        ("m2", C.c_double),
        ("m3", C.c_double),
        ("beta", C.c_double),
        ("pm", C.c_int),
        ("t_bc", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("converged", C.c_int),
        ("true_res", C.c_double),
        ("recur_res", C.c_double),
    ]


@dataclass
class Action:
    """Physics parameters of one EOFA system (Moebius b5 = b, c5 = c)."""
    dims: tuple
    Ls: int
    M5: float = 1.8
    b: float = 1.5
    c: float = 0.5
    m1: float = 0.04
    m2: float = 1.0
    m3: float = 0.04
    beta: float = -1.0
    pm: int = 1
    t_bc: int = -1

    def cparams(self) -> Params:
        p = Params()
        for i in range(4):
            p.dims[i] = int(self.dims[i])
        p.Ls = int(self.Ls)
        p.M5, p.b, p.c = float(self.M5), float(self.b), float(self.c)
        p.m1, p.m2, p.m3 = float(self.m1), float(self.m2), float(self.m3)
        p.beta, p.pm, p.t_bc = float(self.beta), int(self.pm), int(self.t_bc)
        return p

    def replace(self, **kw) -> "Action":
        d = dict(self.__dict__)
        d.update(kw)
        return Action(**d)


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER(Params)
        vp = C.c_void_p
        d = C.c_double
        for name, args in [
            ("oracle_dw4", [P, vp, vp, vp, C.c_int]),
            ("oracle_dw5", [P, vp, vp, vp, C.c_int]),
            ("oracle_L", [P, d, vp, vp, C.c_int]),
            ("oracle_ddwf", [P, vp, d, vp, vp, C.c_int]),
            ("oracle_dtilde", [P, d, vp, vp, C.c_int]),
            ("oracle_dtilde_inv", [P, d, vp, vp]),
            ("oracle_deofa", [P, vp, d, vp, vp, C.c_int]),
            ("oracle_g5r5", [P, vp, vp]),
            ("oracle_h", [P, vp, d, vp, vp]),
            ("oracle_apply_hsys", [P, vp, vp, vp]),
            ("oracle_apply_asys", [P, vp, vp, vp, C.c_int]),
            ("oracle_apply_k", [P, vp, vp, vp, C.c_int]),
            ("oracle_L_matrices", [P, d, vp, vp]),
            ("oracle_omega", [P, C.c_int, vp]),
            ("oracle_delta", [P, d, d, C.c_int, vp]),
            ("oracle_mpm", [P, d, vp, vp]),
            ("oracle_dtilde_inv_matrices", [P, d, vp, vp]),
            ("oracle_uv", [P, vp, vp]),
            ("oracle_gamma", [C.c_int, vp]),
            ("oracle_set_threads", [C.c_int]),
        ]:
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None
        L.oracle_apply_k_sites.argtypes = [P, vp, vp, vp, C.c_long, vp]
        L.oracle_apply_k_sites.restype = None
        L.oracle_k.argtypes = [P, d, d]
        L.oracle_k.restype = d
        L.oracle_norm2.argtypes = [vp, C.c_long]
        L.oracle_norm2.restype = d
        for name in ("oracle_solve_h", "oracle_solve_k"):
            f = getattr(L, name)
            f.argtypes = [P, vp, vp, vp, d, C.c_int, C.c_int, C.POINTER(Stats)]
            f.restype = C.c_int
        L.oracle_num_threads.argtypes = []
        L.oracle_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """Bound (action, gauge field) pair; all methods return new arrays."""

    def __init__(self, action: Action, U: np.ndarray):
        self.a = action
        self.p = action.cparams()
        self.U = _c(U)
        X, Y, Z, T = action.dims
        assert self.U.shape == (T, Z, Y, X, 4, 3, 3)
        self.shape5 = (T, Z, Y, X, action.Ls, 4, 3)
        self.shape4 = (T, Z, Y, X, 4, 3)

    # -- 5D operators -------------------------------------------------
    def _op5(self, fn, x, *pre, dag=None):
        x = _c(x)
        out = np.empty_like(x)
        args = [C.byref(self.p)] + list(pre) + [_ptr(x), _ptr(out)]
        if dag is not None:
            args.append(int(dag))
        fn(*args)
        return out

    def dw5(self, x, dag=False):
        return self._op5(lib().oracle_dw5, x, _ptr(self.U), dag=dag)

    def dw4(self, x, dag=False):
        return self._op5(lib().oracle_dw4, x, _ptr(self.U), dag=dag)

    def L(self, x, m, dag=False):
        return self._op5(lib().oracle_L, x, C.c_double(m), dag=dag)

    def ddwf(self, x, m, dag=False):
        return self._op5(lib().oracle_ddwf, x, _ptr(self.U), C.c_double(m), dag=dag)

    def dtilde(self, x, m, dag=False):
        return self._op5(lib().oracle_dtilde, x, C.c_double(m), dag=dag)

    def dtilde_inv(self, x, m):
        return self._op5(lib().oracle_dtilde_inv, x, C.c_double(m))

    def deofa(self, x, m, dag=False):
        return self._op5(lib().oracle_deofa, x, _ptr(self.U), C.c_double(m), dag=dag)

    def g5r5(self, x):
        return self._op5(lib().oracle_g5r5, x)

    def h(self, x, m):
        return self._op5(lib().oracle_h, x, _ptr(self.U), C.c_double(m))

    def hsys(self, x):
        """(H(m1) + beta Delta_pm(m2,m3) P_pm) x."""
        return self._op5(lib().oracle_apply_hsys, x, _ptr(self.U))

    def asys(self, x, dag=False):
        """(D_EOFA(m1) + beta g5 R5 Delta_pm P_pm) x, or its adjoint."""
        return self._op5(lib().oracle_apply_asys, x, _ptr(self.U), dag=dag)

    def k(self, x, dag=False):
        """Cayley-form K = D_DWF(m1) + pm beta u (x) v P_pm, or K^dag."""
        return self._op5(lib().oracle_apply_k, x, _ptr(self.U), dag=dag)

    def k_sites(self, x, sites):
        """(K x)(site, s) at the given lexicographic 4D sites, shape (n, Ls, 4, 3)."""
        x = _c(x)
        sites = np.ascontiguousarray(sites, dtype=np.int64)
        out = np.empty((len(sites), self.a.Ls, 4, 3), dtype=np.complex128)
        lib().oracle_apply_k_sites(C.byref(self.p), _ptr(self.U), _ptr(x), _ptr(sites), len(sites), _ptr(out))
        return out

    # -- solves -------------------------------------------------------
    def _solve(self, fn, rhs, tol, maxit, guess):
        rhs = _c(rhs)
        x = np.zeros_like(rhs) if guess is None else _c(guess).copy()
        st = Stats()
        fn(C.byref(self.p), _ptr(self.U), _ptr(rhs), _ptr(x), float(tol),
           int(maxit), int(guess is not None), C.byref(st))
        return x, st

    def solve_h(self, phi, tol=1e-12, maxit=100000, guess=None):
        """psi with (H(m1) + beta Delta_pm P_pm) psi = phi; returns (psi, stats)."""
        return self._solve(lib().oracle_solve_h, phi, tol, maxit, guess)

    def solve_k(self, b, tol=1e-12, maxit=100000, guess=None):
        """psi' with K psi' = b; returns (psi', stats)."""
        return self._solve(lib().oracle_solve_k, b, tol, maxit, guess)

    # -- fifth-dimension matrices (App. A) ----------------------------
    def _mat(self):
        return np.zeros((self.a.Ls, self.a.Ls), dtype=np.float64)

    def L_matrices(self, m):
        Lp, Lm = self._mat(), self._mat()
        lib().oracle_L_matrices(C.byref(self.p), m, _ptr(Lp), _ptr(Lm))
        return Lp, Lm

    def mpm(self, m):
        Mp, Mm = self._mat(), self._mat()
        lib().oracle_mpm(C.byref(self.p), m, _ptr(Mp), _ptr(Mm))
        return Mp, Mm

    def delta(self, mA, mB, pm):
        D = self._mat()
        lib().oracle_delta(C.byref(self.p), mA, mB, int(pm), _ptr(D))
        return D

    def omega(self, pm):
        o = np.zeros(self.a.Ls)
        lib().oracle_omega(C.byref(self.p), int(pm), _ptr(o))
        return o

    def kcoef(self, mA, mB):
        return lib().oracle_k(C.byref(self.p), mA, mB)

    def dtilde_inv_matrices(self, m):
        Ip, Im = self._mat(), self._mat()
        lib().oracle_dtilde_inv_matrices(C.byref(self.p), m, _ptr(Ip), _ptr(Im))
        return Ip, Im

    def uv(self):
        u = np.zeros(self.a.Ls)
        k = np.zeros(1)
        lib().oracle_uv(C.byref(self.p), _ptr(u), _ptr(k))
        return u, float(k[0])


def gamma(mu: int) -> np.ndarray:
    """The oracle's gamma matrix: mu 0..3 -> gamma_1..gamma_4, 4 -> gamma_5."""
    g = np.zeros((4, 4), dtype=np.complex128)
    lib().oracle_gamma(int(mu), _ptr(g))
    return g


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def norm2(v: np.ndarray) -> float:
    v = _c(v)
    return float(lib().oracle_norm2(_ptr(v), v.size))
