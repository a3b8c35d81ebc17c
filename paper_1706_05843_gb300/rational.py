"""Rational approximation of x^(-1/2) for the EOFA heatbath.

The heatbath draws phi = M_EOFA^(-1/2) eta (Sec. III.B).  Its Woodbury form,
Eq. (eofa_heatbath), needs the coefficients of a rational approximation

    x^(-1/2) ~ alpha_0 + sum_l alpha_l / (x + beta_l),   x in [lo, hi],

over an interval that holds the spectrum of M_EOFA.  The paper obtains them
with the Remez algorithm.  For x^(-1/2) the best approximation in the
relative-error norm is known in closed form (Zolotarev's solution, in Jacobi
elliptic functions), so this module evaluates that closed form instead of
iterating: it is the approximation the Remez exchange converges to, and its
error equioscillates at 2n + 2 points (the Chebyshev alternation certificate
that the tests check).

On [1, b], with k'^2 = 1 - 1/b, K' = K(k'^2) and
c_j = sn^2(j K'/(2n+1)) / cn^2(j K'/(2n+1)), j = 1 .. 2n,

    x^(-1/2) ~ d prod_{l=1..n} (x + c_{2l}) / (x + c_{2l-1}),

and d centres the relative error.  The partial fractions of that product and
the map x -> x / lo give the coefficients on [lo, hi].  Host-side set-up only
(numpy, scipy); nothing here runs per solve.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class InvSqrt:
    """alpha_0 + sum_l alpha[l] / (x + beta[l]) ~ x^(-1/2) on [lo, hi]."""
    alpha0: float
    alpha: np.ndarray
    beta: np.ndarray
    lo: float
    hi: float
    err: float          # max |sqrt(x) r(x) - 1| on a dense grid of [lo, hi]

    def __call__(self, x):
        x = np.asarray(x, dtype=np.float64)
        return self.alpha0 + sum(a / (x + b) for a, b in zip(self.alpha, self.beta))

    @property
    def poles(self) -> int:
        return len(self.alpha)


def _grid(lo: float, hi: float, n: int = 200001) -> np.ndarray:
    return np.geomspace(lo, hi, n)


def inv_sqrt(n_poles: int, lo: float, hi: float) -> InvSqrt:
    """Best relative-error rational approximation of x^(-1/2) on [lo, hi] with
    n_poles poles and a constant term (numerator and denominator of degree
    n_poles)."""
    from scipy.special import ellipj, ellipk

    n = int(n_poles)
    if n < 1:
        raise ValueError("need at least one pole")
    if not (0.0 < lo < hi):
        raise ValueError("need 0 < lo < hi")
    b = hi / lo
    m = 1.0 - 1.0 / b
    K = ellipk(m)
    j = np.arange(1, 2 * n + 1)
    sn, cn, _, _ = ellipj(j * K / (2 * n + 1), m)
    c = (sn / cn) ** 2
    zeros, poles = c[1::2], c[0::2]      # c_{2l}, c_{2l-1}
    # residues of prod (y + zeros) / prod (y + poles) at y = -poles[l]
    res = np.empty(n)
    for l in range(n):
        p = poles[l]
        res[l] = np.prod(zeros - p) / np.prod(np.delete(poles, l) - p)
    # centre the relative error on [1, b]
    y = _grid(1.0, b)
    r = np.ones_like(y)
    for z, p in zip(zeros, poles):
        r *= (y + z) / (y + p)
    r *= np.sqrt(y)
    d = 2.0 / (r.max() + r.min())
    # x = lo y:  x^(-1/2) = lo^(-1/2) y^(-1/2)
    s = np.sqrt(lo)
    out = InvSqrt(alpha0=d / s, alpha=d * res * s, beta=poles * lo, lo=lo, hi=hi, err=0.0)
    x = _grid(lo, hi)
    out.err = float(np.abs(np.sqrt(x) * out(x) - 1.0).max())
    return out


def poles_for(tol: float, lo: float, hi: float, max_poles: int = 40) -> InvSqrt:
    """The fewest poles whose relative error on [lo, hi] is below tol."""
    for n in range(1, max_poles + 1):
        r = inv_sqrt(n, lo, hi)
        if r.err <= tol:
            return r
    raise ValueError(f"no approximation with <= {max_poles} poles reaches {tol:g} on [{lo:g}, {hi:g}]")
