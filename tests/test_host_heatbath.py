"""Host logic of the heatbath set-up (paper_1706_05843_gb300/heatbath.py),
without a GPU: a stand-in solver applies a dense Hermitian positive definite
matrix in place of M_EOFA and perturbs each solve's contribution in
proportion to its stopping tolerance, so the spectrum estimate, the
heatbath error and the tolerance tuning of Sec. V.B can be checked against
exact linear algebra."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1706_05843_gb300 import heatbath as H  # noqa: E402
from paper_1706_05843_gb300 import rational  # noqa: E402


class DenseSolver:
    """apply_meofa / heatbath of a dense M; solve j of the heatbath carries
    a relative error of its tolerance (a fixed random direction)."""

    def __init__(self, n=48, lo=1.0, hi=6.0, seed=0):
        rng = np.random.default_rng(seed)
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        # a spectrum in [lo, hi] whose top eigenvalue is well separated
        self.w = np.concatenate([np.linspace(lo, 0.7 * hi, n - 1), [hi]])
        self.M = (Q * self.w) @ Q.conj().T
        self.n = n
        self.noise = rng.standard_normal((64, n)) + 1j * rng.standard_normal((64, n))
        self.calls = 0

    def dot(self, a, b):
        return complex(np.vdot(a.numpy(), b.numpy()))

    def apply_meofa(self, phi, m1, m2, tol=1e-12, **_):
        self.calls += 1
        return torch.from_numpy(self.M @ phi.numpy()), [None, None]

    def heatbath(self, eta, m1, m2, approx, pole_tol=None, forecast=0, tol=1e-10, **_):
        e = eta.numpy()
        out = approx.alpha0 * e
        for l, (a, b) in enumerate(zip(approx.alpha, approx.beta)):
            x = np.linalg.solve(self.M + b * np.eye(self.n), e)
            for t in range(2):  # the two solves of pole l share the term here
                tl = pole_tol[2 * l + t] if pole_tol is not None else tol
                d = self.noise[2 * l + t]
                x = x + 0.5 * tl * np.linalg.norm(x) * d / np.linalg.norm(d)
            out = out + a * x
        return torch.from_numpy(out), [None] * (2 * len(approx.beta))


def test_largest_eigenvalue():
    s = DenseSolver()
    v0 = torch.from_numpy(np.random.default_rng(1).standard_normal(s.n) + 0j)
    lam, hist = H.largest_eigenvalue(s, 0.04, 1.0, v0, iters=80)
    assert abs(lam - s.w[-1]) < 1e-3 * s.w[-1]
    assert all(a <= b * (1 + 1e-12) for a, b in zip(hist, hist[1:]))


def test_heatbath_error_definition():
    s = DenseSolver()
    rng = np.random.default_rng(2)
    eta = torch.from_numpy(rng.standard_normal(s.n) + 1j * rng.standard_normal(s.n))
    w, Q = np.linalg.eigh(s.M)
    exact = Q @ ((Q.conj().T @ eta.numpy()) / np.sqrt(w))
    phi = torch.from_numpy(exact)
    assert H.heatbath_error(s, eta, phi, s.apply_meofa(phi, 0, 0)[0]) < 1e-13
    bad = torch.from_numpy(1.01 * exact)
    assert abs(H.heatbath_error(s, eta, bad, s.apply_meofa(bad, 0, 0)[0]) - (1.01 ** 2 - 1)) < 1e-12


def test_tune_pole_tolerances():
    s = DenseSolver()
    rng = np.random.default_rng(3)
    eta = torch.from_numpy(rng.standard_normal(s.n) + 1j * rng.standard_normal(s.n))
    r = rational.poles_for(1e-13, 0.9, 7.0)
    tols, eps, trials = H.tune_pole_tolerances(s, eta, 0.04, 1.0, r, eps_tol=1e-8, tol=1e-12, factor=10.0,
                                               max_tol=1e-3)
    assert len(tols) == 2 * r.poles
    assert eps <= 1e-8
    assert max(tols) > 1e-12          # something was relaxed
    assert all(1e-12 <= t <= 1e-3 for t in tols)
    # the returned error is that of the returned tolerances
    _, e, _ = H.measure(s, eta, 0.04, 1.0, r, tols, tol=1e-12)
    assert e == pytest.approx(eps, rel=1e-12, abs=1e-18)
    with pytest.raises(ValueError):
        H.tune_pole_tolerances(s, eta, 0.04, 1.0, rational.inv_sqrt(1, 0.9, 7.0), eps_tol=1e-12)
