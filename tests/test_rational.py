"""The heatbath's rational approximation of x^(-1/2) (host set-up, no GPU).

Pinned to what makes it the best relative-error approximation: its error
equioscillates at 2n + 2 points of [lo, hi] (Chebyshev's alternation
theorem, the fixed point of the Remez exchange the paper uses), the error
falls with the number of poles, and the partial fractions equal the product
form they were expanded from.
"""
import numpy as np
import pytest

pytest.importorskip("scipy")
from paper_1706_05843_gb300 import rational as R  # noqa: E402


def alternation_points(e):
    """Indices of the successive extrema of the error curve e."""
    idx = np.where(np.diff(np.sign(np.diff(e))) != 0)[0] + 1
    pts = np.concatenate(([0], idx, [len(e) - 1]))
    # keep only extrema of near-maximal size and alternating sign
    big = pts[np.abs(e[pts]) > 0.99 * np.abs(e).max()]
    alt = [big[0]]
    for p in big[1:]:
        if np.sign(e[p]) != np.sign(e[alt[-1]]):
            alt.append(p)
    return alt


@pytest.mark.parametrize("n,lo,hi", [(1, 1.0, 10.0), (3, 0.5, 50.0), (5, 0.99, 3.2), (6, 0.2, 400.0)])
def test_equioscillation(n, lo, hi):
    r = R.inv_sqrt(n, lo, hi)
    x = np.geomspace(lo, hi, 400001)
    e = np.sqrt(x) * r(x) - 1.0
    assert len(alternation_points(e)) == 2 * n + 2
    assert abs(e.max() + e.min()) < 1e-3 * r.err      # centred
    assert np.all(r.beta > 0) and np.all(r.alpha > 0) and r.alpha0 > 0


def test_error_falls_with_poles():
    errs = [R.inv_sqrt(n, 0.9, 5.0).err for n in range(1, 7)]
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-12


def test_partial_fractions_match_product():
    """sum form at random points equals the ratio of polynomials with the same
    poles and the zeros recovered from the sum form, and x^(-1/2) to err."""
    r = R.inv_sqrt(4, 0.5, 20.0)
    x = np.random.default_rng(3).uniform(0.5, 20.0, 64)
    num = np.poly1d([r.alpha0])
    for b in r.beta:
        num = num * np.poly1d([1.0, b])
    for l, (a, b) in enumerate(zip(r.alpha, r.beta)):
        others = np.poly1d([a])
        for j, bj in enumerate(r.beta):
            if j != l:
                others = others * np.poly1d([1.0, bj])
        num = num + others
    den = np.poly1d([1.0])
    for b in r.beta:
        den = den * np.poly1d([1.0, b])
    assert np.allclose(r(x), num(x) / den(x), rtol=1e-13)
    assert np.all(np.abs(np.sqrt(x) * r(x) - 1) <= r.err * (1 + 1e-9))
    # the zeros of the numerator interlace the poles (Zolotarev's structure)
    z = np.sort(-np.real(num.roots))
    p = np.sort(r.beta)
    assert np.all(p[:-1] < z[1:]) and np.all(z[:-1] < p[1:])


def test_poles_for_tolerance():
    r = R.poles_for(1e-10, 0.98, 3.3)
    assert r.err <= 1e-10
    assert R.inv_sqrt(r.poles - 1, 0.98, 3.3).err > 1e-10


def test_rejects_bad_interval():
    with pytest.raises(ValueError):
        R.inv_sqrt(3, 2.0, 1.0)
    with pytest.raises(ValueError):
        R.inv_sqrt(0, 1.0, 2.0)
