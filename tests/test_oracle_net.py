"""Pins of the network oracle (oracle/net.py) to facts fixed by its definition:
a single-tap network is an explicit neighbour lookup, the adjoint and
weight-gradient identities of a convolution, positive homogeneity, and
central finite differences of the whole backward pass."""
import numpy as np
import pytest

from oracle import net as N


def rnd(shape, seed, scale=1.0):
    return np.random.default_rng(seed).standard_normal(shape) * scale


def test_single_tap_is_a_neighbour_lookup():
    """W = identity at one tap: y[x] = in[x + off(tap)] (pins tap order and direction)."""
    S, T, Z, Y, X = 1, 4, 3, 5, 6
    a = rnd((S, T, Z, Y, X, 4), 1)
    for tap in (0, 13, 40, 58, 80):
        W = np.zeros((81, 4, 4))
        W[tap] = np.eye(4)
        y = N.conv(a, W)
        dx, dy, dz, dt = N.offsets(tap)
        for (t, z, yy, x) in [(0, 0, 0, 0), (3, 2, 4, 5), (1, 1, 2, 3)]:
            src = a[0, (t + dt) % T, (z + dz) % Z, (yy + dy) % Y, (x + dx) % X]
            assert np.allclose(y[0, t, z, yy, x], src)


def test_adjoint_identities():
    a = rnd((2, 4, 2, 2, 4, 5), 2)
    d = rnd((2, 4, 2, 2, 4, 3), 3)
    W = rnd((81, 3, 5), 4)
    lhs = np.vdot(d, N.conv(a, W))
    assert abs(lhs - np.vdot(N.conv_adjoint(d, W), a)) < 1e-10 * abs(lhs)
    assert abs(lhs - np.vdot(N.conv_wgrad(a, d), W)) < 1e-10 * abs(lhs)


def test_positive_homogeneity():
    x = rnd((1, 2, 2, 2, 4, 24), 5)
    w = rnd(N.NET_WEIGHTS, 6, 0.05)
    assert np.allclose(N.forward(3.7 * x, w), 3.7 * N.forward(x, w))


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(7)
    x = rnd((2, 2, 2, 2, 4, 24), 8)
    w = rnd(N.NET_WEIGHTS, 9, 0.05)
    g = rnd((2, 2, 2, 2, 4, 24), 10)
    loss = lambda w_, x_: np.vdot(g, N.forward(x_, w_))
    dw, dx = N.backward(x, w, g)
    h = 1e-6
    for i in rng.choice(N.NET_WEIGHTS, 12, replace=False):
        e = np.zeros_like(w)
        e[i] = h
        fd = (loss(w + e, x) - loss(w - e, x)) / (2 * h)
        assert abs(fd - dw[i]) < 1e-6 * max(1.0, abs(fd)), i
    for i in rng.choice(x.size, 8, replace=False):
        e = np.zeros(x.size)
        e[i] = h
        e = e.reshape(x.shape)
        fd = (loss(w, x + e) - loss(w, x - e)) / (2 * h)
        assert abs(fd - dx.ravel()[i]) < 1e-6 * max(1.0, abs(fd)), i


def test_bf16_round():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.14159])
    r = N.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0          # tie to even
    assert r[2] == 1.0 + 2 ** -7
    assert r[3] == -2.5
    assert abs(r[4] - 3.14159) < 2 ** -7 * 4
