"""FP64 numpy oracle of the learned preconditioner's network (test infrastructure).

Only tests/ may import this module.  The network is defined by the C ABI
(include/eofa.h): three 3^4 convolutions over a periodic 4D lattice applied
to each slice on its own, channels 24 -> 32 -> 32 -> 24, no biases,
LeakyReLU(0.1) after the first two layers.  Weights are one flat array, the
three layers one after another, each W[tap][co][ci] with
tap = ((dt*3 + dz)*3 + dy)*3 + dx for the neighbour offset (dx-1, ..., dt-1):

    y[x][co] = sum_tap sum_ci W[tap][co][ci] in[x + off(tap)][ci]

Fields are arrays of shape (S, T, Z, Y, X, C).  Everything here is the plain
definition: np.roll for the neighbour shift, einsum for the channel sums,
and hand-written adjoints for the backward pass (pinned by finite
differences and adjoint identities in tests/test_oracle_net.py).
"""
from __future__ import annotations

import numpy as np

LEAKY = 0.1
CIN = (24, 32, 32)
COUT = (32, 32, 24)
NET_WEIGHTS = sum(81 * i * o for i, o in zip(CIN, COUT))


def offsets(tap: int):
    """(dx, dy, dz, dt) of a tap."""
    return (tap % 3 - 1, (tap // 3) % 3 - 1, (tap // 9) % 3 - 1, tap // 27 - 1)


def split(weights):
    w = np.asarray(weights, dtype=np.float64)
    out, off = [], 0
    for ci, co in zip(CIN, COUT):
        n = 81 * co * ci
        out.append(w[off:off + n].reshape(81, co, ci))
        off += n
    return out


def shift(a, tap, sign=+1):
    """b[x] = a[x + sign * off(tap)] on the periodic lattice (axes t, z, y, x = 1..4)."""
    dx, dy, dz, dt = offsets(tap)
    return np.roll(a, shift=(-sign * dt, -sign * dz, -sign * dy, -sign * dx), axis=(1, 2, 3, 4))


def conv(a, W):
    """y[x][co] = sum_tap sum_ci W[tap][co][ci] a[x + off(tap)][ci]."""
    out = np.zeros(a.shape[:-1] + (W.shape[1],))
    for tap in range(81):
        out += np.einsum("stzyxi,oi->stzyxo", shift(a, tap), W[tap])
    return out


def conv_adjoint(d, W):
    """The adjoint of conv in its input: a_bar[x][ci] = sum_tap sum_co W[tap][co][ci] d[x - off(tap)][co]."""
    out = np.zeros(d.shape[:-1] + (W.shape[2],))
    for tap in range(81):
        out += np.einsum("stzyxo,oi->stzyxi", shift(d, tap, -1), W[tap])
    return out


def conv_wgrad(a, d):
    """dW[tap][co][ci] = sum_x d[x][co] a[x + off(tap)][ci]."""
    return np.stack([np.einsum("stzyxo,stzyxi->oi", d, shift(a, tap)) for tap in range(81)])


def leaky(z):
    return np.where(z > 0, z, LEAKY * z)


def dleaky(z):
    return np.where(z > 0, 1.0, LEAKY)


def forward(x, weights, cache=False):
    W = split(weights)
    z1 = conv(x, W[0])
    a1 = leaky(z1)
    z2 = conv(a1, W[1])
    a2 = leaky(z2)
    out = conv(a2, W[2])
    if cache:
        return out, (x, z1, a1, z2, a2)
    return out


def backward(x, weights, dout):
    """(dL/dW flat, dL/dx) for dL/d(out) = dout."""
    W = split(weights)
    out, (x, z1, a1, z2, a2) = forward(x, weights, cache=True)
    dW2 = conv_wgrad(a2, dout)
    dz2 = conv_adjoint(dout, W[2]) * dleaky(z2)
    dW1 = conv_wgrad(a1, dz2)
    dz1 = conv_adjoint(dz2, W[1]) * dleaky(z1)
    dW0 = conv_wgrad(x, dz1)
    dx = conv_adjoint(dz1, W[0])
    return np.concatenate([dW0.ravel(), dW1.ravel(), dW2.ravel()]), dx


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
