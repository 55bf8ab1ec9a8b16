"""FP64 CPU reference of the warm-start network (test infrastructure only).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: it checks the CUDA
library's hand-written BF16 network kernels (forward, backward, loss) and
is never called by the library.  It shares no code with the CUDA path.

The network maps input planes of a G x G grid (channels last, NHWC) to two
output planes (the real and imaginary parts of a proposed wave function).
It is a convolutional encoder-decoder with additive skips; every
convolution is 3 x 3, stride 1, zero padding 1:

    e0 = relu(conv(x, 0))          G,    Cin -> 32
    e1 = relu(conv(e0, 1))         G,    32  -> 32       (skip s1)
    e2 = relu(conv(pool(e1), 2))   G/2,  32  -> 64
    e3 = relu(conv(e2, 3))         G/2,  64  -> 64       (skip s2)
    e4 = relu(conv(pool(e3), 4))   G/4,  64  -> 128
    e5 = relu(conv(e4, 5))         G/4,  128 -> 128      (skip s3)
    b6 = relu(conv(pool(e5), 6))   G/8,  128 -> 128
    b7 = relu(conv(b6, 7))         G/8,  128 -> 128
    d8 = relu(conv(up(b7) + e5, 8))  G/4, 128 -> 64
    d9 = relu(conv(up(d8) + e3, 9))  G/2, 64  -> 32
    d10 = relu(conv(up(d9) + e1, 10)) G,  32  -> 32
    y  = conv(d10, 11)             G,    32  -> 2

pool = mean of each 2 x 2 block, up = nearest-neighbour doubling.  Weights
of layer i: W_i[ky][kx][ci][co] and bias b_i[co]; the flat parameter vector
is (W_0, b_0, W_1, b_1, ...) in that order.  Loss = mean over all output
elements of (y - target)^2.
"""
from __future__ import annotations

import numpy as np

CIN = 6
LAYERS = [(CIN, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 128),
          (128, 128), (128, 64), (64, 32), (32, 32), (32, 2)]


def param_shapes():
    out = []
    for ci, co in LAYERS:
        out.append((3, 3, ci, co))
        out.append((co,))
    return out


def n_params() -> int:
    return int(sum(np.prod(s) for s in param_shapes()))


def unflatten(flat: np.ndarray):
    ps, off = [], 0
    for s in param_shapes():
        n = int(np.prod(s))
        ps.append(np.asarray(flat[off:off + n], dtype=np.float64).reshape(s))
        off += n
    return [(ps[2 * i], ps[2 * i + 1]) for i in range(len(LAYERS))]


def conv(x, w, b):
    """3 x 3 convolution, stride 1, zero padding 1: x [B,H,W,C], w [3,3,C,O]."""
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, W, w.shape[3]))
    for ky in range(3):
        for kx in range(3):
            y += xp[:, ky:ky + H, kx:kx + W, :] @ w[ky, kx]
    return y + b


def conv_backward(x, w, dy):
    """Gradients of conv(x, w, b) given dL/dy: (dL/dx, dL/dw, dL/db)."""
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + H, kx:kx + W, :]
            dw[ky, kx] = np.einsum("bhwc,bhwo->co", patch, dy)
            dxp[:, ky:ky + H, kx:kx + W, :] += dy @ w[ky, kx].T
    return dxp[:, 1:-1, 1:-1, :], dw, dy.sum(axis=(0, 1, 2))


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(dy):
    B, H, W, C = dy.shape
    return dy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(flat, x):
    """Output y and the cache of every layer's input and output."""
    P = unflatten(flat)
    cache = []

    def layer(i, inp, act=True):
        z = conv(inp, *P[i])
        out = np.maximum(z, 0.0) if act else z
        cache.append((inp, out, act))
        return out

    e0 = layer(0, x)
    e1 = layer(1, e0)
    e2 = layer(2, pool(e1))
    e3 = layer(3, e2)
    e4 = layer(4, pool(e3))
    e5 = layer(5, e4)
    b6 = layer(6, pool(e5))
    b7 = layer(7, b6)
    d8 = layer(8, up(b7) + e5)
    d9 = layer(9, up(d8) + e3)
    d10 = layer(10, up(d9) + e1)
    y = layer(11, d10, act=False)
    return y, cache


def loss(y, target) -> float:
    return float(np.mean((y - target) ** 2))


def gradients(flat, x, target):
    """(loss, flat gradient of the loss) by backpropagation."""
    P = unflatten(flat)
    y, cache = forward(flat, x)
    L = loss(y, target)
    grads = [None] * len(LAYERS)

    def back(i, dout):
        inp, out, act = cache[i]
        dz = dout * (out > 0) if act else dout
        dx, dw, db = conv_backward(inp, P[i][0], dz)
        grads[i] = (dw, db)
        return dx

    dy = 2.0 * (y - target) / y.size
    g10 = back(11, dy)
    g_sum10 = back(10, g10)          # d/d(up(d9) + e1)
    g_e1 = g_sum10.copy()
    g9 = back(9, up_backward(g_sum10))
    g_e3 = g9.copy()
    g8 = back(8, up_backward(g9))
    g_e5 = g8.copy()
    g7 = back(7, up_backward(g8))
    g6 = back(6, g7)
    g_e5 = g_e5 + pool_backward(g6)
    g5 = back(5, g_e5)
    g4 = back(4, g5)
    g_e3 = g_e3 + pool_backward(g4)
    g3 = back(3, g_e3)
    g2 = back(2, g3)
    g_e1 = g_e1 + pool_backward(g2)
    g1 = back(1, g_e1)
    back(0, g1)
    flat_g = np.concatenate([np.concatenate([dw.ravel(), db.ravel()]) for dw, db in grads])
    return L, flat_g


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases (any start is fine for a reference)."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co in LAYERS:
        out.append(rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), size=(3, 3, ci, co)).ravel())
        out.append(np.zeros(co))
    return np.concatenate(out)
