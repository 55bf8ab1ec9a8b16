"""Pins of the FP64 CPU reference of the warm-start network (CPU only).

The reference's backpropagation is checked against central finite
differences of its own loss (so a dropped term, a wrong skip or a transposed
weight in the backward pass fails), its convolution against scipy's
correlation, and its pooling and upsampling backward maps against the
adjoint identity <A x, y> = <x, A^T y>."""
import numpy as np
import pytest
from scipy.signal import correlate

from oracle import warmstart_ref as ref


def test_conv_matches_scipy_correlation():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 9, 7, 3))
    w = rng.normal(size=(3, 3, 3, 4))
    b = rng.normal(size=4)
    y = ref.conv(x, w, b)
    for bb in range(2):
        for o in range(4):
            want = sum(correlate(x[bb, :, :, c], w[:, :, c, o], mode="same") for c in range(3)) + b[o]
            assert np.max(np.abs(y[bb, :, :, o] - want)) < 1e-12


def test_pool_and_up_backward_are_adjoints():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 8, 8, 3))
    y = rng.normal(size=(2, 4, 4, 3))
    assert abs(np.sum(ref.pool(x) * y) - np.sum(x * ref.pool_backward(y))) < 1e-12
    x2 = rng.normal(size=(2, 4, 4, 3))
    y2 = rng.normal(size=(2, 8, 8, 3))
    assert abs(np.sum(ref.up(x2) * y2) - np.sum(x2 * ref.up_backward(y2))) < 1e-12


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    G = 16
    x = rng.normal(size=(2, G, G, ref.CIN))
    target = rng.normal(size=(2, G, G, 2))
    p = ref.init_params(4)
    # nonzero biases so that every ReLU mask and bias gradient matters
    p += 0.01 * rng.normal(size=p.size)
    L, g = ref.gradients(p, x, target)
    # indices in every layer's weights and biases
    offs, off = [], 0
    for s in ref.param_shapes():
        n = int(np.prod(s))
        offs.append((off, n))
        off += n
    idx = [o + int(rng.integers(n)) for o, n in offs]
    eps = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (ref.loss(ref.forward(pp, x)[0], target) - ref.loss(ref.forward(pm, x)[0], target)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-5 * max(abs(fd), 1e-6 * abs(L)) + 1e-12, (i, fd, g[i])


def test_parameter_count():
    assert ref.n_params() == sum(9 * ci * co + co for ci, co in ref.LAYERS)
    assert 600_000 < ref.n_params() < 800_000
