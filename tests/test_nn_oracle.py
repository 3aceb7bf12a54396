"""Pins of the float64 conv-net reference (learned initial guess): adjointness
of the transposed convolution and central finite differences of every
parameter and of the input."""

import numpy as np
import pytest

from oracle import nn_oracle as NN


def test_transpose_is_adjoint():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, 4, 4, 4, 3))
    g = rng.standard_normal((2, 4, 4, 4, 5))
    W = rng.standard_normal((3, 3, 3, 3, 5))
    lhs = np.sum(NN.conv3(a, W, np.zeros(5)) * g)
    rhs = np.sum(a * NN.conv3_transpose(g, W))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_conv_is_a_local_stencil_with_zero_border():
    """A delta at an element corner only reaches the 2x2x2 nodes next to it."""
    W = np.ones((3, 3, 3, 1, 1))
    a = np.zeros((1, 3, 3, 3, 1))
    a[0, 0, 0, 0, 0] = 1.0
    y = NN.conv3(a, W, np.zeros(1))[0, ..., 0]
    assert y[:2, :2, :2].min() == 1.0 and y.sum() == 8.0


@pytest.mark.parametrize("name", ["W1", "b1", "W2", "b2", "W3", "b3", "x"])
def test_gradients_match_finite_differences(name):
    rng = np.random.default_rng(1)
    p = NN.init_params(3, cin=2, hidden=4, cout=2)
    x = rng.standard_normal((2, 3, 3, 3, 2))
    gout = rng.standard_normal((2, 3, 3, 3, 2))

    def loss(params, xx):
        out, _ = NN.forward(params, xx)
        return np.sum(out * gout)

    _, cache = NN.forward(p, x)
    grads = NN.backward(p, cache, gout)
    target = x if name == "x" else p[name]
    flat = target.reshape(-1)
    idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
    for i in idx:
        old = flat[i]
        flat[i] = old + 1e-6
        lp = loss(p, x)
        flat[i] = old - 1e-6
        lm = loss(p, x)
        flat[i] = old
        fd = (lp - lm) / 2e-6
        an = grads[name].reshape(-1)[i]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, an)
