"""Float64 CPU reference of the per-element 3-D convolutional network used for
the learned initial guess. TEST INFRASTRUCTURE ONLY: the product path runs its
own CUDA kernels; tests compare them with this reference.

The network is not in the paper: it maps, element by element, two input
channels on the element's (p+1)^3 nodes (the scaled source and a scaled
coarse-grid solution) through three 3x3x3 convolutions with zero padding at
the element border (2 -> 32 -> 32 -> 2 channels, ReLU after the first two).

Layout: activations are [n_elem, n1, n1, n1, C] with index (z, y, x),
channels last; weights W_l are [3, 3, 3, C_in, C_out] indexed by the tap
(dz + 1, dy + 1, dx + 1); biases b_l are [C_out]. A tap (dz, dy, dx) reads the
input at (z + dz, y + dy, x + dx).
"""

from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3(a, W, b):
    """y[e, z, y, x, co] = b[co] + sum_taps sum_ci W[tap, ci, co] a[e, z+dz, y+dy, x+dx, ci]."""
    ne, n1 = a.shape[0], a.shape[1]
    cout = W.shape[-1]
    pad = np.zeros((ne, n1 + 2, n1 + 2, n1 + 2, a.shape[-1]))
    pad[:, 1:-1, 1:-1, 1:-1, :] = a
    y = np.broadcast_to(b, (ne, n1, n1, n1, cout)).copy()
    for (dz, dy, dx) in TAPS:
        sl = pad[:, 1 + dz:1 + dz + n1, 1 + dy:1 + dy + n1, 1 + dx:1 + dx + n1, :]
        y += sl @ W[dz + 1, dy + 1, dx + 1]
    return y


def conv3_transpose(g, W):
    """Adjoint of conv3 with respect to its input: x[.., ci] = sum_taps W[tap, ci, :] g[.. - tap, :]."""
    ne, n1 = g.shape[0], g.shape[1]
    cin = W.shape[-2]
    out = np.zeros((ne, n1 + 2, n1 + 2, n1 + 2, cin))
    for (dz, dy, dx) in TAPS:
        out[:, 1 + dz:1 + dz + n1, 1 + dy:1 + dy + n1, 1 + dx:1 + dx + n1, :] += g @ W[dz + 1, dy + 1, dx + 1].T
    return out[:, 1:-1, 1:-1, 1:-1, :]


def conv3_weight_grad(a, g):
    """dW[tap, ci, co] = sum over elements and nodes of g[.., co] a[.. + tap, ci]."""
    ne, n1 = a.shape[0], a.shape[1]
    pad = np.zeros((ne, n1 + 2, n1 + 2, n1 + 2, a.shape[-1]))
    pad[:, 1:-1, 1:-1, 1:-1, :] = a
    dW = np.zeros((3, 3, 3, a.shape[-1], g.shape[-1]))
    for (dz, dy, dx) in TAPS:
        sl = pad[:, 1 + dz:1 + dz + n1, 1 + dy:1 + dy + n1, 1 + dx:1 + dx + n1, :]
        dW[dz + 1, dy + 1, dx + 1] = np.einsum("ezyxi,ezyxo->io", sl, g)
    return dW


def forward(params, x):
    """params: dict W1, b1, W2, b2, W3, b3. x: [ne, n1, n1, n1, 2].
    Returns (out, cache)."""
    z1 = conv3(x, params["W1"], params["b1"])
    a1 = np.maximum(z1, 0.0)
    z2 = conv3(a1, params["W2"], params["b2"])
    a2 = np.maximum(z2, 0.0)
    out = conv3(a2, params["W3"], params["b3"])
    return out, (x, z1, a1, z2, a2)


def backward(params, cache, gout):
    """Gradients of sum(gout * out) with respect to every parameter and the input."""
    x, z1, a1, z2, a2 = cache
    grads = {}
    grads["W3"] = conv3_weight_grad(a2, gout)
    grads["b3"] = gout.sum(axis=(0, 1, 2, 3))
    g2 = conv3_transpose(gout, params["W3"]) * (z2 > 0)
    grads["W2"] = conv3_weight_grad(a1, g2)
    grads["b2"] = g2.sum(axis=(0, 1, 2, 3))
    g1 = conv3_transpose(g2, params["W2"]) * (z1 > 0)
    grads["W1"] = conv3_weight_grad(x, g1)
    grads["b1"] = g1.sum(axis=(0, 1, 2, 3))
    grads["x"] = conv3_transpose(g1, params["W1"])
    return grads


def init_params(seed, cin=2, hidden=32, cout=2):
    """He-style random initialisation for tests."""
    rng = np.random.default_rng(seed)

    def w(ci, co):
        return rng.standard_normal((3, 3, 3, ci, co)) * np.sqrt(2.0 / (27 * ci))

    return {"W1": w(cin, hidden), "b1": np.zeros(hidden), "W2": w(hidden, hidden), "b2": np.zeros(hidden),
            "W3": w(hidden, cout) * 0.1, "b3": np.zeros(cout)}
