"""FP64 CPU reference of the corrector MLP (test infrastructure only).

Plain numpy forward and backward of the multilayer perceptron that the CUDA
library trains in BF16 with FP32 accumulation: layers in -> 64 -> 64 -> 64 ->
out, GELU (tanh form) after each hidden layer, mean-squared-error loss.  The
backward pass is written out layer by layer (no autograd) and is checked by
central finite differences in tests/test_mlp_reference.py.

Parameter layout (flat, FP64 here, FP32 in the library): for each layer l,
W_l as [n_out][n_in] row-major, then b_l [n_out].
"""
from __future__ import annotations

import math

import numpy as np

SQ2PI = math.sqrt(2.0 / math.pi)


def layer_shapes(n_in=47, width=64, n_hidden=3, n_out=6):
    dims = [n_in] + [width] * n_hidden + [n_out]
    return [(dims[k + 1], dims[k]) for k in range(len(dims) - 1)]


def n_params(shapes):
    return sum(o * i + o for o, i in shapes)


def unpack(p, shapes):
    out, off = [], 0
    for o, i in shapes:
        W = p[off:off + o * i].reshape(o, i)
        off += o * i
        b = p[off:off + o]
        off += o
        out.append((W, b))
    return out


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(SQ2PI * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    t = np.tanh(SQ2PI * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * SQ2PI * (1.0 + 3.0 * 0.044715 * x * x)


def forward(p, x, shapes):
    """Returns the output and the pre-activations of every layer."""
    layers = unpack(np.asarray(p, dtype=np.float64), shapes)
    a = np.asarray(x, dtype=np.float64)
    zs, acts = [], [a]
    for k, (W, b) in enumerate(layers):
        z = a @ W.T + b
        zs.append(z)
        a = gelu(z) if k < len(layers) - 1 else z
        acts.append(a)
    return a, zs, acts


def loss(p, x, y, shapes):
    out, _, _ = forward(p, x, shapes)
    return float(np.mean(np.sum((out - y) ** 2, axis=1)))


def backward(p, x, y, shapes):
    """Gradient of loss() with respect to the flat parameters (backprop)."""
    layers = unpack(np.asarray(p, dtype=np.float64), shapes)
    out, zs, acts = forward(p, x, shapes)
    m = x.shape[0]
    d = 2.0 * (out - y) / m                      # dL/d(output)
    grads = []
    for k in range(len(layers) - 1, -1, -1):
        W, _ = layers[k]
        if k < len(layers) - 1:
            d = d * gelu_grad(zs[k])             # through the activation
        gW = d.T @ acts[k]
        gb = d.sum(axis=0)
        grads.append((gW, gb))
        d = d @ W
    g = []
    for gW, gb in reversed(grads):
        g += [gW.ravel(), gb]
    return np.concatenate(g)


def init_params(shapes, seed):
    """Uniform(-1/sqrt(n_in), 1/sqrt(n_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in shapes:
        lim = 1.0 / math.sqrt(i)
        parts += [rng.uniform(-lim, lim, o * i), np.zeros(o)]
    return np.concatenate(parts)
