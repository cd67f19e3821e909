"""The FP64 reference MLP's backward pass against central finite differences."""
import numpy as np

from oracle import mlp


def test_backward_matches_central_differences():
    shapes = mlp.layer_shapes(n_in=7, width=9, n_hidden=3, n_out=3)
    p = mlp.init_params(shapes, seed=5)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((11, 7))
    y = rng.standard_normal((11, 3))
    g = mlp.backward(p, x, y, shapes)
    h = 1e-6
    num = np.zeros_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        num[k] = (mlp.loss(p + e, x, y, shapes) - mlp.loss(p - e, x, y, shapes)) / (2 * h)
    assert np.abs(g - num).max() <= 1e-6 * max(1.0, np.abs(num).max())


def test_gelu_matches_its_definition_and_derivative():
    x = np.linspace(-5, 5, 101)
    ref = 0.5 * x * (1 + np.tanh(np.sqrt(2 / np.pi) * (x + 0.044715 * x ** 3)))
    assert np.allclose(mlp.gelu(x), ref, rtol=0, atol=1e-15)
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)
