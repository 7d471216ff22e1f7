"""Pins for the oracle network (warm-start MLP): gradients against central
differences, GELU against its closed form at special points, and the first Adam step,
which reduces to w - lr * sign(g) for zero initial moments."""
import numpy as np
from scipy.stats import norm

from oracle import mlp as OM


def test_gelu_closed_form():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    assert np.allclose(OM.gelu(z), z * norm.cdf(z), rtol=1e-14, atol=1e-16)
    h = 1e-6
    assert np.allclose(OM.gelu_grad(z), (OM.gelu(z + h) - OM.gelu(z - h)) / (2 * h), rtol=1e-8, atol=1e-10)
    assert OM.gelu(0.0) == 0.0 and abs(OM.gelu_grad(0.0) - 0.5) < 1e-15


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    sizes = [3, 7, 5, 4]
    params = [(rng.standard_normal((a, b)) * 0.5, rng.standard_normal(b) * 0.1) for a, b in zip(sizes[:-1], sizes[1:])]
    X = rng.standard_normal((6, 3))
    T = rng.standard_normal((6, 4))
    _, grads = OM.loss_and_grads(params, X, T)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for (arr, g) in ((W, grads[li][0]), (b, grads[li][1])):
            for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(4)]:
                old = arr[idx]
                arr[idx] = old + h
                lp, _ = OM.loss_and_grads(params, X, T)
                arr[idx] = old - h
                lm, _ = OM.loss_and_grads(params, X, T)
                arr[idx] = old
                assert abs((lp - lm) / (2 * h) - g[idx]) <= 1e-7 * max(1.0, abs(g[idx]))


def test_first_adam_step_is_signed_learning_rate():
    g = np.array([0.3, -2.0, 1e-3])
    w, m1, m2 = OM.adam(np.zeros(3), g, 0.0, 0.0, 1, lr=0.01)
    assert np.allclose(w, -0.01 * np.sign(g), rtol=1e-4)
