"""Pins of the learned path's oracle (oracle/mlp.py): the hand-written gradient
against central finite differences of the loss, closed forms of the forward
pass and of Adam, and the bucket function's monotonicity."""
import numpy as np
import pytest

from oracle import mlp


def _params(seed, scale=0.5):
    return np.random.default_rng(seed).normal(0.0, scale, mlp.NPARAM)


def test_param_count():
    assert mlp.NPARAM == 1153


def test_forward_closed_forms():
    p = _params(1)
    p[mlp.W3:mlp.B3] = 0.0
    p[mlp.B3] = 0.0
    y, _ = mlp.forward(p, np.linspace(0, 1, 7))
    assert np.all(y == 0.0)                       # tanh(0): no correction
    assert np.array_equal(mlp.cdf_estimate(p, [0.25, 0.5]), [0.25, 0.5])
    p = np.zeros(mlp.NPARAM)
    p[mlp.B3] = np.log(3.0) / 2                   # tanh(log(3)/2) = 1/2
    y, _ = mlp.forward(p, [0.3])
    assert abs(y[0] - 0.5) < 1e-15
    assert abs(mlp.cdf_estimate(p, [0.3])[0] - (0.3 + 0.5 / 64)) < 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(100 + seed)
    p = _params(seed)
    x = rng.random(64)
    t = np.sort(rng.random(64))
    _, g = mlp.loss_grad(p, x, t)
    h = 1e-6
    idx = np.concatenate([np.arange(0, mlp.NPARAM, 7), [mlp.B3, mlp.W2 + 33, mlp.B2 + 5]])
    for i in idx:
        d = np.zeros(mlp.NPARAM)
        d[i] = h
        num = (mlp.loss(p + d, x, t) - mlp.loss(p - d, x, t)) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)) + 1e-9, i


def test_adam_closed_form():
    """With beta1 = beta2 = 0 the Adam step is -lr * g / (|g| + eps)."""
    p = _params(3)
    g = np.random.default_rng(3).normal(size=mlp.NPARAM)
    q, m1, m2 = mlp.adam_step(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr=0.1, beta1=0.0, beta2=0.0, eps=0.0)
    assert np.allclose(q, p - 0.1 * np.sign(g), atol=1e-15)
    assert np.array_equal(m1, g) and np.allclose(m2, g * g)


def test_bucket_function_monotone_and_tie_consistent():
    rng = np.random.default_rng(5)
    spl = np.sort(rng.integers(0, 1 << 40, 4095).astype(np.uint64))
    e = np.sort(rng.integers(0, 1 << 40, 100000).astype(np.uint64))
    b = mlp.buckets_from_splitters(e, spl)
    assert np.all(np.diff(b) >= 0) and b.min() >= 0 and b.max() <= 4095
    assert np.array_equal(mlp.buckets_from_splitters(spl, spl),
                          np.searchsorted(spl, spl, side="right"))
