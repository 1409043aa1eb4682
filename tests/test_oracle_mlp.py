"""Pins of the learned path's oracle (oracle/mlp.py): the hand-written gradient
against central finite differences of the loss, closed forms of the forward
pass (including which index of the W2 block is the input unit) and of Adam,
and the bucket function against a brute-force count in plain Python.

GNS_ORACLE_MLP may name another copy of mlp.py: the mutation test points it
at copies with planted mistakes, which these pins must catch."""
import importlib.util
import os

import numpy as np
import pytest


def _load_mlp():
    path = os.environ.get("GNS_ORACLE_MLP")
    if not path:
        from oracle import mlp
        return mlp
    spec = importlib.util.spec_from_file_location("mlp_under_test", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


mlp = _load_mlp()


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


def test_forward_w2_orientation():
    """Row j of the W2 block holds the inputs of layer-2 unit j: with only
    w1[1] = 1, W2[0][1] = 2 and w3[0] = 1 non-zero, the output is
    tanh(tanh(2 tanh(x))); the transposed reading gives 0."""
    p = np.zeros(mlp.NPARAM)
    p[mlp.W1 + 1] = 1.0
    p[mlp.W2 + 0 * mlp.H + 1] = 2.0
    p[mlp.W3 + 0] = 1.0
    x = np.array([-0.7, 0.2, 1.3])
    y, _ = mlp.forward(p, x)
    assert np.allclose(y, np.tanh(np.tanh(2.0 * np.tanh(x))), rtol=0, atol=1e-15)


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


def test_adam_bias_correction_closed_form():
    """With the default betas and eps = 0, a gradient that stays the same gives
    bias-corrected moments g and g^2 at every step (Kingma and Ba), so each of
    the first steps moves every parameter by exactly -lr * sign(g)."""
    p = _params(4)
    g = np.random.default_rng(4).normal(size=mlp.NPARAM)
    m1 = np.zeros_like(p)
    m2 = np.zeros_like(p)
    q = p
    for step in (1, 2, 3):
        q, m1, m2 = mlp.adam_step(q, g, m1, m2, step, lr=0.01, eps=0.0)
        assert np.allclose(q, p - 0.01 * step * np.sign(g), rtol=0, atol=1e-12), step


def _count_at_or_below(spl, key):
    """Brute force: how many splitters are <= key (plain Python integers)."""
    c = 0
    for s in spl:
        if int(s) <= int(key):
            c += 1
    return c


@pytest.mark.parametrize("seed", range(6))
def test_bucket_function_brute_force(seed):
    """Small splitter arrays with repeated values, and keys equal to splitters,
    below the first and above the last: the bucket is the number of splitters
    at or below the key."""
    rng = np.random.default_rng(50 + seed)
    m = int(rng.integers(1, 12))
    spl = np.sort(rng.integers(3, 20, m)).astype(np.uint64)
    keys = np.concatenate([spl, np.arange(0, 24)]).astype(np.uint64)
    rng.shuffle(keys)
    got = mlp.buckets_from_splitters(keys, spl)
    want = [_count_at_or_below(spl, k) for k in keys]
    assert [int(b) for b in got] == want


def test_bucket_function_special_cases():
    spl = np.array([5, 5, 9], dtype=np.uint64)
    assert list(mlp.buckets_from_splitters(np.array([4, 5, 6, 9, 10], dtype=np.uint64), spl)) == [0, 2, 2, 3, 3]
    assert list(mlp.buckets_from_splitters(np.array([0, 7], dtype=np.uint64), np.array([], dtype=np.uint64))) == [0, 0]
    top = np.uint64((1 << 53) - 1)                      # the largest 53-bit prefix
    assert int(mlp.buckets_from_splitters(np.array([top], dtype=np.uint64), np.array([top], dtype=np.uint64))[0]) == 1


def test_bucket_function_monotone_and_tie_consistent():
    rng = np.random.default_rng(5)
    spl = np.sort(rng.integers(0, 1 << 40, 4095).astype(np.uint64))
    e = np.sort(rng.integers(0, 1 << 40, 100000).astype(np.uint64))
    b = mlp.buckets_from_splitters(e, spl)
    assert np.all(np.diff(b) >= 0) and b.min() >= 0 and b.max() <= 4095
    # equal keys share a bucket
    dup = np.repeat(e[:1000], 3)
    bd = mlp.buckets_from_splitters(dup, spl)
    assert np.array_equal(bd[0::3], bd[1::3]) and np.array_equal(bd[1::3], bd[2::3])
