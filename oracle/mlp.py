"""Oracle for the learned-splitter path -- TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper has no learned component; this restates, in float64 NumPy, what the
library's learned path computes, so that the GPU kernels can be compared with
it step by step:

* the network: 1 input, two tanh layers of 32 units, one tanh output unit;
  parameters packed as [w1(32), b1(32), W2(32x32, row j = inputs of unit j),
  b2(32), w3(32), b3(1)] -- 1153 numbers.  It is the second stage of the CDF
  model: its input is the first-stage coordinate x (linear interpolation
  through 64 sample-quantile intervals) and its output the correction r, so
  that the CDF estimate is x + r / 64 (the correction stays inside one
  first-stage interval);
* the loss: mean squared error to the target correction 64 (t - x);
* its gradient (backpropagation written out by hand) -- pinned in the tests
  by central finite differences of the loss, which share no code with it;
* one Adam step;
* the integer bucket function defined by a splitter array: the number of
  splitters at or below a key's 53-bit order-mapped prefix.

The final result of the learned sort is the plain stable sort, so it is
checked against ``oracle.stable_sort``, not against anything here.
"""
from __future__ import annotations

import numpy as np

H = 32
NPARAM = H + H + H * H + H + H + 1
W1, B1, W2, B2, W3, B3 = 0, H, 2 * H, 2 * H + H * H, 3 * H + H * H, 4 * H + H * H


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[W1:B1], p[B1:W2], p[W2:B2].reshape(H, H), p[B2:W3], p[W3:B3], p[B3])


NKNOTS = 64


def forward(p, x):
    """y = tanh(w3 . tanh(W2 tanh(w1 x + b1) + b2) + b3) for every x."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.tanh(np.outer(x, w1) + b1)            # (m, H)
    h2 = np.tanh(h1 @ w2.T + b2)                  # (m, H)
    z3 = h2 @ w3 + b3                             # (m,)
    y = np.tanh(z3)
    return y, (x, h1, h2)


def cdf_estimate(p, x):
    """The two-stage CDF estimate x + net(x) / 64."""
    y, _ = forward(p, x)
    return np.asarray(x, dtype=np.float64) + y / NKNOTS


def loss(p, x, t):
    y, _ = forward(p, x)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def loss_grad(p, x, t):
    """Mean squared error and its gradient with respect to the packed params."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    y, (x, h1, h2) = forward(p, x)
    t = np.asarray(t, dtype=np.float64)
    m = x.size
    dy = 2.0 * (y - t) / m                       # dL/dy
    dz3 = dy * (1.0 - y * y)                     # tanh'
    g_w3 = h2.T @ dz3
    g_b3 = dz3.sum()
    dz2 = np.outer(dz3, w3) * (1.0 - h2 ** 2)    # (m, H)
    g_w2 = dz2.T @ h1                            # row j, column i
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ w2) * (1.0 - h1 ** 2)           # (m, H)
    g_w1 = dz1.T @ x
    g_b1 = dz1.sum(axis=0)
    g = np.concatenate([g_w1, g_b1, g_w2.ravel(), g_b2, g_w3, [g_b3]])
    return float(np.mean((y - t) ** 2)), g


def adam_step(p, g, m1, m2, step, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), step counted from 1.  Returns new p, m1, m2."""
    m1 = beta1 * m1 + (1 - beta1) * g
    m2 = beta2 * m2 + (1 - beta2) * g * g
    mh = m1 / (1 - beta1 ** step)
    vh = m2 / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2


def buckets_from_splitters(e53, spl53):
    """Bucket of each key: the number of splitters at or below it (monotone, so
    equal keys always share a bucket)."""
    return np.searchsorted(np.asarray(spl53, dtype=np.uint64), np.asarray(e53, dtype=np.uint64), side="right")
