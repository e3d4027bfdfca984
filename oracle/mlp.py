"""A plain multilayer perceptron in FP64: forward pass, gradients of the mean squared error, Adam.

Test infrastructure only (see the package header).  The network is not from the paper: it is the
learned warm start that proposes an interval's starting gains from earlier solutions (the paper's
Sect. 3.4 notes that gains do not vary arbitrarily in time and frequency, which is what
makes earlier solutions informative).  Everything here is the textbook definition:

  h1 = relu(x W1 + b1),  h2 = relu(h1 W2 + b2),  y = h2 W3 + b3,
  loss = mean over all n * out entries of (y - t)^2,

with gradients by the chain rule (the derivative of relu taken as 0 at 0) and Adam with
bias correction (Kingma & Ba 2015, Algorithm 1).  ``forward_bf16`` is the inference precision of
the warm start: weights, inputs and hidden activations rounded to bfloat16 (round to nearest, ties
to even, from float32), products and sums exact here (FP64).

Parameters are one flat vector: W1 [in][h1] | b1 [h1] | W2 [h1][h2] | b2 [h2] | W3 [h2][out] | b3 [out],
each matrix row-major.
"""
from __future__ import annotations

import numpy as np


def n_params(dims):
    i, h1, h2, o = dims
    return i * h1 + h1 + h1 * h2 + h2 + h2 * o + o


def unpack(params, dims):
    """Views W1, b1, W2, b2, W3, b3 of the flat parameter vector."""
    i, h1, h2, o = dims
    p = np.asarray(params, np.float64)
    sizes = [i * h1, h1, h1 * h2, h2, h2 * o, o]
    shapes = [(i, h1), (h1,), (h1, h2), (h2,), (h2, o), (o,)]
    out, at = [], 0
    for sz, sh in zip(sizes, shapes):
        out.append(p[at:at + sz].reshape(sh))
        at += sz
    return out


def init_params(dims, rng):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases."""
    i, h1, h2, o = dims
    parts = [rng.normal(0.0, np.sqrt(2.0 / i), i * h1), np.zeros(h1),
             rng.normal(0.0, np.sqrt(2.0 / h1), h1 * h2), np.zeros(h2),
             rng.normal(0.0, np.sqrt(2.0 / h2), h2 * o), np.zeros(o)]
    return np.concatenate(parts)


def forward(params, dims, x):
    """Returns (h1, h2, y), all float64."""
    W1, b1, W2, b2, W3, b3 = unpack(params, dims)
    x = np.asarray(x, np.float64)
    h1 = np.maximum(x @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    y = h2 @ W3 + b3
    return h1, h2, y


def bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(params, dims, x):
    """Output of the network with bfloat16 weights, inputs and hidden activations."""
    W1, b1, W2, b2, W3, b3 = (bf16(np.asarray(w, np.float32)) for w in unpack(params, dims))
    h1 = bf16(np.maximum(bf16(np.asarray(x, np.float32)) @ W1 + b1, 0.0))
    h2 = bf16(np.maximum(h1 @ W2 + b2, 0.0))
    return h2 @ W3 + b3


def loss_and_grad(params, dims, x, t):
    """Mean squared error and its gradient with respect to the flat parameter vector."""
    W1, b1, W2, b2, W3, b3 = unpack(params, dims)
    x = np.asarray(x, np.float64)
    t = np.asarray(t, np.float64)
    h1, h2, y = forward(params, dims, x)
    n, o = y.shape
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / (n * o)                  # d loss / d y
    gW3 = h2.T @ dy
    gb3 = dy.sum(axis=0)
    d2 = (dy @ W3.T) * (h2 > 0.0)                 # back through relu: pre-activation > 0 <=> h > 0
    gW2 = h1.T @ d2
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (h1 > 0.0)
    gW1 = x.T @ d1
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step >= 1); returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
