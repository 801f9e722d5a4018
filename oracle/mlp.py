"""FP64 NumPy multilayer perceptron: forward pass, backward pass and AdamW step.  Test
infrastructure only (the reference for the GPU surrogate kernels).

Model: x -> h_1 = GELU(W_1 x + b_1) -> ... -> y = W_L h_{L-1} + b_L, GELU(z) = z (1 + erf(z/sqrt 2)) / 2.
Loss: mean over batch x outputs of (y - t)^2.
AdamW (Loshchilov & Hutter, decoupled weight decay): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
p -= lr (m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps) + wd p), weight decay on weight matrices only.
Parameters are one flat vector: for each layer, W (out x in, row-major) then b.

Pinned by tests/test_oracle_mlp.py: gradients against central finite differences, GELU against
math.erf, and the first AdamW step against its closed form.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def layout(dims: List[int]):
    """[(w_offset, b_offset, in, out)] for consecutive layer sizes dims."""
    out, off = [], 0
    for i, o in zip(dims[:-1], dims[1:]):
        out.append((off, off + i * o, i, o))
        off += i * o + o
    return out, off


def unpack(params, dims):
    lay, _ = layout(dims)
    return [(params[w:w + i * o].reshape(o, i), params[b:b + o]) for w, b, i, o in lay]


def forward(params, dims, X, keep=False):
    zs, hs = [], [X]
    h = X
    layers = unpack(params, dims)
    for li, (W, b) in enumerate(layers):
        z = h @ W.T + b
        zs.append(z)
        h = z if li == len(layers) - 1 else gelu(z)
        hs.append(h)
    return (h, zs, hs) if keep else h


def loss_and_grad(params, dims, X, T):
    Y, zs, hs = forward(params, dims, X, keep=True)
    n = Y.size
    loss = float(np.sum((Y - T) ** 2) / n)
    lay, total = layout(dims)
    g = np.zeros(total)
    d = 2.0 * (Y - T) / n                       # dL/dy
    layers = unpack(params, dims)
    for li in range(len(layers) - 1, -1, -1):
        w, b, i, o = lay[li]
        g[w:w + i * o] = (d.T @ hs[li]).reshape(-1)   # dL/dW = d^T h_{l-1}
        g[b:b + o] = d.sum(axis=0)
        if li > 0:
            d = (d @ layers[li][0]) * gelu_grad(zs[li - 1])
    return loss, g


class AdamW:
    def __init__(self, dims, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
        self.lay, total = layout(dims)
        self.m = np.zeros(total)
        self.v = np.zeros(total)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps, self.wd = lr, b1, b2, eps, wd
        self.decay = np.zeros(total)
        for w, b, i, o in self.lay:
            self.decay[w:w + i * o] = 1.0

    def step(self, p, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return p - self.lr * (mh / (np.sqrt(vh) + self.eps) + self.wd * self.decay * p)
