"""Pins for the FP64 MLP reference: finite differences, the erf definition of GELU, and the closed
form of the first AdamW step."""
import math

import numpy as np

from oracle import mlp as M


def test_gelu_is_the_erf_definition():
    for z in (-3.0, -0.7, 0.0, 0.4, 2.5):
        assert abs(M.gelu(np.array(z)) - 0.5 * z * (1 + math.erf(z / math.sqrt(2)))) < 1e-15
        h = 1e-6
        fd = (M.gelu(np.array(z + h)) - M.gelu(np.array(z - h))) / (2 * h)
        assert abs(M.gelu_grad(np.array(z)) - fd) < 1e-8


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    dims = [5, 7, 6, 3]
    _, total = M.layout(dims)
    p = rng.normal(scale=0.5, size=total)
    X = rng.normal(size=(11, 5))
    T = rng.normal(size=(11, 3))
    loss, g = M.loss_and_grad(p, dims, X, T)
    for idx in rng.choice(total, size=25, replace=False):
        e = np.zeros(total)
        e[idx] = 1e-6
        fd = (M.loss_and_grad(p + e, dims, X, T)[0] - M.loss_and_grad(p - e, dims, X, T)[0]) / 2e-6
        assert abs(fd - g[idx]) < 1e-7 * max(1.0, abs(fd))


def test_first_adamw_step_closed_form():
    dims = [2, 1]
    _, total = M.layout(dims)  # W (1 x 2) then b (1)
    p = np.array([0.5, -1.0, 0.25])
    g = np.array([0.3, -0.2, 0.1])
    opt = M.AdamW(dims, lr=1e-2, eps=1e-8, wd=0.1)
    q = opt.step(p, g)
    # t = 1: mhat = g, vhat = g^2, so the step is lr (g / (|g| + eps) + wd p) on weights, no decay on b
    expect = p - 1e-2 * (g / (np.abs(g) + 1e-8) + 0.1 * np.array([1, 1, 0]) * p)
    assert np.max(np.abs(q - expect)) < 1e-15
