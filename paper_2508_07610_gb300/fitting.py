"""Gradient-based fitting of noise-model strengths through the MPDO (Sec. IV.A, Fig. 10).

The paper fits the parameters of a standard noise model so that the simulated output distribution of
a circuit matches measured data in Jensen-Shannon divergence.  Here the model is the depolarizing
channel on every gate plus amplitude damping on single-qubit gates, theta = (p1, gamma, p2), passed to
the library as process matrices (Eq. chi).  The loss JSD(p(theta), target) and its gradient come from
the GPU MPDO: the 2P + 1 parameter vectors of a central-difference gradient (steps in log theta) run
as the chains of one batched handle, each chain with its own channels, and every chain's bitstring
distribution is read in one batched prefix contraction (mpdo_distribution) and compared with mpdo_jsd.  The optimiser (Adam in log theta, so strengths stay
positive) runs on the host.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

from . import mpdo as G
from . import workloads as W

PARAMS = ("p1", "gamma", "p2")


def model_channels(theta) -> Tuple[np.ndarray, np.ndarray]:
    """Process matrices of the standard model: 1q AD(gamma) o DEP(p1), 2q DEP2(p2)."""
    p1, g, p2 = theta
    chi1 = W.kraus_to_chi(W.compose(W.amplitude_damping(g), W.depolarizing_1q(p1)))
    chi2 = W.kraus_to_chi(W.depolarizing_2q(p2))
    return chi1, chi2


class NoiseModelFit:
    """The circuit is a list of ideal gates (kind, qubit, U) on n qubits; every 1q gate is followed by
    the model's 1q channel and every 2q gate by its 2q channel."""

    def __init__(self, n: int, gates: Sequence[Tuple[int, int, np.ndarray]], chi_max: int = 16, kappa_max: int = 8,
                 prec: str = "fp64", step: float = 1e-3):
        if n > 15:
            raise ValueError("the loss reads the full 2^n distribution: n <= 15")
        self.n, self.gates = n, list(gates)
        self.chi_max, self.kappa_max, self.prec, self.step = chi_max, kappa_max, prec, step

    def distributions(self, thetas: np.ndarray) -> np.ndarray:
        """Bitstring distributions (len(thetas) x 2^n, qubit 0 most significant), one chain per theta."""
        B = len(thetas)
        st = G.MPDO(self.n, self.chi_max, self.kappa_max, self.prec, batch=B)
        chis = [model_channels(t) for t in thetas]
        ch1 = st.channels(1, [c[0] for c in chis])
        ch2 = st.channels(2, [c[1] for c in chis])
        for kind, q, U in self.gates:
            (st.apply_1q if kind == 1 else st.apply_2q)(q, U, ch1 if kind == 1 else ch2)
        out = st.distribution()
        ch1.free()
        ch2.free()
        st.free()
        return out

    def loss_and_grad(self, theta, target) -> Tuple[float, np.ndarray]:
        """JSD(p(theta), target) and its gradient with respect to log theta (central differences)."""
        x = np.log(np.asarray(theta, dtype=np.float64))
        P = len(x)
        pts = [x] + [x + s * self.step * np.eye(P)[i] for i in range(P) for s in (1, -1)]
        d = self.distributions(np.exp(np.array(pts)))
        f = [G.jsd(d[j], target) for j in range(len(pts))]
        g = np.array([(f[1 + 2 * i] - f[2 + 2 * i]) / (2 * self.step) for i in range(P)])
        return f[0], g

    def fit(self, theta0, target, iters: int = 60, lr: float = 0.15) -> List[dict]:
        """Adam in log theta with a cosine learning-rate schedule; returns the history."""
        x = np.log(np.asarray(theta0, dtype=np.float64))
        m = np.zeros_like(x)
        v = np.zeros_like(x)
        hist = []
        for it in range(iters):
            f, g = self.loss_and_grad(np.exp(x), target)
            hist.append({"iter": it, "jsd": f, "theta": np.exp(x).tolist()})
            m = 0.9 * m + 0.1 * g
            v = 0.999 * v + 0.001 * g * g
            lr_t = lr * 0.5 * (1 + math.cos(math.pi * it / iters))
            x = x - lr_t * (m / (1 - 0.9 ** (it + 1))) / (np.sqrt(v / (1 - 0.999 ** (it + 1))) + 1e-12)
        f, _ = self.loss_and_grad(np.exp(x), target)
        hist.append({"iter": iters, "jsd": f, "theta": np.exp(x).tolist()})
        return hist
