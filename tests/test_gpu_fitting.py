"""Fitting the strengths of the standard noise model through the GPU MPDO (Sec. IV.A, Fig. 10): the
JSD loss and its central-difference gradient against the dense oracle, and the fit recovering the
strengths that generated a target distribution (the dense oracle's, standing in for measured data)."""
import numpy as np
import pytest

from oracle import dense as OD
from oracle import mpdo as OM
from paper_2508_07610_gb300 import fitting as F
from paper_2508_07610_gb300 import mpdo as G
from paper_2508_07610_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _gates(n, rng, layers=3):
    gates = []
    for layer in range(layers):
        for q in range(n):
            gates.append((1, q, W.ry(rng.uniform(-np.pi, np.pi)) @ W.rz(rng.uniform(-np.pi, np.pi))))
        for q in range(layer % 2, n - 1, 2):
            gates.append((2, q, W.cz()))
    return gates


def _oracle_dist(n, gates, theta, caps=None):
    """Bitstring distribution of the dense oracle (exact), or of the MPDO oracle at the given caps."""
    chi1, chi2 = F.model_channels(theta)
    ops = [W.Op(k, q, U, 0 if k == 1 else 1) for k, q, U in gates]
    circ = W.Circuit(n, ops, [(1, chi1), (2, chi2)])
    rho = OD.run_circuit(circ) if caps is None else OM.run_circuit(circ, *caps).dense()
    return OD.probabilities(rho / np.trace(rho).real)


def test_loss_and_gradient_match_the_dense_oracle():
    rng = np.random.default_rng(3)
    n = 4
    gates = _gates(n, rng)
    fit = F.NoiseModelFit(n, gates, chi_max=16, kappa_max=32, prec="fp64")
    tstar = np.array([2e-3, 4e-3, 1.5e-2])
    target = _oracle_dist(n, gates, tstar)
    theta = 2.5 * tstar
    f, g = fit.loss_and_grad(theta, target)
    # parity with the MPDO oracle at the same caps (kappa_max = 32 cuts about 1.5e-5 of the weight
    # of this circuit's Kraus legs): FP64 probabilities agree to 1e-10, so the loss to about that and
    # its central difference over a step of 2e-3 in log theta to 1e-7
    caps = (16, 32)
    f_ref = G.jsd(_oracle_dist(n, gates, theta, caps), target)
    x = np.log(theta)
    g_ref = np.array([(G.jsd(_oracle_dist(n, gates, np.exp(x + 1e-3 * e), caps), target)
                       - G.jsd(_oracle_dist(n, gates, np.exp(x - 1e-3 * e), caps), target)) / 2e-3 for e in np.eye(3)])
    assert abs(f - f_ref) < 1e-10
    assert np.max(np.abs(g - g_ref)) < 1e-7
    # and close to the untruncated loss
    f_exact = G.jsd(_oracle_dist(n, gates, theta), target)
    assert abs(f - f_exact) < 1e-3 * f_exact
    assert f > 1e-4 and np.all(g > 0)  # too much noise: every strength should come down


def test_fit_recovers_the_generating_strengths():
    rng = np.random.default_rng(3)
    n = 4
    gates = _gates(n, rng)
    fit = F.NoiseModelFit(n, gates, chi_max=16, kappa_max=32, prec="fp64")
    tstar = np.array([2e-3, 4e-3, 1.5e-2])
    target = _oracle_dist(n, gates, tstar)
    hist = fit.fit(2.5 * tstar, target, iters=60, lr=0.15)
    ratio = np.array(hist[-1]["theta"]) / tstar
    print(f"fit: JSD {hist[0]['jsd']:.3e} -> {hist[-1]['jsd']:.3e}, theta / theta* = {np.round(ratio, 3)}")
    assert hist[-1]["jsd"] < 1e-3 * hist[0]["jsd"]
    assert np.all(np.abs(np.log(ratio)) < 0.1)
