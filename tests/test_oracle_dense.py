"""Pins for the dense density-matrix simulator against closed forms and the paper's examples."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import dense as D
from paper_2508_07610_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
IDEAL1 = np.diag([1, 0, 0, 0]).astype(complex)            # chi of the identity channel (1q)
IDEAL2 = np.zeros((16, 16), complex)
IDEAL2[0, 0] = 1


def _ghz(n):
    rho = D.zero_state(n)
    rho = D.apply_noisy_gate(rho, n, [0], W.hadamard(), IDEAL1)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], complex)
    for q in range(n - 1):
        rho = D.apply_noisy_gate(rho, n, [q, q + 1], cnot, IDEAL2)
    return rho


@pytest.mark.parametrize("n", [2, 3, 5])
@pytest.mark.parametrize("p", [0.0, 0.01, 0.3])
def test_ghz_uniform_depolarizing_closed_form(n, p):
    rho = _ghz(n)
    chi = W.kraus_to_chi(W.depolarizing_1q(p))
    for q in range(n):
        rho = D.apply_noisy_gate(rho, n, [q], np.eye(2), chi)
    F = 0.5 * ((1 - p / 2) ** n + (p / 2) ** n + (1 - p) ** n)
    assert abs(D.ghz_fidelity(rho, n) - F) < 1e-13
    assert abs(D.expect_zz(rho, n, 0, n - 1) - (1 - p) ** 2) < 1e-13
    assert abs(D.trace(rho) - 1) < 1e-13


@pytest.mark.parametrize("n", [2, 4, 6])
@pytest.mark.parametrize("g", [0.0, 2e-3, 0.25])
def test_ghz_uniform_amplitude_damping_closed_form(n, g):
    rho = _ghz(n)
    chi = W.kraus_to_chi(W.amplitude_damping(g))
    for q in range(n):
        rho = D.apply_noisy_gate(rho, n, [q], np.eye(2), chi)
    F = 0.25 * (1 + g ** n + (1 - g) ** n) + 0.5 * (1 - g) ** (n / 2)
    assert abs(D.ghz_fidelity(rho, n) - F) < 1e-13


def test_product_state_purity():
    rng = np.random.default_rng(3)
    n = 4
    rho = D.zero_state(n)
    prod = 1.0
    for q in range(n):
        p = rng.uniform(0, 0.6)
        rho = D.apply_noisy_gate(rho, n, [q], W.random_unitary(2, rng), W.kraus_to_chi(W.depolarizing_1q(p)))
        r = 1 - p                                    # Bloch length after depolarizing a pure state
        prod *= (1 + r * r) / 2
    assert abs(D.purity(rho) - prod) < 1e-13


def test_cnot_compiled_from_cz_and_ry_fig7():
    # Fig. 7: CNOT = CZ flanked by two RY gates on the target.
    for a, b in itertools.product([0, 1], repeat=2):
        rho = D.zero_state(2)
        if a:
            rho = D.apply_unitary(rho, 2, [0], np.array([[0, 1], [1, 0]], complex))
        if b:
            rho = D.apply_unitary(rho, 2, [1], np.array([[0, 1], [1, 0]], complex))
        rho = D.apply_unitary(rho, 2, [1], W.ry(-math.pi / 2))
        rho = D.apply_unitary(rho, 2, [0, 1], W.cz())
        rho = D.apply_unitary(rho, 2, [1], W.ry(math.pi / 2))
        out = int(np.argmax(np.real(np.diag(rho))))
        assert out == 2 * a + (b ^ a)
        assert abs(np.real(rho[out, out]) - 1) < 1e-14


def _golden_maxcut():
    d = {}
    for line in open(os.path.join(GOLDEN, "maxcut_q4.txt")):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            d[k] = v
    edges = [tuple(int(x) for x in e.split("-")) for e in d["edges"]]
    return edges, int(d["maxcut"][0]), d["optimal"]


def test_maxcut_4cycle_brute_force_fig12():
    edges, best, optimal = _golden_maxcut()
    n = 4
    cuts = {}
    for bits in itertools.product([0, 1], repeat=n):
        rho = D.zero_state(n)
        for q, b in enumerate(bits):
            if b:
                rho = D.apply_unitary(rho, n, [q], np.array([[0, 1], [1, 0]], complex))
        s = "".join(map(str, bits))
        cuts[s] = D.maxcut_expectation(rho, n, edges)
        direct = sum(1 for i, k in edges if bits[i] != bits[k])   # C(z) of Eq. (maxcut)
        assert abs(cuts[s] - direct) < 1e-14
    assert max(cuts.values()) == best
    assert sorted(s for s, c in cuts.items() if c == best) == sorted(optimal)
    # uniform superposition H^n|0>: every edge cut with probability 1/2
    rho = D.zero_state(n)
    for q in range(n):
        rho = D.apply_unitary(rho, n, [q], W.hadamard())
    assert abs(D.maxcut_expectation(rho, n, edges) - len(edges) / 2) < 1e-14


@pytest.mark.parametrize("seed", range(4))
def test_chi_application_matches_kraus_sum(seed):
    # The generator's input Kraus sets and Eq. (chi) describe the same map on a random 3-qubit state.
    rng = np.random.default_rng(100 + seed)
    n = 3
    z = rng.normal(size=(8, 8)) + 1j * rng.normal(size=(8, 8))
    rho = z @ z.conj().T
    rho /= np.trace(rho)
    U = W.random_unitary(4, rng)
    kr = W.random_channel_kraus(2, 5, rng)
    out = D.apply_noisy_gate(rho, n, [1, 2], U, W.kraus_to_chi(kr))
    ref = np.zeros_like(rho)
    for K in kr:
        full = np.kron(np.eye(2), K @ U)
        ref += full @ rho @ full.conj().T
    assert np.allclose(out, ref, atol=1e-13)


# ------------------------------------------------------------------ Uhlmann fidelity (Sec. IV.C)
def _random_state(d, rank, rng):
    G = rng.normal(size=(d, rank)) + 1j * rng.normal(size=(d, rank))
    r = G @ G.conj().T
    return r / np.trace(r).real


def test_uhlmann_fidelity_closed_forms():
    rng = np.random.default_rng(4)
    d = 8
    rho = _random_state(d, d, rng)
    # identical states
    assert abs(D.uhlmann_fidelity(rho, rho) - 1) < 1e-12
    # a pure state against any state: <psi| sigma |psi>.  The square root of the rank-one state's
    # rounding-level zero eigenvalues (about 1e-17) is about sqrt(u) = 1e-8, hence the tolerance
    psi = rng.normal(size=d) + 1j * rng.normal(size=d)
    psi /= np.linalg.norm(psi)
    pure = np.outer(psi, psi.conj())
    assert abs(D.uhlmann_fidelity(pure, rho) - (psi.conj() @ rho @ psi).real) < 1e-7
    # commuting (diagonal) states: the classical fidelity (sum sqrt(p q))^2
    p, q = rng.dirichlet(np.ones(d)), rng.dirichlet(np.ones(d))
    assert abs(D.uhlmann_fidelity(np.diag(p), np.diag(q)) - np.sum(np.sqrt(p * q)) ** 2) < 1e-12
    # against the maximally mixed state: (sum sqrt(lambda))^2 / d
    lam = np.linalg.eigvalsh(rho)
    assert abs(D.uhlmann_fidelity(rho, np.eye(d) / d) - np.sum(np.sqrt(np.clip(lam, 0, None))) ** 2 / d) < 1e-12
    # symmetric, unitarily invariant, in [0, 1], scale-free
    sig = _random_state(d, d, rng)
    U = W.random_unitary(d, rng)
    f = D.uhlmann_fidelity(rho, sig)
    assert abs(f - D.uhlmann_fidelity(sig, rho)) < 1e-10
    assert abs(f - D.uhlmann_fidelity(U @ rho @ U.conj().T, U @ sig @ U.conj().T)) < 1e-10
    assert 0 <= f <= 1 and abs(f - D.uhlmann_fidelity(3 * rho, 0.5 * sig)) < 1e-12
