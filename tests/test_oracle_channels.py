"""Pins for the chi -> Choi -> Kraus conversion of the CPU reference (Sec. III) and for the
input generator's Kraus -> chi synthesis."""
import math
import os

import numpy as np
import pytest

from oracle import channels as C
from paper_2508_07610_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _printed_depolarizing_kraus(p):
    # Typed from the Kraus set printed in Sec. II.A, independently of workloads.depolarizing_1q.
    s0, s1 = math.sqrt(1 - 3 * p / 4), math.sqrt(p / 4)
    return [s0 * np.array([[1, 0], [0, 1]], complex), s1 * np.array([[0, 1], [1, 0]], complex),
            s1 * np.array([[0, -1j], [1j, 0]], complex), s1 * np.array([[1, 0], [0, -1]], complex)]


def _golden_depol():
    rows = []
    for line in open(os.path.join(GOLDEN, "depolarizing_chi.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return rows


@pytest.mark.parametrize("row", _golden_depol())
def test_depolarizing_chi_is_the_printed_diagonal(row):
    p, diag = row[0], row[1:]
    chi = W.kraus_to_chi(_printed_depolarizing_kraus(p))
    assert np.allclose(chi, np.diag(diag), atol=1e-15)
    assert np.allclose(W.kraus_to_chi(W.depolarizing_1q(p)), np.diag(diag), atol=1e-15)


@pytest.mark.parametrize("row", _golden_depol())
def test_depolarizing_chi_to_kraus_gives_the_printed_channel(row):
    p, diag = row[0], row[1:]
    kraus = C.chi_to_kraus(np.diag(diag).astype(complex), 1)
    assert np.allclose(C.superop(kraus), C.superop(_printed_depolarizing_kraus(p)), atol=1e-14)
    rank = sum(1 for d in diag if d > 0)
    assert len(kraus) == rank
    # the paper prunes by descending eigenvalue: the first Kraus operator carries weight 1 - 3p/4 (p < 1)
    if 0 < p < 1:
        assert abs(np.linalg.norm(kraus[0]) ** 2 / 2 - (1 - 3 * p / 4)) < 1e-14


@pytest.mark.parametrize("g", [0.0, 2e-3, 0.1, 0.7, 1.0])
def test_amplitude_damping_chi_closed_form(g):
    # K0 = diag(1, s), K1 = sqrt(g)|0><1|, s = sqrt(1-g).  Expanding in I, X, Y, Z by hand:
    # K0 = (1+s)/2 I + (1-s)/2 Z,  K1 = sqrt(g)/2 (X + iY), so
    s = math.sqrt(1 - g)
    expect = np.zeros((4, 4), complex)
    expect[0, 0] = (1 + s) ** 2 / 4
    expect[3, 3] = (1 - s) ** 2 / 4
    expect[0, 3] = expect[3, 0] = (1 + s) * (1 - s) / 4  # = g/4
    expect[1, 1] = expect[2, 2] = g / 4
    expect[1, 2] = -1j * g / 4
    expect[2, 1] = 1j * g / 4
    chi = W.kraus_to_chi(W.amplitude_damping(g))
    assert np.allclose(chi, expect, atol=1e-15)
    assert abs(np.trace(chi) - 1) < 1e-15
    kraus = C.chi_to_kraus(chi, 1)
    assert np.allclose(C.superop(kraus), C.superop(W.amplitude_damping(g)), atol=1e-13)
    assert len(kraus) == (1 if g in (0.0,) else 2)


@pytest.mark.parametrize("nq,rank,seed", [(1, 1, 0), (1, 2, 1), (1, 4, 2), (2, 1, 3), (2, 3, 4), (2, 7, 5), (2, 16, 6)])
def test_round_trip_random_channels(nq, rank, seed):
    rng = np.random.default_rng(seed)
    kraus_in = W.random_channel_kraus(nq, rank, rng)
    chi = W.kraus_to_chi(kraus_in)
    kraus = C.chi_to_kraus(chi, nq)
    assert len(kraus) == rank                      # #Kraus = rank of the Choi matrix
    assert C.is_trace_preserving(kraus, 1e-12)     # sum K^dag K = I
    assert np.allclose(C.superop(kraus), C.superop(kraus_in), atol=1e-13)
    # Eq. (chi) applied directly agrees with the Kraus form on a random state
    d = 2 ** nq
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    rho = z @ z.conj().T
    rho /= np.trace(rho)
    assert np.allclose(C.apply_chi(chi, rho), sum(K @ rho @ K.conj().T for K in kraus), atol=1e-13)
    # Choi matrix is positive semidefinite with trace d
    lam = C.chi_to_choi(chi, nq)
    assert np.linalg.eigvalsh(lam).min() > -1e-13
    assert abs(np.trace(lam) - d) < 1e-12


def test_kraus_sorted_by_descending_weight():
    rng = np.random.default_rng(7)
    chi = W.kraus_to_chi(W.random_channel_kraus(2, 9, rng))
    w = [np.linalg.norm(K) ** 2 for K in C.chi_to_kraus(chi, 2)]
    assert all(w[i] >= w[i + 1] - 1e-15 for i in range(len(w) - 1))


def test_invalid_process_matrices_raise():
    good = W.kraus_to_chi(W.depolarizing_1q(0.1))
    with pytest.raises(C.ChannelError):
        C.chi_to_kraus(good * 1.1, 1)                     # Tr chi != 1
    bad = good.copy()
    bad[0, 1] += 0.1
    with pytest.raises(C.ChannelError):
        C.chi_to_kraus(bad, 1)                            # not Hermitian
    notcp = np.diag([1.2, -0.2, 0.0, 0.0]).astype(complex)
    with pytest.raises(C.ChannelError):
        C.chi_to_kraus(notcp, 1)                          # negative Choi eigenvalue
    with pytest.raises(C.ChannelError):
        C.chi_to_kraus(np.full((4, 4), np.nan, complex), 1)


def test_two_qubit_depolarizing_chi_and_pauli_order():
    p = 0.05
    chi = W.kraus_to_chi(W.depolarizing_2q(p))
    expect = np.full(16, p / 16)
    expect[0] = 1 - 15 * p / 16
    assert np.allclose(chi, np.diag(expect), atol=1e-15)
    # m = 4a + b with a on the first qubit: X (x) I is index 4, I (x) X is index 1
    basis = C.pauli_basis(2)
    X = np.array([[0, 1], [1, 0]], complex)
    assert np.allclose(basis[4], np.kron(X, np.eye(2)))
    assert np.allclose(basis[1], np.kron(np.eye(2), X))
