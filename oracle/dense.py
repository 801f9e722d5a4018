"""Dense 2^n x 2^n density-matrix simulator.  FP64 NumPy.  Test infrastructure only.

This is the exact object the MPDO represents (Sec. II.C): with no truncation,
rho_out = E_L o ... o E_1 (|0..0><0..0|), each noisy gate being
E(rho) = eps(U rho U^dagger) with eps given by its process matrix through
Eq. (chi).  Channels are applied from chi directly, never through Kraus
operators, so this simulator is independent of the chi -> Kraus conversion.

Pinned by tests/test_oracle_dense.py against closed forms: GHZ fidelity and
<Z Z> under uniform depolarizing / amplitude damping, product-state purity, the
CNOT compilation of Fig. 7, and brute-force MaxCut on the 4-cycle of Fig. 12.
"""
from __future__ import annotations

import numpy as np

from .channels import pauli_basis


def zero_state(n: int) -> np.ndarray:
    rho = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
    rho[0, 0] = 1.0
    return rho


def local_superop_from_chi(chi: np.ndarray, nq: int) -> np.ndarray:
    """S[(i,j),(a,b)] = sum_mn chi_mn sigma_m[i,a] conj(sigma_n[j,b]): Eq. (chi) on one block."""
    basis = pauli_basis(nq)
    d = 2 ** nq
    S = np.zeros((d, d, d, d), dtype=np.complex128)
    for m, sm in enumerate(basis):
        for n, sn in enumerate(basis):
            if chi[m, n] != 0:
                S += chi[m, n] * np.einsum("ia,jb->ijab", sm, sn.conj())
    return S.reshape(d * d, d * d)


def apply_superop(rho: np.ndarray, n: int, S: np.ndarray, qubits) -> np.ndarray:
    """Apply a local superoperator S (on row-major vec of the local block) to `qubits`."""
    k = len(qubits)
    d = 2 ** k
    t = rho.reshape([2] * (2 * n))
    ket = list(qubits)
    bra = [n + q for q in qubits]
    rest = [i for i in range(2 * n) if i not in ket + bra]
    t = np.transpose(t, ket + bra + rest).reshape(d * d, -1)
    t = (S @ t).reshape([2] * (2 * k) + [2] * (2 * n - 2 * k))
    inv = np.argsort(ket + bra + rest)
    return np.transpose(t, inv).reshape(2 ** n, 2 ** n)


def apply_noisy_gate(rho: np.ndarray, n: int, qubits, U: np.ndarray, chi: np.ndarray) -> np.ndarray:
    """rho -> eps(U rho U^dag) on `qubits` (consecutive, first is most significant)."""
    nq = len(qubits)
    S = local_superop_from_chi(chi, nq) @ np.kron(U, U.conj())
    return apply_superop(rho, n, S, qubits)


def apply_unitary(rho: np.ndarray, n: int, qubits, U: np.ndarray) -> np.ndarray:
    return apply_superop(rho, n, np.kron(U, U.conj()), qubits)


def run_circuit(circuit) -> np.ndarray:
    """Simulate a workloads.Circuit exactly."""
    n = circuit.n
    rho = zero_state(n)
    for op in circuit.ops:
        if op.kind == 8:  # a bond-truncation directive: the exact state is left as it is
            continue
        nq, chi = circuit.chis[op.chan]
        qs = list(range(op.q, op.q + op.kind))
        rho = apply_noisy_gate(rho, n, qs, op.U, chi)
    return rho


# ---------------------------------------------------------------- readouts
def z_string(n: int, sites) -> np.ndarray:
    """Diagonal of prod_{i in sites} Z_i in the computational basis (qubit 0 = MSB)."""
    idx = np.arange(2 ** n)
    sign = np.ones(2 ** n)
    for s in sites:
        bit = (idx >> (n - 1 - s)) & 1
        sign = sign * (1 - 2 * bit)
    return sign


def trace(rho) -> float:
    return float(np.trace(rho).real)


def expect_zz(rho, n, i, j) -> float:
    return float(np.real(np.sum(np.diag(rho) * z_string(n, [i, j]))) / trace(rho))


def ghz_fidelity(rho, n) -> float:
    """<GHZ| rho |GHZ> / Tr rho with |GHZ> = (|0..0> + |1..1>)/sqrt(2)."""
    g = np.zeros(2 ** n, dtype=np.complex128)
    g[0] = g[-1] = 1 / np.sqrt(2)
    return float(np.real(g.conj() @ rho @ g) / trace(rho))


def purity(rho) -> float:
    return float(np.real(np.trace(rho @ rho)) / trace(rho) ** 2)


def maxcut_expectation(rho, n, edges) -> float:
    """sum over edges of (1 - <Z_i Z_k>) / 2  (Eqs. maxcut, maxcut_obj)."""
    return sum(0.5 * (1 - expect_zz(rho, n, i, k)) for i, k in edges)


def probabilities(rho) -> np.ndarray:
    return np.real(np.diag(rho)) / trace(rho)


def _psd_sqrt(rho: np.ndarray) -> np.ndarray:
    """The positive square root of a Hermitian PSD matrix through its eigendecomposition (negative
    rounding-level eigenvalues clipped to 0)."""
    w, V = np.linalg.eigh((rho + rho.conj().T) / 2)
    return (V * np.sqrt(np.clip(w, 0.0, None))) @ V.conj().T


def uhlmann_fidelity(rho: np.ndarray, sigma: np.ndarray) -> float:
    """F(rho, sigma) = (tr sqrt(sqrt(rho) sigma sqrt(rho)))^2 (Sec. IV.C, Eq. fidelity), both states
    normalised to unit trace first (the MPDO keeps the trace that truncation removed)."""
    r = rho / np.trace(rho).real
    s = sigma / np.trace(sigma).real
    sr = _psd_sqrt(r)
    M = sr @ s @ sr
    w = np.linalg.eigvalsh((M + M.conj().T) / 2)
    return float(np.sum(np.sqrt(np.clip(w, 0.0, None))) ** 2)
