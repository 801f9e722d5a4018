"""Channel representations (Sec. II.A and Sec. III).  FP64 NumPy.  Test infrastructure only.

Pinned by tests/test_oracle_channels.py against the depolarizing Kraus set and
chi matrix printed in Sec. II.A (tests/golden/depolarizing_chi.txt), the
amplitude-damping chi matrix in closed form, CPTP and rank invariants, and the
equality of superoperators under a Kraus -> chi -> Kraus round trip.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np

_P1 = (
    np.eye(2, dtype=np.complex128),
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


class ChannelError(ValueError):
    """Raised for a process matrix that is not Hermitian, not trace preserving or not CP."""


def pauli_basis(nq: int) -> List[np.ndarray]:
    """Unnormalised Pauli strings sigma_m, m = sum_j a_j 4^(nq-1-j) (first qubit most significant)."""
    basis = [np.ones((1, 1), dtype=np.complex128)]
    for _ in range(nq):
        basis = [np.kron(b, p) for b in basis for p in _P1]
    return basis


def vec(A: np.ndarray) -> np.ndarray:
    """|A>> with the row-major convention vec(A)[i*d + j] = A[i, j]."""
    return np.asarray(A).reshape(-1)


def unvec(v: np.ndarray, d: int) -> np.ndarray:
    return np.asarray(v).reshape(d, d)


def apply_chi(chi: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """eps(rho) = sum_mn chi_mn sigma_m rho sigma_n^dagger  (Eq. chi)."""
    d = rho.shape[0]
    nq = int(round(math.log2(d)))
    basis = pauli_basis(nq)
    out = np.zeros_like(rho, dtype=np.complex128)
    for m, sm in enumerate(basis):
        for n, sn in enumerate(basis):
            if chi[m, n] != 0:
                out += chi[m, n] * (sm @ rho @ sn.conj().T)
    return out


def check_process_matrix(chi: np.ndarray, nq: int, tol_herm: float = 1e-10, tol_trace: float = 1e-8) -> None:
    """Hermiticity and Tr(chi) = 1 (trace preservation in the unnormalised Pauli basis)."""
    chi = np.asarray(chi, dtype=np.complex128)
    if chi.shape != (4 ** nq, 4 ** nq):
        raise ChannelError(f"chi must be {4 ** nq}x{4 ** nq}")
    if not np.all(np.isfinite(chi)):
        raise ChannelError("chi has non-finite entries")
    if np.max(np.abs(chi - chi.conj().T)) > tol_herm:
        raise ChannelError("chi is not Hermitian")
    if abs(np.trace(chi).real - 1.0) > tol_trace or abs(np.trace(chi).imag) > tol_trace:
        raise ChannelError("Tr(chi) != 1: not trace preserving")


def chi_to_choi(chi: np.ndarray, nq: int) -> np.ndarray:
    """Lambda = sum_mn chi_mn |sigma_m>> <<sigma_n|  (Sec. III, change of basis)."""
    basis = pauli_basis(nq)
    d2 = 4 ** nq
    lam = np.zeros((d2, d2), dtype=np.complex128)
    for m in range(d2):
        for n in range(d2):
            lam += chi[m, n] * np.outer(vec(basis[m]), vec(basis[n]).conj())
    return lam


def choi_to_kraus(lam: np.ndarray, nq: int, tol: float = 1e-12, neg_tol: float = 1e-8) -> List[np.ndarray]:
    """Lambda = sum_i eta_i |psi_i><psi_i|, K_i = sqrt(eta_i) unvec(psi_i)  (Sec. III).

    Kraus operators are ordered by descending eta; eta <= tol * max(eta) is pruned
    (the paper prunes by descending eigenvalue).  A negative mass (sum of |eta| over
    negative eta) above neg_tol means the map is not completely positive.
    """
    d = 2 ** nq
    eta, psi = np.linalg.eigh(lam)
    order = np.argsort(-eta, kind="stable")
    eta, psi = eta[order], psi[:, order]
    if -np.sum(eta[eta < 0]) > neg_tol:
        raise ChannelError("Choi matrix has negative eigenvalues: not completely positive")
    emax = max(float(eta[0]), 0.0)
    keep = [i for i in range(len(eta)) if eta[i] > tol * emax and eta[i] > 0]
    return [math.sqrt(eta[i]) * unvec(psi[:, i], d) for i in keep]


def chi_to_kraus(chi: np.ndarray, nq: int, tol: float = 1e-12) -> List[np.ndarray]:
    """chi -> Choi -> Kraus, with the input and output checks of a CPTP channel."""
    check_process_matrix(chi, nq)
    kraus = choi_to_kraus(chi_to_choi(np.asarray(chi, dtype=np.complex128), nq), nq, tol)
    if not is_trace_preserving(kraus, 1e-8):
        raise ChannelError("sum_i K_i^dagger K_i != I")
    return kraus


def superop(kraus) -> np.ndarray:
    """S = sum_i K_i (x) conj(K_i), so that vec(sum_i K_i rho K_i^dag) = S vec(rho) (row-major vec)."""
    return sum(np.kron(K, K.conj()) for K in kraus)


def is_trace_preserving(kraus, tol: float = 1e-12) -> bool:
    d = kraus[0].shape[0]
    s = sum(K.conj().T @ K for K in kraus)
    return float(np.max(np.abs(s - np.eye(d)))) <= tol
