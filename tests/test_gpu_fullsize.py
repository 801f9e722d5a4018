"""Parity at the benchmark's full size (n = 20, chi_max = 64, kappa_max = 8, two-qubit channel of
Kraus rank 16), where the CPU reference can only afford single updates.

A seeded random right-canonical chain with every bond at 64 and every Kraus leg at 8 is loaded into
both implementations; one noisy CZ update is applied; the discarded weights and the reduced density
matrix of the two touched qubits (a gauge-invariant output; with the centre on the pair it needs no
environment) are compared element by element.  A second test runs whole ansatz layers at full size
in the complex64 mode and in FP64 on the GPU and compares every <Z_i Z_j>.
"""
import math

import numpy as np
import pytest

from oracle import channels as OC
from oracle import mpdo as OM
from paper_2508_07610_gb300 import mpdo as G
from paper_2508_07610_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N, CHI, KAP = 20, 64, 8


def _pair_rdm(A1, A2):
    """rho[(p1 p2), (p1' p2')] of two adjacent sites whose environments are identities."""
    th = np.einsum("lanb,bcmr->lacnmr", A1, A2)  # [l, p1, p2, n1, n2, r]
    m = th.reshape(th.shape[0], 4, -1, th.shape[-1])
    return np.einsum("lxkr,lykr->xy", m, m.conj())


def _state(seed):
    rng = np.random.default_rng(seed)
    return W.random_right_canonical_sites(N, CHI, KAP, rng)


@pytest.fixture(scope="module")
def one_update():
    sites = _state(2026)
    chi2 = W.kraus_to_chi(W.compose(W.depolarizing_2q(1e-2), W.unitary_channel(W.zz_phase(0.013))))
    q = 9
    orc = OM.MPDO(N, CHI, KAP)
    orc.sites = [s.copy() for s in sites]
    orc.centre = 0
    orc.apply_2q(q, W.cz(), OC.chi_to_kraus(chi2, 2))
    return sites, chi2, q, orc


@pytest.mark.parametrize("batch", [1, 160])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-6), ("fp32", 1e-6)])
def test_single_update_full_size(prec, tol, batch, one_update):
    """batch = 160 runs the same update on 160 identical chains: more matrices than the GPU has SMs
    for the cluster QR, so the centre moves and the reduction take the blocked one-CTA-per-matrix QR."""
    sites, chi2, q, orc = one_update
    st = G.MPDO(N, CHI, KAP, prec, batch=batch)
    for i, s in enumerate(sites):
        st.set_site(i, s)
    st.set_centre(0)
    ch = st.channels(2, [chi2])
    st.apply_2q(q, W.cz(), ch)
    st.sync()

    bg, kg = st.dims()
    assert bg == orc.bond_dims() and kg == orc.kraus_dims()
    r_o = _pair_rdm(orc.sites[q], orc.sites[q + 1])
    scale = np.trace(r_o).real
    disc = st.discarded()
    zz = st.zz(q, q + 1)
    first = None
    for b in sorted({0, batch // 2, batch - 1}):
        d = disc[b]
        assert abs(d[0] - orc.discarded_chi) < tol, (b, d[0], orc.discarded_chi)
        assert abs(d[1] - orc.discarded_kappa) < tol, (b, d[1], orc.discarded_kappa)
        r_g = _pair_rdm(st.get_site(q, b), st.get_site(q + 1, b))
        err = np.max(np.abs(r_g - r_o)) / scale
        print(f"full-size single update {prec} batch {batch} chain {b}: rdm err {err:.2e}, "
              f"discarded {d[0]:.3e} / {d[1]:.3e}")
        assert err < tol
        assert abs(zz[b] - orc.expect_zz(q, q + 1)) < tol
        # identical chains give identical results
        if first is None:
            first = r_g
        else:
            assert np.array_equal(r_g, first)


def _perturbed(circ, rel, seed):
    """The same circuit with every chi matrix moved by a Hermitian, trace-free perturbation of
    relative size `rel` (a stand-in for rounding of the inputs)."""
    rng = np.random.default_rng(seed)
    out = W.Circuit(circ.n, circ.ops, [], circ.kraus, dict(circ.meta))
    for nq, chi in circ.chis:
        d = chi.shape[0]
        h = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
        h = (h + h.conj().T) / 2
        h -= np.trace(h) / d * np.eye(d)
        out.chis.append((nq, chi + rel * np.abs(chi).max() * h / np.abs(h).max()))
    return out


def test_complex64_layers_track_fp64_at_full_size():
    """Six ansatz layers of the benchmark workload (n = 20, chi = 64, kappa = 8) in MIXED and FP64.

    The two-qubit channels DEP2(p2) o ZZ(phi) have a 15-fold degenerate Kraus spectrum (p2/16 each),
    so a kappa cut can fall inside a degenerate cluster, where the kept subspace is not unique.  The
    intrinsic uncertainty of the truncated readouts is measured by running FP64 twice, once with the
    channel inputs moved by 1e-13 (relative); the complex64 path must stay within 1e-6 or within a
    small multiple of that intrinsic spread, whichever is larger."""
    circ = W.hea(n=N, depth=6, seed=W.MASTER_SEED + 2)
    zz = {}
    for name, c, prec in (("fp64", circ, "fp64"), ("fp64_perturbed", _perturbed(circ, 1e-13, 7), "fp64"),
                          ("mixed", circ, "mixed")):
        st = G.run_circuit(c, CHI, KAP, prec)
        zz[name] = st.zz_map()[0]
        bonds, _ = st.dims()
        assert max(bonds) == CHI
    spread = float(np.max(np.abs(zz["fp64_perturbed"] - zz["fp64"])))
    err = float(np.max(np.abs(zz["mixed"] - zz["fp64"])))
    print(f"n=20 chi=64 kappa=8, 6 layers: max|ZZ_mixed - ZZ_fp64| = {err:.2e}; "
          f"FP64 spread under 1e-13 input perturbation = {spread:.2e}")
    assert err < max(1e-6, 10 * spread)
