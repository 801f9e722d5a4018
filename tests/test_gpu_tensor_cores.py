"""The tensor-core complex64 GEMM (tcgen05.mma kind::tf32, split TF32 operands, compensated folding
of the tensor-memory accumulator) against the CUDA-core GEMM with compensated FP32 sums, on the
shapes of the two-site update, ragged tiles and a long inner dimension; and the full-size update with
the tensor cores on and off."""
import numpy as np
import pytest

from oracle import channels as OC
from oracle import mpdo as OM
from paper_2508_07610_gb300 import mpdo as G
from paper_2508_07610_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 64, 16), (2048, 512, 128), (130, 70, 24), (256, 128, 128),
                                   (512, 128, 128), (128, 128, 8192)])
def test_tc_gemm_matches_cuda_core_gemm(M, N, K):
    err, flag = G.tc_selftest(M, N, K)
    print(f"tc gemm {M}x{N}x{K}: max relative difference {err:.2e}")
    assert flag == 0
    # both sides carry FP32 rounding of about u = 6e-8 per folded block; 1e-6 is the
    # per-result bound of the complex64 path
    assert err < 1e-6


def test_tc_gemm_rejects_small_shapes():
    with pytest.raises(G.MPDOError):
        G.tc_selftest(64, 64, 16)


def _pair_rdm(A1, A2):
    th = np.einsum("lanb,bcmr->lacnmr", A1, A2)
    m = th.reshape(th.shape[0], 4, -1, th.shape[-1])
    return np.einsum("lxkr,lykr->xy", m, m.conj())


@pytest.mark.parametrize("tc", [False, True])
def test_full_size_update_with_and_without_tensor_cores(tc):
    """n = 20, chi = 64, kappa = 8, a rank-16 two-qubit channel: one update in MIXED with the tensor
    cores on and off, against the oracle, at the per-result bound of 1e-6."""
    rng = np.random.default_rng(2026)
    sites = W.random_right_canonical_sites(20, 64, 8, rng)
    chi2 = W.kraus_to_chi(W.compose(W.depolarizing_2q(1e-2), W.unitary_channel(W.zz_phase(0.013))))
    q = 9
    orc = OM.MPDO(20, 64, 8)
    orc.sites = [s.copy() for s in sites]
    orc.centre = 0
    orc.apply_2q(q, W.cz(), OC.chi_to_kraus(chi2, 2))
    st = G.MPDO(20, 64, 8, "mixed")
    st.set_tensor_cores(tc)
    for i, s in enumerate(sites):
        st.set_site(i, s)
    st.set_centre(0)
    st.apply_2q(q, W.cz(), st.channels(2, [chi2]))
    st.sync()
    r_o = _pair_rdm(orc.sites[q], orc.sites[q + 1])
    r_g = _pair_rdm(st.get_site(q), st.get_site(q + 1))
    err = np.max(np.abs(r_g - r_o)) / np.trace(r_o).real
    d = st.discarded()[0]
    print(f"full-size update, tensor cores {tc}: rdm err {err:.2e}")
    assert err < 1e-6
    assert abs(d[0] - orc.discarded_chi) < 1e-6 and abs(d[1] - orc.discarded_kappa) < 1e-6
