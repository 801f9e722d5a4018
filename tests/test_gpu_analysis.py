"""Analysis readouts of Sec. IV.C on the GPU against the oracle: the Uhlmann fidelity of a truncated
state against the untruncated one (Eq. fidelity), for single handles and per instance of two batches,
on the random RX/RY/RZ + CNOT circuits of the truncation study (Fig. 13a)."""
import numpy as np
import pytest

from oracle import dense as OD
from oracle import mpdo as OM
from paper_2508_07610_gb300 import batched as BR
from paper_2508_07610_gb300 import mpdo as G
from paper_2508_07610_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m,chi,kap", [(3, 4, 2, 1), (4, 5, 2, 2), (5, 4, 4, 2)])
def test_fidelity_of_truncated_state_matches_oracle(n, m, chi, kap):
    rng = np.random.default_rng(60 + n)
    circ = W.random_rot_cnot(n, m, rng)
    exact_caps = (64, 32)
    t = G.run_circuit(circ, chi, kap, "fp64")
    e = G.run_circuit(circ, *exact_caps, "fp64")
    f_gpu = t.fidelity(e)
    ot, oe = OM.run_circuit(circ, chi, kap), OM.run_circuit(circ, *exact_caps)
    f_ref = OD.uhlmann_fidelity(ot.dense(), oe.dense())
    # the reference keeps every bond and all but a small part of the Kraus weight (kappa_max = 32 is
    # the library's largest Kraus cap), while the truncation under test costs far more fidelity
    assert oe.discarded_chi < 1e-24 and oe.discarded_kappa < 1e-4
    assert f_ref < 1 - 1e-2
    assert abs(f_ref - OD.uhlmann_fidelity(ot.dense(), OD.run_circuit(circ))) < 1e-3
    print(f"fidelity n={n} m={m} chi={chi} kappa={kap}: GPU {f_gpu:.10f}, oracle {f_ref:.10f}")
    # the square root of the truncated state's rounding-level zero eigenvalues (about 1e-16) enters
    # at about sqrt(u) = 1e-8
    assert abs(f_gpu - f_ref) < 1e-7
    assert abs(e.fidelity(e) - 1) < 1e-7
    # a complex64 truncated state against the FP64 one
    tm = G.run_circuit(circ, chi, kap, "mixed")
    assert abs(tm.fidelity(e) - f_ref) < 1e-5


def test_batched_fidelity_per_instance_matches_oracle():
    rng = np.random.default_rng(81)
    circs = [W.random_rot_cnot(3, 4, rng) for _ in range(12)]
    t = BR.BatchedRun(circs, 2, 2, "fp64")
    e = BR.BatchedRun(circs, 8, 32, "fp64")
    t.run()
    e.run()
    f = t.fidelity(e)
    for i, c in enumerate(circs):
        ref = OD.uhlmann_fidelity(OM.run_circuit(c, 2, 2).dense(), OM.run_circuit(c, 8, 32).dense())
        assert abs(f[i] - ref) < 1e-7, (i, f[i], ref)


def test_fidelity_rejects_large_chains():
    a = G.MPDO(8, 4, 2, "fp64")
    with pytest.raises(G.MPDOError):
        a.fidelity(a)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_distribution_matches_oracle_and_per_bitstring_readout(prec):
    """mpdo_distribution (all 2^n prefixes carried through each site at once) against the oracle's
    dense diagonal, and against the one-sweep-per-bitstring readout."""
    from tolerances import readout_limit
    rng = np.random.default_rng(1500)
    circ = W.random_circuit(5, 18, rng, rank1=3, rank2=5)
    st = G.run_circuit(circ, 6, 3, prec)
    orc = OM.run_circuit(circ, 6, 3)
    d = st.distribution()
    ref = np.real(np.diag(orc.dense()))
    ref = ref / ref.sum()
    assert d.shape == (1, 32) and abs(d.sum() - 1) < 1e-12
    assert np.max(np.abs(d[0] - ref)) < readout_limit(orc, prec)
    per = np.array([st.probability([(z >> (4 - i)) & 1 for i in range(5)])[0] for z in range(32)])
    assert np.max(np.abs(d[0] - per)) < 2 * readout_limit(orc, prec)
    assert G.jsd(d[0], ref) < 1e-6


def test_distribution_rejects_long_chains():
    st = G.MPDO(16, 2, 2, "fp64")
    with pytest.raises(G.MPDOError):
        st.distribution()
