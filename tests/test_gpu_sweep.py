"""The crosstalk / truncation sweep workload (random 1D circuits with simultaneous CZ layers and
crosstalk channels on the idle neighbouring pairs) against the CPU oracle, at several (chi, kappa)
caps and in every precision mode; and the chunked purity contraction against its unchunked form.

Tolerances as in the parity tests (tests/tolerances.py): 1e-10 (FP64) and 1e-6 (complex64) on
normalised readouts, plus the oracle's allowance for cuts inside near-degenerate eigenvalue clusters;
the raw trace relative to its value; discarded weights against the derived Gram-error bound.
"""
import numpy as np
import pytest

from oracle import mpdo as OM
from paper_2508_07610_gb300 import mpdo as G
from paper_2508_07610_gb300 import workloads as W
from tolerances import allowance, discarded_limit, readout_limit

pytestmark = pytest.mark.gpu

TRACE_TOL = {"fp64": 1e-10, "mixed": 1e-5, "fp32": 1e-5}


def _compare(st, o, prec, label):
    lim = readout_limit(o, prec)
    errs = {
        "zz": float(np.max(np.abs(st.zz_map()[0] - o.zz_map()))),
        "purity": abs(st.purity()[0] - o.purity()) / 2,  # two normalised factors
        "ghz": abs(st.ghz_fidelity()[0] - o.ghz_fidelity()),
    }
    tr = abs(st.trace()[0] - o.trace()) / o.trace()
    d = st.discarded()[0]
    derr = {"disc_chi": abs(d[0] - o.discarded_chi), "disc_kappa": abs(d[1] - o.discarded_kappa)}
    dlim = {"disc_chi": discarded_limit(o, prec, "chi"), "disc_kappa": discarded_limit(o, prec, "kappa")}
    print(f"sweep {label} {prec}: limit {lim:.2e} (allowance {allowance(o, prec):.2e}) trace_rel={tr:.2e} "
          + " ".join(f"{k}={v:.2e}" for k, v in errs.items())
          + " " + " ".join(f"{k}={v:.2e}/{dlim[k]:.1e}" for k, v in derr.items()))
    for k, v in errs.items():
        assert v < lim, (k, v, lim)
    assert tr < TRACE_TOL[prec] + allowance(o, prec), ("trace", tr)
    for k, v in derr.items():
        assert v < dlim[k], (k, v, dlim[k])


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("chi,kap", [(4, 2), (8, 4), (16, 8)])
def test_crosstalk_small_matches_oracle(prec, chi, kap):
    c = W.crosstalk_sweep(n=8, depth=6)
    o = OM.run_circuit(c, chi, kap)
    st = G.run_circuit(c, chi, kap, prec)
    _compare(st, o, prec, f"n=8 chi={chi} kappa={kap}")


@pytest.fixture(scope="module")
def n40():
    c = W.crosstalk_sweep(n=40, depth=4)
    return c, OM.run_circuit(c, 32, 4)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_crosstalk_n40_matches_oracle(prec, n40):
    """The sweep's chain length (n = 40) at its smallest caps, four layers."""
    c, o = n40
    st = G.run_circuit(c, 32, 4, prec)
    _compare(st, o, prec, "n=40 chi=32 kappa=4")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_purity_in_chunks_equals_one_pass(prec):
    """A purity budget small enough to split the chi^4 contraction into chunks of 3 environment
    indices (16 = 5 x 3 + 1: a ragged last chunk) gives the same value as one pass and the oracle."""
    c = W.crosstalk_sweep(n=10, depth=8)
    chi, kap = 16, 4
    o = OM.run_circuit(c, chi, kap)
    st = G.run_circuit(c, chi, kap, prec)
    bonds, _ = st.dims()
    assert max(bonds) == chi
    one = st.purity()[0]
    esize = 16 if prec == "fp64" else 8
    per_d = 2 * kap * chi ** 3  # largest intermediate per environment index at the caps
    st.set_purity_memory(2 * 3 * per_d * esize)
    chunked = st.purity()[0]
    # purity is quadratic in rho: twice the readout bound of an operator of norm 1, for each pass
    lim = readout_limit(o, prec, 2.0)
    assert abs(one - o.purity()) < lim
    assert abs(chunked - o.purity()) < lim
    if prec == "fp64":
        assert abs(chunked - one) < 1e-12, (chunked, one)
    st.set_purity_memory(0)
    assert abs(st.purity()[0] - o.purity()) < lim
