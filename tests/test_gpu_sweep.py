"""The crosstalk / truncation sweep workload (random 1D circuits with simultaneous CZ layers and
crosstalk channels on the idle neighbouring pairs) against the CPU oracle, at several (chi, kappa)
caps and in every precision mode; and the chunked purity contraction against its unchunked form.

Tolerances as in the parity tests: 1e-10 (FP64) and 1e-6 (complex64) on normalised readouts, plus
4 x the oracle's cut_sensitivity(eps) for truncations that cut inside near-degenerate eigenvalues.
"""
import numpy as np
import pytest

from oracle import mpdo as OM
from paper_2508_07610_gb300 import mpdo as G
from paper_2508_07610_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-10, 1e-13, 1e-9), "mixed": (1e-6, 5e-7, 2e-5), "fp32": (1e-6, 5e-7, 2e-5)}  # readout, eps, disc


def _compare(st, o, prec, label):
    tol, eps, dtol = TOL[prec]
    lim = tol + 4 * o.cut_sensitivity(eps)
    errs = {
        "trace": abs(st.trace()[0] - o.trace()),
        "zz": float(np.max(np.abs(st.zz_map()[0] - o.zz_map()))),
        "purity": abs(st.purity()[0] - o.purity()),
        "ghz": abs(st.ghz_fidelity()[0] - o.ghz_fidelity()),
    }
    d = st.discarded()[0]
    derr = {"disc_chi": abs(d[0] - o.discarded_chi), "disc_kappa": abs(d[1] - o.discarded_kappa)}
    print(f"sweep {label} {prec}: lim {lim:.2e} " + " ".join(f"{k}={v:.2e}" for k, v in {**errs, **derr}.items()))
    for k, v in errs.items():
        assert v < lim, (k, v, lim)
    # a cut inside a near-degenerate cluster keeps one of several equally valid subspaces, and the later
    # truncations' discarded weights depend on which: the same allowance as the readouts
    for k, v in derr.items():
        assert v < dtol + 4 * o.cut_sensitivity(eps), (k, v, dtol)


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
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert abs(chunked - one) < tol, (chunked, one)
    assert abs(one - o.purity()) < TOL[prec][0] + 4 * o.cut_sensitivity(TOL[prec][1])
    st.set_purity_memory(0)
    assert abs(st.purity()[0] - one) < tol
