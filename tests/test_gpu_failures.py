"""Failure reporting through the C ABI, with every failure made on the host side (no GPU fault):
non-finite site data reaches the truncation eigensolver, which flags its result; a kernel's bounded
wait on a barrier that nothing signals gives up and reports a timeout; in both cases the context
stays usable afterwards."""
import numpy as np
import pytest

from paper_2508_07610_gb300 import mpdo as G
from paper_2508_07610_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_non_finite_site_reports_no_convergence(prec):
    st = G.MPDO(3, 4, 2, prec)
    site = np.zeros((1, 2, 1, 1), dtype=np.complex128)
    site[0, 0, 0, 0] = np.nan
    st.set_site(0, site)
    ch = st.channels(1, [W.kraus_to_chi(W.depolarizing_1q(0.1))])
    st.apply_1q(0, W.ry(0.3), ch)  # enqueued; the Kraus-leg eigensolver sees a NaN Gram matrix
    with pytest.raises(G.MPDOError) as e:
        st.sync()
    assert e.value.status == 5
    # the word is cleared once read, and the device keeps working
    st.sync()
    ok = G.MPDO(3, 4, 2, prec)
    ok.apply_1q(1, W.ry(0.3), ok.channels(1, [W.kraus_to_chi(W.depolarizing_1q(0.1))]))
    ok.sync()
    assert abs(ok.trace()[0] - 1) < 1e-6


def test_bounded_wait_times_out_and_context_survives():
    for limit_us in (50, 2000):
        st, word = G.wait_selftest(limit_us)
        assert st == 6 and word == 2
    assert G.wait_selftest(0)[0] == 1  # limits outside 1 us .. 1 s are rejected
    ok = G.MPDO(2, 2, 2, "fp64")
    ok.apply_2q(0, W.cz(), ok.channels(2, [W.kraus_to_chi([np.eye(4)])]))  # ideal CZ: nothing truncated
    ok.sync()
    assert abs(ok.trace()[0] - 1) < 1e-12
