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


# ------------------------------------------------------------------ trace guard
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-7), ("mixed", 1e-4), ("fp32", 1e-4)])
def test_trace_guard_passes_lossy_circuits_without_changing_them(prec, tol):
    """Truncations only lower Tr rho and the channels preserve it, so a guarded run of a lossy circuit
    (one-, two- and three-qubit channels, both caps cutting) raises nothing; the guard only reads, so
    the state is bit for bit the unguarded one."""
    circ = W.random_circuit(6, 40, np.random.default_rng(31), rank1=3, rank2=6, p3q=0.2)
    ref = G.run_circuit(circ, 4, 2, prec)
    st = G.run_circuit(circ, 4, 2, prec, trace_guard=tol)
    assert st.discarded()[0][0] > 1e-4 and st.discarded()[0][1] > 1e-4
    assert np.array_equal(st.trace(), ref.trace())
    assert np.array_equal(st.zz_map(), ref.zz_map())


def test_trace_guard_reports_growth_between_calls():
    """An edit that doubles one chain's orthogonality centre (Tr rho x 4) is caught at the next
    guarded call (status 9, after the call's work is done), for that chain only; the reading then
    becomes the baseline, reset brings it back to 1, and with the guard off nothing is checked."""
    st = G.MPDO(3, 4, 2, "fp64", batch=2)
    ch = st.channels(1, [W.kraus_to_chi(W.depolarizing_1q(0.05))])
    st.set_trace_guard(1e-7)
    st.apply_1q(0, W.ry(0.3), ch)  # the centre is now site 0
    s0, s1 = st.get_site(0, 0), st.get_site(0, 1)
    st.set_site(0, [2 * s0, s1])
    with pytest.raises(G.MPDOError) as e:
        st.apply_1q(0, W.ry(0.2), ch)
    assert e.value.status == 9
    tr = st.trace()
    assert abs(tr[0] - 4) < 1e-9 and abs(tr[1] - 1) < 1e-9
    st.apply_1q(1, W.ry(0.1), ch)  # compared with the grown trace: passes
    st.reset()
    st.apply_1q(0, W.ry(0.3), ch)
    st.set_trace_guard(0)
    st.set_site(0, [2 * st.get_site(0, 0), st.get_site(0, 1)])
    st.apply_1q(0, W.ry(0.2), ch)  # guard off
    with pytest.raises(G.MPDOError) as e:
        st.set_trace_guard(float("nan"))
    assert e.value.status == 1
