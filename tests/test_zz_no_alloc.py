"""The allocation-free chi -> Kraus entry point, for callers that cannot allocate device memory (a
plug-in living inside another application's memory pool, or code that must not grow its device
footprint after start-up).  Its channels must equal the oracle's conversion (Sec. III) and the
allocating entry point's, compared through the superoperator sum_i K_i (x) conj(K_i), which does not
depend on the gauge freedom of a Kraus set, on two calls in a row that share its fixed scratch array.
Kept in its own file, collected last."""
import ctypes as C

import numpy as np
import pytest

from oracle import channels as OC
from paper_2508_07610_gb300 import mpdo as G
from paper_2508_07610_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    lib = G.lib()
    lib.channel_kraus_noalloc.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                          C.c_void_p]
    lib.channel_kraus_noalloc.restype = C.c_int
    return lib


def _noalloc(torch, nq, chis):
    d2 = 4 ** nq
    chi_dev = torch.tensor(np.stack(chis), dtype=torch.complex128, device="cuda")
    kraus_dev = torch.full((len(chis), d2, 2 ** nq, 2 ** nq), complex(np.nan, np.nan), dtype=torch.complex128,
                           device="cuda")
    ranks_dev = torch.full((len(chis),), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = _lib().channel_kraus_noalloc(nq, len(chis), C.c_void_p(chi_dev.data_ptr()), 0.0,
                                      C.c_void_p(kraus_dev.data_ptr()), C.c_void_p(ranks_dev.data_ptr()),
                                      C.c_void_p(stream or None))
    assert st == 0
    torch.cuda.synchronize()
    return kraus_dev.cpu().numpy(), ranks_dev.cpu().numpy()


@pytest.mark.parametrize("nq", [1, 2])
def test_noalloc_matches_oracle_and_allocating_entry_point(nq):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(40 + nq)
    st = G.MPDO(2, 2, 2)
    for call in range(2):  # two calls in a row on the shared scratch array
        ranks_in = [1, 2, 3, 4] if nq == 1 else [1, 5, 11, 16]
        chis = [W.kraus_to_chi(W.random_channel_kraus(nq, r, rng)) for r in ranks_in]
        ref = st.channels(nq, chis)  # the allocating entry point
        kr, ranks = _noalloc(torch, nq, chis)
        assert list(ranks) == list(ref.ranks) == ranks_in
        for c in range(len(chis)):
            r = int(ranks[c])
            s_na = OC.superop(list(kr[c, :r]))
            assert np.max(np.abs(s_na - OC.superop(OC.chi_to_kraus(chis[c], nq)))) < 1e-12
            assert np.max(np.abs(s_na - OC.superop(list(ref.kraus(c))))) < 1e-12
            assert OC.is_trace_preserving(list(kr[c, :r]), 1e-12)
            if r < kr.shape[1]:
                assert np.max(np.abs(kr[c, r:])) == 0.0
        ref.free()


def test_noalloc_flags_invalid_channels():
    """A process matrix with negative Choi mass, and one that is not trace preserving, get the
    sentinel ranks -1 and -2 (the allocating entry point returns MPDO_ENOTCP / MPDO_ENOTTP)."""
    torch = pytest.importorskip("torch")
    good = W.kraus_to_chi(W.depolarizing_1q(0.1))
    not_cp = np.diag([1.2, -0.2, 0, 0]).astype(complex)
    not_tp = np.diag([0.9, 0.2, 0, 0]).astype(complex)  # trace 1.1: sum K^H K = 1.1 I
    kr, ranks = _noalloc(torch, 1, [good, not_cp, not_tp])
    assert list(ranks) == [4, -1, -2]
    assert np.max(np.abs(kr[1:])) == 0.0


def test_noalloc_rejects_too_many_channels():
    lib = _lib()
    dummy = C.c_void_p(1)
    assert lib.channel_kraus_noalloc(2, 65, dummy, 0.0, dummy, dummy, None) == 1
    assert lib.channel_kraus_noalloc(3, 1, dummy, 0.0, dummy, dummy, None) == 1
