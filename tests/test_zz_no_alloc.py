"""The allocation-free chi -> Kraus entry point (for callers that cannot allocate device memory)
must reproduce the allocating conversion, on two calls in a row that share its fixed scratch array.
Kept in its own file, collected last."""
import ctypes as C

import numpy as np
import pytest

from paper_2508_07610_gb300 import mpdo as G
from paper_2508_07610_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(lib, torch, nq, chis):
    d2 = 4 ** nq
    chi_dev = torch.tensor(np.stack(chis), dtype=torch.complex128, device="cuda")
    kraus_dev = torch.full((len(chis), d2, 2 ** nq, 2 ** nq), complex(np.nan, np.nan), dtype=torch.complex128,
                           device="cuda")
    ranks_dev = torch.full((len(chis),), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.channel_kraus_noalloc(nq, len(chis), C.c_void_p(chi_dev.data_ptr()), 0.0,
                                   C.c_void_p(kraus_dev.data_ptr()), C.c_void_p(ranks_dev.data_ptr()),
                                   C.c_void_p(stream or None))
    assert st == 0
    torch.cuda.synchronize()
    return kraus_dev.cpu().numpy(), ranks_dev.cpu().numpy()


@pytest.mark.parametrize("nq", [1, 2])
def test_noalloc_matches_allocating_entry_point(nq):
    torch = pytest.importorskip("torch")
    lib = G.lib()
    lib.channel_kraus_noalloc.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                          C.c_void_p]
    lib.channel_kraus_noalloc.restype = C.c_int
    rng = np.random.default_rng(40 + nq)
    st = G.MPDO(2, 2, 2)
    for call in range(2):  # two calls in a row on the shared scratch array
        ranks_in = [1, 2, 3, 4] if nq == 1 else [1, 5, 11, 16]
        chis = [W.kraus_to_chi(W.random_channel_kraus(nq, r, rng)) for r in ranks_in]
        ref = st.channels(nq, chis)  # the allocating entry point
        kr, ranks = _noalloc(lib, torch, nq, chis)
        assert list(ranks) == list(ref.ranks) == ranks_in
        for c in range(len(chis)):
            r = int(ranks[c])
            k_ref = ref.kraus(c)
            assert np.max(np.abs(kr[c, :r] - k_ref[:r])) < 1e-12
            if r < kr.shape[1]:
                assert np.max(np.abs(kr[c, r:])) == 0.0
        ref.free()


def test_noalloc_rejects_too_many_channels():
    lib = G.lib()
    lib.channel_kraus_noalloc.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                          C.c_void_p]
    lib.channel_kraus_noalloc.restype = C.c_int
    dummy = C.c_void_p(1)
    assert lib.channel_kraus_noalloc(2, 65, dummy, 0.0, dummy, dummy, None) == 1
    assert lib.channel_kraus_noalloc(3, 1, dummy, 0.0, dummy, dummy, None) == 1
