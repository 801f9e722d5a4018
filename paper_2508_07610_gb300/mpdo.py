"""ctypes binding of the C ABI in include/mpdo.h (argument marshalling only).

Every computation runs in libmpdo.so's sm_103a kernels; there is no CPU fallback.  If the library
is missing this module raises instead of computing anything.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# MPDO_LIBRARY=bounds loads the address-checked debug build (build.build(bounds=True)) instead
LIB_PATH = os.path.join(HERE, "libmpdo_bounds.so" if os.environ.get("MPDO_LIBRARY") == "bounds" else "libmpdo.so")

FP64, MIXED, FP32 = 0, 1, 2
PREC = {"fp64": FP64, "mixed": MIXED, "fp32": FP32}
TRACE, ZZ, ZZ_MAP, GHZ, MAXCUT, PURITY, DISCARDED, DIMS, PROB = range(9)
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "not completely positive",
          4: "not trace preserving", 5: "non-finite result", 6: "timeout", 7: "CUDA error", 8: "invalid state",
          9: "trace guard: Tr rho grew or became non-finite"}


class MPDOError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


_lib = None


def lib():
    """Load libmpdo.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2508_07610_gb300.build.build()"
                          + ("  (bounds=True)" if LIB_PATH.endswith("_bounds.so") else ""))
    L = C.CDLL(LIB_PATH)
    vp, ip, dp, i32 = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int
    sig = {
        "mpdo_init": [i32, i32, i32, i32, vp, C.POINTER(vp)],
        "mpdo_init_batch": [i32, i32, i32, i32, i32, vp, C.POINTER(vp)],
        "mpdo_free": [vp],
        "mpdo_reset": [vp],
        "mpdo_sync": [vp],
        "channel_from_process_matrix": [vp, i32, dp, C.c_double, C.POINTER(vp), ip],
        "channel_set_from_process_matrices": [vp, i32, i32, dp, C.c_double, C.POINTER(vp), ip],
        "channel_kraus": [vp, i32, dp, ip],
        "channel_free": [vp],
        "apply_1q": [vp, i32, dp, vp],
        "apply_2q": [vp, i32, dp, vp],
        "apply_3q": [vp, i32, dp, vp],
        "apply_3q_batch": [vp, i32, vp, vp, vp],
        "apply_1q_batch": [vp, i32, vp, vp, vp],
        "apply_2q_batch": [vp, i32, vp, vp, vp],
        "truncate_kraus": [vp, i32, i32, dp],
        "truncate_bonds": [vp, i32, dp],
        "expect": [vp, i32, ip, i32, dp],
        "mpdo_save": [vp, C.c_char_p],
        "mpdo_load": [C.c_char_p, vp, C.POINTER(vp)],
        "mpdo_capture_begin": [vp],
        "mpdo_capture_end": [vp, i32, C.POINTER(vp)],
        "mpdo_graph_launch": [vp],
        "mpdo_graph_free": [vp],
        "mpdo_get_site": [vp, i32, i32, dp, ip],
        "mpdo_set_site": [vp, i32, i32, i32, i32, dp],
        "mpdo_set_centre": [vp, i32],
        "mpdo_profile": [vp, i32],
        "mpdo_set_neighbour_truncation": [vp, i32],
        "mpdo_set_trace_guard": [vp, C.c_double],
        "mpdo_set_tensor_cores": [vp, i32],
        "mpdo_set_purity_memory": [vp, C.c_longlong],
        "mpdo_profile_read": [vp, dp, dp, C.POINTER(C.c_longlong)],
        "mpdo_wait_selftest": [i32, ip],
        "mpdo_set_trunc_order": [vp, i32],
        "mpdo_tc_selftest": [i32, i32, i32, dp, ip],
        "mpdo_fidelity": [vp, i32, vp, i32, dp],
        "mpdo_distribution": [vp, dp],
        "mpdo_jsd": [dp, dp, i32, dp],
        "mpdo_bounds_register": [vp, C.c_size_t],
        "mpdo_bounds_unregister": [vp],
        "mpdo_bounds_read": [C.POINTER(C.c_ulonglong), C.c_char_p, i32, ip, C.POINTER(C.c_ulonglong),
                             C.POINTER(C.c_ulonglong)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.mpdo_launch_count.argtypes = [vp]
    L.mpdo_launch_count.restype = C.c_longlong
    L.mpdo_status_string.argtypes = [C.c_int]
    L.mpdo_status_string.restype = C.c_char_p
    L.mpdo_bounds_enabled.argtypes = []
    L.mpdo_bounds_enabled.restype = C.c_int
    _lib = L
    return L


def bounds_enabled() -> bool:
    """True when the loaded library is the address-checked debug build."""
    return bool(lib().mpdo_bounds_enabled())


def bounds_register(ptr: int, nbytes: int):
    """Declare a caller-owned device buffer (e.g. a torch tensor passed as U_dev) to the address
    checks of the debug build; a no-op in the release library."""
    _check(lib().mpdo_bounds_register(C.c_void_p(ptr), nbytes), "mpdo_bounds_register")


def bounds_unregister(ptr: int):
    _check(lib().mpdo_bounds_unregister(C.c_void_p(ptr)), "mpdo_bounds_unregister")


def bounds_read() -> dict:
    """Failed address checks since the last read (the debug build only), and the first one's site."""
    fails, line, addr, nb = C.c_ulonglong(), C.c_int(), C.c_ulonglong(), C.c_ulonglong()
    buf = C.create_string_buffer(64)
    _check(lib().mpdo_bounds_read(C.byref(fails), buf, 64, C.byref(line), C.byref(addr), C.byref(nb)),
           "mpdo_bounds_read")
    return {"failures": fails.value, "file": buf.value.decode(), "line": line.value, "address": addr.value,
            "bytes": nb.value}


def _check(status: int, where: str):
    if status != 0:
        raise MPDOError(status, where)


def _cdata(a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


class ChannelSet:
    """Channels converted on the GPU from their Pauli-basis process matrices (Sec. III)."""

    def __init__(self, state: "MPDO", nq: int, chis: Sequence[np.ndarray], tol: float = 1e-12):
        L = lib()
        arr, p = _cdata(np.stack([np.asarray(c, dtype=np.complex128) for c in chis]))
        self.nq, self.count = nq, arr.shape[0]
        self.ranks = np.zeros(self.count, dtype=np.int32)
        h = C.c_void_p()
        _check(L.channel_set_from_process_matrices(state.h, nq, self.count, p, tol, C.byref(h),
                                                   self.ranks.ctypes.data_as(C.POINTER(C.c_int))),
               "channel_set_from_process_matrices")
        self.h = h

    def kraus(self, idx: int) -> np.ndarray:
        d = 2 ** self.nq
        out = np.zeros((int(self.ranks.max()) if self.count else 1, d, d), dtype=np.complex128)  # r_pad = max rank
        r = C.c_int()
        _check(lib().channel_kraus(self.h, idx, out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(r)),
               "channel_kraus")
        return out[: r.value]

    def free(self):
        if getattr(self, "h", None):
            lib().channel_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Graph:
    def __init__(self, h):
        self.h = h

    def launch(self):
        _check(lib().mpdo_graph_launch(self.h), "mpdo_graph_launch")

    def free(self):
        if self.h:
            lib().mpdo_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class MPDO:
    """A batch of `batch` MPDO chains of n qubits on the GPU."""

    def __init__(self, n: int, chi_max: int, kappa_max: int, prec="fp64", batch: int = 1, stream: int = 0):
        L = lib()
        self.n, self.batch = n, batch
        self.chi_max, self.kappa_max = chi_max, kappa_max
        self.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        h = C.c_void_p()
        _check(L.mpdo_init_batch(batch, n, chi_max, kappa_max, self.prec, C.c_void_p(stream or None), C.byref(h)),
               "mpdo_init_batch")
        self.h = h

    # -------------------------------------------------------------- lifecycle
    def free(self):
        if getattr(self, "h", None):
            lib().mpdo_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def reset(self):
        _check(lib().mpdo_reset(self.h), "mpdo_reset")

    def sync(self):
        _check(lib().mpdo_sync(self.h), "mpdo_sync")

    def launch_count(self) -> int:
        return int(lib().mpdo_launch_count(self.h))

    def profile(self, enable: bool = True):
        _check(lib().mpdo_profile(self.h, 1 if enable else 0), "mpdo_profile")

    PROFILE_CLASSES = ("gemm", "qr", "eig", "other", "gemm_gram", "gemm_theta", "eig_bond", "eig_kraus",
                       "one_qubit")

    def profile_read(self):
        """{class: (ms, flops, launches)}; gemm, qr, eig and other partition every launch, the last
        five are single call sites inside them (Kraus-leg Gram, the gate+channel product on the right
        site, the bond and the Kraus-leg eigensolvers, and the site-streaming products of the 1q
        update, for which the second entry is algorithmic bytes)."""
        nc = len(self.PROFILE_CLASSES)
        ms, fl = np.zeros(nc), np.zeros(nc)
        cnt = np.zeros(nc, dtype=np.int64)
        _check(lib().mpdo_profile_read(self.h, ms.ctypes.data_as(C.POINTER(C.c_double)),
                                       fl.ctypes.data_as(C.POINTER(C.c_double)),
                                       cnt.ctypes.data_as(C.POINTER(C.c_longlong))), "mpdo_profile_read")
        return {name: (float(ms[i]), float(fl[i]), int(cnt[i])) for i, name in enumerate(self.PROFILE_CLASSES)}

    # -------------------------------------------------------------- channels and gates
    def channels(self, nq: int, chis, tol: float = 1e-12) -> ChannelSet:
        return ChannelSet(self, nq, chis, tol)

    def apply_1q(self, q: int, U: np.ndarray, ch: ChannelSet):
        u, p = _cdata(U)
        _check(lib().apply_1q(self.h, q, p, ch.h), "apply_1q")

    def apply_2q(self, q: int, U: np.ndarray, ch: ChannelSet):
        u, p = _cdata(U)
        _check(lib().apply_2q(self.h, q, p, ch.h), "apply_2q")

    def apply_3q(self, q: int, U: np.ndarray, ch: ChannelSet):
        u, p = _cdata(U)
        _check(lib().apply_3q(self.h, q, p, ch.h), "apply_3q")

    def apply_1q_batch(self, q: int, U_dev_ptr: int, ch: ChannelSet, idx_dev_ptr: Optional[int] = None):
        _check(lib().apply_1q_batch(self.h, q, C.c_void_p(U_dev_ptr), ch.h, C.c_void_p(idx_dev_ptr)),
               "apply_1q_batch")

    def apply_2q_batch(self, q: int, U_dev_ptr: int, ch: ChannelSet, idx_dev_ptr: Optional[int] = None):
        _check(lib().apply_2q_batch(self.h, q, C.c_void_p(U_dev_ptr), ch.h, C.c_void_p(idx_dev_ptr)),
               "apply_2q_batch")

    def set_tensor_cores(self, enable: bool):
        _check(lib().mpdo_set_tensor_cores(self.h, 1 if enable else 0), "mpdo_set_tensor_cores")

    def set_purity_memory(self, nbytes: int):
        _check(lib().mpdo_set_purity_memory(self.h, C.c_longlong(nbytes)), "mpdo_set_purity_memory")

    TRUNC_ORDERS = {"split_first": 0, "kraus_first": 1}

    def set_trunc_order(self, order: str):
        """'split_first' (bond split, then the Kraus leg of q+1) or 'kraus_first' (the merged tensor's
        new Kraus leg first, then the split), for every later apply_2q."""
        _check(lib().mpdo_set_trunc_order(self.h, self.TRUNC_ORDERS[order]), "mpdo_set_trunc_order")

    def set_neighbour_truncation(self, enable: bool):
        _check(lib().mpdo_set_neighbour_truncation(self.h, 1 if enable else 0), "mpdo_set_neighbour_truncation")

    def set_trace_guard(self, tol: float):
        """With tol > 0 every gate and truncation checks afterwards that no chain's Tr rho grew by more
        than tol relative since the previous one (MPDOError status 9 otherwise); 0 switches it off."""
        _check(lib().mpdo_set_trace_guard(self.h, float(tol)), "mpdo_set_trace_guard")

    def truncate_kraus(self, q: int, kappa: int = 0) -> np.ndarray:
        out = np.zeros(self.batch)
        _check(lib().truncate_kraus(self.h, q, kappa, out.ctypes.data_as(C.POINTER(C.c_double))), "truncate_kraus")
        return out

    def truncate_bonds(self, chi: int) -> np.ndarray:
        """Global bond truncation (Sec. II.D): QR sweep into canonical form, every bond cut to chi."""
        out = np.zeros(self.batch)
        _check(lib().truncate_bonds(self.h, chi, out.ctypes.data_as(C.POINTER(C.c_double))), "truncate_bonds")
        return out

    # -------------------------------------------------------------- readouts
    def _expect(self, kind: int, args=(), size: Optional[int] = None) -> np.ndarray:
        a = np.asarray(args, dtype=np.int32).reshape(-1)
        size = size or self.batch
        out = np.zeros(size)
        _check(lib().expect(self.h, kind, a.ctypes.data_as(C.POINTER(C.c_int)) if a.size else None, int(a.size),
                            out.ctypes.data_as(C.POINTER(C.c_double))), f"expect({kind})")
        return out

    def trace(self):
        return self._expect(TRACE)

    def zz(self, i: int, j: int):
        return self._expect(ZZ, (i, j))

    def zz_map(self):
        return self._expect(ZZ_MAP, size=self.batch * self.n * self.n).reshape(self.batch, self.n, self.n)

    def ghz_fidelity(self):
        return self._expect(GHZ)

    def maxcut(self, edges):
        return self._expect(MAXCUT, [x for e in edges for x in e])

    def probability(self, bits):
        """<z| rho |z> / Tr rho per chain for the bitstring z (bits[i] is qubit i's outcome)."""
        return self._expect(PROB, tuple(int(v) for v in bits))

    def distribution(self) -> np.ndarray:
        """The whole bitstring distribution per chain, batch x 2^n (qubit 0 most significant), from one
        batched prefix contraction (mpdo_distribution; n <= 15)."""
        out = np.zeros((self.batch, 1 << self.n))
        _check(lib().mpdo_distribution(self.h, out.ctypes.data_as(C.POINTER(C.c_double))), "mpdo_distribution")
        return out

    def probabilities(self) -> np.ndarray:
        """The full output distribution per chain, batch x 2^n, basis index with qubit 0 most
        significant (small n only: one readout sweep per bitstring)."""
        if self.n > 16:
            raise ValueError("probabilities(): n > 16")
        out = np.zeros((self.batch, 1 << self.n))
        for z in range(1 << self.n):
            bits = [(z >> (self.n - 1 - i)) & 1 for i in range(self.n)]
            out[:, z] = self.probability(bits)
        return out

    def purity(self):
        return self._expect(PURITY)

    def fidelity(self, other: "MPDO", chain: int = 0, other_chain: int = 0) -> float:
        """Uhlmann fidelity (Sec. IV.C) of this state's chain against another handle's chain (n <= 7)."""
        out = C.c_double()
        _check(lib().mpdo_fidelity(self.h, chain, other.h, other_chain, C.byref(out)), "mpdo_fidelity")
        return out.value

    def discarded(self):
        return self._expect(DISCARDED, size=3 * self.batch).reshape(self.batch, 3)

    def dims(self):
        d = self._expect(DIMS, size=2 * self.n - 1).astype(int)
        return list(d[: self.n - 1]), list(d[self.n - 1:])

    # -------------------------------------------------------------- site access / checkpoint
    def get_site(self, q: int, chain: int = 0) -> np.ndarray:
        dims = np.zeros(3, dtype=np.int32)
        buf = np.zeros(2 * self.kappa_max * self.chi_max * self.chi_max, dtype=np.complex128)
        _check(lib().mpdo_get_site(self.h, chain, q, buf.ctypes.data_as(C.POINTER(C.c_double)),
                                   dims.ctypes.data_as(C.POINTER(C.c_int))), "mpdo_get_site")
        dl, dn, dr = (int(x) for x in dims)
        return buf[: dl * 2 * dn * dr].reshape(dl, 2, dn, dr).copy()

    def set_site(self, q: int, tensors) -> None:
        """tensors: one [dl, 2, dn, dr] array per chain (or one array used for all chains)."""
        if isinstance(tensors, np.ndarray):
            tensors = [tensors] * self.batch
        dl, _, dn, dr = tensors[0].shape
        arr, p = _cdata(np.stack(tensors))
        _check(lib().mpdo_set_site(self.h, q, dl, dn, dr, p), "mpdo_set_site")

    def set_centre(self, q: int):
        _check(lib().mpdo_set_centre(self.h, q), "mpdo_set_centre")

    def sites(self, chain: int = 0):
        return [self.get_site(q, chain) for q in range(self.n)]

    def save(self, path: str):
        _check(lib().mpdo_save(self.h, path.encode()), "mpdo_save")

    @classmethod
    def load(cls, path: str, stream: int = 0) -> "MPDO":
        h = C.c_void_p()
        _check(lib().mpdo_load(path.encode(), C.c_void_p(stream or None), C.byref(h)), "mpdo_load")
        obj = cls.__new__(cls)
        obj.h = h
        # read the shape back from a DIMS query is not enough for n; keep a header reader here
        import struct
        with open(path, "rb") as f:
            f.read(8)
            B, n, chi, kap, prec, _ = struct.unpack("6i", f.read(24))
        obj.n, obj.batch, obj.chi_max, obj.kappa_max, obj.prec = n, B, chi, kap, prec
        return obj

    # -------------------------------------------------------------- graphs
    def capture_begin(self):
        _check(lib().mpdo_capture_begin(self.h), "mpdo_capture_begin")

    def capture_end(self, restore: bool = False) -> Graph:
        g = C.c_void_p()
        _check(lib().mpdo_capture_end(self.h, 1 if restore else 0, C.byref(g)), "mpdo_capture_end")
        return Graph(g)


def tc_selftest(M: int, N: int, K: int):
    """Random complex64 M x K times K x N on the tensor cores and on the CUDA cores: returns (largest
    entry-wise difference relative to the largest entry, the tensor-core kernel's status word)."""
    err, flag = C.c_double(), C.c_int()
    _check(lib().mpdo_tc_selftest(M, N, K, C.byref(err), C.byref(flag)), "mpdo_tc_selftest")
    return err.value, flag.value


def wait_selftest(limit_us: int):
    """Run the bounded-wait probe (a wait on an mbarrier that nothing arrives on); returns
    (status, device status word).  Status 6 (timeout) is the expected outcome."""
    word = C.c_int(0)
    st = lib().mpdo_wait_selftest(int(limit_us), C.byref(word))
    return st, word.value


def run_circuit(circuit, chi_max: int, kappa_max: int, prec="fp64", stream: int = 0,
                trunc_order: str = "split_first", trace_guard: float = 0.0) -> MPDO:
    """Apply a workloads.Circuit on one chain; each channel is converted on the GPU once.  With
    trace_guard > 0 every op is followed by the trace guard (MPDO.set_trace_guard)."""
    st = MPDO(circuit.n, chi_max, kappa_max, prec, 1, stream)
    st.set_trunc_order(trunc_order)
    if trace_guard > 0:
        st.set_trace_guard(trace_guard)
    chans = {}
    for op in circuit.ops:
        if op.kind == 8:
            st.truncate_bonds(op.q)
            continue
        ch = chans.get(op.chan)
        if ch is None:
            ch = chans[op.chan] = st.channels(op.kind, [circuit.chis[op.chan][1]])
        (st.apply_1q, st.apply_2q, st.apply_3q)[op.kind - 1](op.q, op.U, ch)
    st._channels = chans
    return st


def jsd(p, q) -> float:
    """Jensen-Shannon divergence (natural log) between two distributions over the same outcomes, the
    distance the paper uses to compare output distributions: 0 for equal ones, ln 2 for disjoint ones
    (mpdo_jsd)."""
    a = np.ascontiguousarray(p, dtype=np.float64).reshape(-1)
    b = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    if a.size != b.size:
        raise ValueError("jsd: distributions of different lengths")
    out = C.c_double()
    _check(lib().mpdo_jsd(a.ctypes.data_as(C.POINTER(C.c_double)), b.ctypes.data_as(C.POINTER(C.c_double)),
                          int(a.size), C.byref(out)), "mpdo_jsd")
    return out.value
