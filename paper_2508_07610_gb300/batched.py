"""Binding of the batched runtime of include/mpdo.h (mpdo_batch_*): argument marshalling only.

Circuits are flattened into the C ABI's op arrays and process-matrix table; the library groups them
by gate-position signature, builds one or more batched handles per group (schedule from its
autotuner when a tuning file is given), captures every handle's circuit into a CUDA graph on its own
stream and replays them all per run.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import mpdo as G

_sig_done = False


def _lib():
    global _sig_done
    L = G.lib()
    if not _sig_done:
        vp, ip, dp, i32 = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int
        sig = {
            "mpdo_batch_create": [i32, ip, ip, ip, ip, dp, ip, i32, ip, dp, i32, i32, i32, C.c_char_p, C.POINTER(vp)],
            "mpdo_batch_run": [vp],
            "mpdo_batch_sync": [vp],
            "mpdo_batch_expect": [vp, i32, ip, ip, dp],
            "mpdo_batch_info": [vp, ip, ip, C.POINTER(C.c_longlong)],
            "mpdo_batch_schedule": [vp, i32, ip, ip, ip, ip, dp],
            "mpdo_batch_free": [vp],
            "mpdo_batch_fidelity": [vp, vp, dp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        _sig_done = True
    return L


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class BatchedRun:
    """All circuits of a workload through mpdo_batch_create / _run / _expect."""

    def __init__(self, circuits: Sequence, chi_max: int, kappa_max: int, prec="mixed", stream: int = 0,
                 torch=None, tuning: Optional[str] = None):
        L = _lib()
        self.circuits = list(circuits)
        count = len(self.circuits)
        # the process-matrix table: each distinct chi array once
        table, index = [], {}
        n = np.array([c.n for c in self.circuits], dtype=np.int32)
        begin = np.zeros(count + 1, dtype=np.int32)
        kinds, qs, chi_of, Us = [], [], [], []
        for ci, c in enumerate(self.circuits):
            begin[ci + 1] = begin[ci] + len(c.ops)
            for op in c.ops:
                if op.kind == 8:  # global bond truncation to chi = op.q: no gate, no channel
                    kinds.append(8)
                    qs.append(op.q)
                    chi_of.append(0)
                    Us.append(np.zeros(16, dtype=np.complex128))
                    continue
                if op.kind not in (1, 2):
                    raise ValueError("the batched runtime takes one- and two-qubit gates (apply_3q_batch on a "
                                     "handle takes three-qubit gates)")
                nq, chi = c.chis[op.chan]
                key = id(chi)
                if key not in index:
                    index[key] = len(table)
                    table.append((nq, np.ascontiguousarray(chi, dtype=np.complex128)))
                kinds.append(op.kind)
                qs.append(op.q)
                chi_of.append(index[key])
                u = np.zeros(16, dtype=np.complex128)
                u[: op.U.size] = np.asarray(op.U, dtype=np.complex128).reshape(-1)
                Us.append(u)
        self._n = n
        self._begin = begin
        kinds = np.array(kinds, dtype=np.int32)
        qs = np.array(qs, dtype=np.int32)
        chi_of = np.array(chi_of, dtype=np.int32)
        U = np.ascontiguousarray(np.stack(Us) if Us else np.zeros((0, 16), np.complex128))
        chi_nq = np.array([t[0] for t in table], dtype=np.int32)
        chis = np.ascontiguousarray(np.concatenate([t[1].reshape(-1) for t in table]))
        h = C.c_void_p()
        prec_i = G.PREC[prec] if isinstance(prec, str) else int(prec)
        G._check(L.mpdo_batch_create(count, _ip(n), _ip(begin), _ip(kinds), _ip(qs), U.ctypes.data_as(C.POINTER(C.c_double)),
                                     _ip(chi_of), len(table), _ip(chi_nq), chis.ctypes.data_as(C.POINTER(C.c_double)),
                                     chi_max, kappa_max, prec_i, tuning.encode() if tuning else None, C.byref(h)),
                 "mpdo_batch_create")
        self.h = h
        ng, nh, n2 = C.c_int(), C.c_int(), C.c_longlong()
        G._check(L.mpdo_batch_info(self.h, C.byref(ng), C.byref(nh), C.byref(n2)), "mpdo_batch_info")
        self.n_groups, self.n_handles, self._n2q = ng.value, nh.value, n2.value

    @property
    def groups(self):
        """Per group: (qubits, instances, handles, tensor cores, tuned ms per replay)."""
        out = []
        for g in range(self.n_groups):
            v = [C.c_int() for _ in range(4)]
            ms = C.c_double()
            G._check(_lib().mpdo_batch_schedule(self.h, g, *[C.byref(x) for x in v], C.byref(ms)),
                     "mpdo_batch_schedule")
            out.append(tuple(x.value for x in v) + (ms.value,))
        return out

    def launch(self):
        G._check(_lib().mpdo_batch_run(self.h), "mpdo_batch_run")

    def sync(self):
        G._check(_lib().mpdo_batch_sync(self.h), "mpdo_batch_sync")

    def run(self, graphs: bool = True):
        self.launch()
        self.sync()

    def n_2q(self) -> int:
        return int(self._n2q)

    def _expect(self, kind, per, args_begin=None, args=None):
        out = np.zeros(per)
        ab = None if args_begin is None else _ip(args_begin)
        aa = None if args is None or args.size == 0 else _ip(args)
        G._check(_lib().mpdo_batch_expect(self.h, kind, ab, aa, _dp(out)), f"mpdo_batch_expect({kind})")
        return out

    def maxcut(self) -> np.ndarray:
        """<H_MaxCut> per circuit, edges mapped to chain positions through meta['perm']."""
        begin = [0]
        args = []
        for c in self.circuits:
            pos = {v: i for i, v in enumerate(c.meta["perm"])}
            for u, v in c.meta["edges"]:
                args += [pos[u], pos[v]]
            begin.append(len(args))
        return self._expect(G.MAXCUT, len(self.circuits), np.array(begin, dtype=np.int32),
                            np.array(args, dtype=np.int32))

    def ghz(self) -> np.ndarray:
        return self._expect(G.GHZ, len(self.circuits))

    def trace(self) -> np.ndarray:
        return self._expect(G.TRACE, len(self.circuits))

    def discarded(self) -> np.ndarray:
        return self._expect(G.DISCARDED, 3 * len(self.circuits)).reshape(-1, 3)

    def fidelity(self, other: "BatchedRun") -> np.ndarray:
        """Uhlmann fidelity of every instance against the same instance of `other` (Sec. IV.C)."""
        out = np.zeros(len(self.circuits))
        G._check(_lib().mpdo_batch_fidelity(self.h, other.h, _dp(out)), "mpdo_batch_fidelity")
        return out

    def free(self):
        if getattr(self, "h", None):
            _lib().mpdo_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
