"""Batched runtime: many independent noisy circuits through the C ABI.

Circuits whose gates sit on the same positions in the same order (same qubit count, same sequence of
(1q/2q, site)) form one group and run as one batch of chains: every call of the group advances all
chains at once, each chain with its own gate matrix and its own channel (per-chain channel sets,
uploaded once).  Each group's whole circuit is captured into one CUDA graph (reset included), so a
replay runs the full circuit on the GPU without host involvement.  Different groups are
independent and run concurrently, each group on its own CUDA stream.
"""
from __future__ import annotations

import collections
from typing import Dict, List, Sequence

import numpy as np

from . import mpdo as G


class Group:
    def __init__(self, circuits, idx, chi_max, kappa_max, prec, stream, torch):
        self.idx = idx
        self.n = circuits[0].n
        self.B = len(circuits)
        self.ops = circuits[0].ops
        self.st = G.MPDO(self.n, chi_max, kappa_max, prec, batch=self.B, stream=stream)
        self.slots = []  # (kind, q, U_dev, channel set)
        chan_cache: Dict[tuple, G.ChannelSet] = {}
        for k, op in enumerate(self.ops):
            d = 2 ** op.kind
            U = np.stack([c.ops[k].U for c in circuits]).astype(np.complex128).reshape(self.B, d, d)
            key = tuple(id(c.chis[c.ops[k].chan][1]) for c in circuits)
            cs = chan_cache.get(key)
            if cs is None:
                cs = self.st.channels(op.kind, [c.chis[c.ops[k].chan][1] for c in circuits])
                chan_cache[key] = cs
            self.slots.append((op.kind, op.q, torch.tensor(U, device="cuda"), cs))
        self.graph = None

    def run_direct(self):
        self.st.reset()
        for kind, q, U, cs in self.slots:
            (self.st.apply_1q_batch if kind == 1 else self.st.apply_2q_batch)(q, U.data_ptr(), cs)

    def capture(self):
        self.st.capture_begin()
        self.run_direct()
        self.graph = self.st.capture_end(restore=False)

    def launch(self):
        if self.graph is None:
            self.capture()
        self.graph.launch()

    def n_2q(self) -> int:
        return sum(1 for k, *_ in self.slots if k == 2) * self.B


class BatchedRun:
    """All circuits of a workload, grouped by gate-position signature."""

    def __init__(self, circuits: Sequence, chi_max: int, kappa_max: int, prec="mixed", stream: int = 0,
                 torch=None, concurrent: bool = True):
        if torch is None:
            import torch as _t
            torch = _t
        self.torch = torch
        self.circuits = list(circuits)
        by_sig = collections.OrderedDict()
        for i, c in enumerate(self.circuits):
            sig = (c.n, tuple((o.kind, o.q) for o in c.ops))
            by_sig.setdefault(sig, []).append(i)
        self.groups: List[Group] = []
        self.streams = []
        for sig, idx in by_sig.items():
            s = stream
            if concurrent:
                self.streams.append(torch.cuda.Stream())
                s = self.streams[-1].cuda_stream
            self.groups.append(Group([self.circuits[i] for i in idx], idx, chi_max, kappa_max, prec, s, torch))

    def run(self, graphs: bool = True):
        for g in self.groups:
            if graphs:
                g.launch()
            else:
                g.run_direct()
        for g in self.groups:
            g.st.sync()

    def n_2q(self) -> int:
        return sum(g.n_2q() for g in self.groups)

    def maxcut(self) -> np.ndarray:
        """<H_MaxCut> per circuit, edges mapped to chain positions through meta['perm']."""
        out = np.zeros(len(self.circuits))
        for g in self.groups:
            # edges differ per chain: evaluate the ZZ map once and sum each chain's own edges
            zz = g.st.zz_map()
            for b, ci in enumerate(g.idx):
                c = self.circuits[ci]
                pos = {v: i for i, v in enumerate(c.meta["perm"])}
                out[ci] = sum(0.5 * (1 - zz[b, pos[u], pos[v]]) for u, v in c.meta["edges"])
        return out

    def discarded(self) -> np.ndarray:
        out = np.zeros((len(self.circuits), 3))
        for g in self.groups:
            d = g.st.discarded()
            for b, ci in enumerate(g.idx):
                out[ci] = d[b]
        return out
