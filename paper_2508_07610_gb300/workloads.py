"""Seeded synthetic inputs for the noisy-circuit MPDO update.

This module only prepares inputs: gate unitaries, standard noise channels as
Kraus sets, their Pauli-basis process (chi) matrices, and circuits shaped like
the workloads the simulator is run on.  None of the simulator's own arithmetic
(chi -> Choi -> Kraus conversion, site contraction, truncation, readout) lives
here.  Both the CPU reference and the CUDA library take these objects as inputs.

Conventions (shared by every consumer):
  * Pauli order I, X, Y, Z; a two-qubit Pauli index is m = 4*a + b with a on the
    first (lower-numbered) qubit.
  * Two-qubit matrices use the basis index 2*p_q + p_{q+1} (q is the MSB).
  * A channel's chi matrix follows Eq. (chi) of Sec. III with unnormalised Pauli
    strings, so a trace-preserving channel has Tr(chi) = 1.
  * Rotations R_P(t) = exp(-i t P / 2); the QAOA mixer is exp(-i b X) and the
    cost gate exp(-i g (1 - Z Z) / 2) as written in Sec. IV.B.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULIS = (I2, PX, PY, PZ)

MASTER_SEED = 0x2508076100


# --------------------------------------------------------------------------
# gates
# --------------------------------------------------------------------------
def rot(P: np.ndarray, theta: float) -> np.ndarray:
    """exp(-i theta P / 2) for a Pauli-like P with P @ P = I."""
    n = P.shape[0]
    return math.cos(theta / 2) * np.eye(n, dtype=np.complex128) - 1j * math.sin(theta / 2) * P


def rx(t):
    return rot(PX, t)


def ry(t):
    return rot(PY, t)


def rz(t):
    return rot(PZ, t)


def hadamard() -> np.ndarray:
    return np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2)


def cz() -> np.ndarray:
    return np.diag([1, 1, 1, -1]).astype(np.complex128)


def swap() -> np.ndarray:
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = m[3, 3] = 1
    m[1, 2] = m[2, 1] = 1
    return m


def zz_phase(phi: float) -> np.ndarray:
    """exp(-i phi Z Z / 2): the coherent ZZ error of the two-qubit channels."""
    zz = np.array([1, -1, -1, 1], dtype=np.float64)
    return np.diag(np.exp(-0.5j * phi * zz))


def qaoa_cost(gamma: float) -> np.ndarray:
    """exp(-i gamma (1 - Z Z) / 2) on one edge (Sec. IV.B)."""
    zz = np.array([1, -1, -1, 1], dtype=np.float64)
    return np.diag(np.exp(-0.5j * gamma * (1.0 - zz)))


def qaoa_mixer(beta: float) -> np.ndarray:
    """exp(-i beta X) (Sec. IV.B)."""
    return math.cos(beta) * I2 - 1j * math.sin(beta) * PX


# --------------------------------------------------------------------------
# channels as Kraus sets
# --------------------------------------------------------------------------
def depolarizing_1q(p: float) -> List[np.ndarray]:
    """The printed single-qubit Kraus set of Sec. II.A: sqrt(1-3p/4) I, sqrt(p/4) X/Y/Z."""
    return [math.sqrt(1 - 3 * p / 4) * I2] + [math.sqrt(p / 4) * P for P in (PX, PY, PZ)]


def depolarizing_2q(p: float) -> List[np.ndarray]:
    """(1-p) rho + p I/4: sqrt(1-15p/16) II and sqrt(p/16) for the 15 other Pauli pairs."""
    pauli_strings(2)
    w = np.full(16, math.sqrt(p / 16))
    w[0] = math.sqrt(1 - 15 * p / 16)
    return list(w[:, None, None] * _PAULI_CACHE[2])


def amplitude_damping(g: float) -> List[np.ndarray]:
    k0 = np.array([[1, 0], [0, math.sqrt(1 - g)]], dtype=np.complex128)
    k1 = np.array([[0, math.sqrt(g)], [0, 0]], dtype=np.complex128)
    return [k0, k1]


def phase_damping(f: float) -> List[np.ndarray]:
    """Pure dephasing that scales the off-diagonal elements by f (0 <= f <= 1):
    sqrt((1+f)/2) I, sqrt((1-f)/2) Z."""
    return [math.sqrt((1 + f) / 2) * I2, math.sqrt((1 - f) / 2) * PZ]


def thermal_relaxation(t: float, T1: float, T2: float) -> List[np.ndarray]:
    """The thermal relaxation channel (TRC) of Sec. II.B for a gate of duration t: energy relaxation
    towards |0> with time constant T1 (amplitude damping, gamma = 1 - exp(-t/T1)) and loss of coherence
    with time constant T2 <= 2 T1 (the off-diagonal elements decay by exp(-t/T2); amplitude damping
    accounts for exp(-t/2T1) of it, pure dephasing for the rest).  The paper gives no gate durations:
    t, T1 and T2 are the caller's."""
    if not (t >= 0 and T1 > 0 and 0 < T2 <= 2 * T1):
        raise ValueError("thermal relaxation needs t >= 0, T1 > 0 and 0 < T2 <= 2 T1")
    g = 1 - math.exp(-t / T1)
    f = math.exp(-t / T2 + t / (2 * T1))
    return compose(phase_damping(f), amplitude_damping(g))


def state_prep_error(p: float) -> List[np.ndarray]:
    """SPAM at preparation (Sec. II.B): the qubit starts flipped with probability p."""
    return [math.sqrt(1 - p) * I2, math.sqrt(p) * PX]


def readout_error(e01: float, e10: float) -> List[np.ndarray]:
    """SPAM before measurement (Sec. II.B, probability p_M): a measure-and-reprepare channel with
    P(read 1 | 0) = e01 and P(read 0 | 1) = e10, so that the diagonal of the final state is the
    distribution a confused measurement reports."""
    k = [np.zeros((2, 2), dtype=np.complex128) for _ in range(4)]
    k[0][0, 0] = math.sqrt(1 - e01)
    k[1][1, 0] = math.sqrt(e01)
    k[2][0, 1] = math.sqrt(e10)
    k[3][1, 1] = math.sqrt(1 - e10)
    return k


def on_qubit(kraus: Sequence[np.ndarray], which: int) -> List[np.ndarray]:
    """A single-qubit Kraus set as a two-qubit one acting on the first (which = 0) or the second
    (which = 1) qubit of the pair (basis index 2 p_q + p_{q+1})."""
    return [np.kron(K, I2) if which == 0 else np.kron(I2, K) for K in kraus]


def both_qubits(first: Sequence[np.ndarray], second: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Kraus set of the product channel first (x) second on a pair."""
    return [np.kron(A, B) for A in first for B in second]


def crosstalk_3q(p2: float, phi: float, phi_xt: float, p_xt: float) -> List[np.ndarray]:
    """A three-qubit channel of the kind the tomography of a two-qubit gate together with its
    neighbour yields (Fig. 13b): the gate pair (q, q+1) gets DEP2(p2) o ZZ(phi), the spectator q+2 a
    ZZ(phi_xt) coupling to q+1 and DEP(p_xt).  As 8 x 8 Kraus operators, qubit q most significant."""
    pair = [np.kron(K, I2) for K in compose(depolarizing_2q(p2), unitary_channel(zz_phase(phi)))]
    xt = [np.kron(I2, zz_phase(phi_xt))]
    spec = [np.kron(np.eye(4, dtype=np.complex128), K) for K in depolarizing_1q(p_xt)]
    return compose(spec, compose(xt, pair))


def unitary_channel(U: np.ndarray) -> List[np.ndarray]:
    return [np.asarray(U, dtype=np.complex128)]


def compose(second: Sequence[np.ndarray], first: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Kraus set of `second` applied after `first` (ordered first-major)."""
    prod = np.einsum("bij,ajk->abik", np.asarray(second), np.asarray(first))
    return list(prod.reshape(-1, prod.shape[-2], prod.shape[-1]))


_PAULI_CACHE = {}


def pauli_strings(nq: int) -> List[np.ndarray]:
    if nq not in _PAULI_CACHE:
        out = [np.ones((1, 1), dtype=np.complex128)]
        for _ in range(nq):
            out = [np.kron(o, P) for o in out for P in PAULIS]
        _PAULI_CACHE[nq] = np.stack(out)
    return list(_PAULI_CACHE[nq])


def kraus_to_chi(kraus: Sequence[np.ndarray]) -> np.ndarray:
    """Process matrix of a Kraus set in the unnormalised Pauli basis.

    Writing K_k = sum_m c_km sigma_m (c_km = Tr(sigma_m K_k) / d) gives
    eps(rho) = sum_mn (sum_k c_km conj(c_kn)) sigma_m rho sigma_n^dagger.
    """
    K = np.asarray(kraus, dtype=np.complex128)
    d = K.shape[-1]
    nq = int(round(math.log2(d)))
    pauli_strings(nq)
    P = _PAULI_CACHE[nq]
    c = np.einsum("mij,kij->km", P.conj(), K) / d  # Tr(sigma_m^dagger K_k) / d (Paulis are Hermitian)
    return c.T @ c.conj()


# --------------------------------------------------------------------------
# circuits
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Op:
    """One noisy gate: `kind` is 1, 2 or 3 (qubits q .. q+kind-1); U is the ideal gate,
    `chan` indexes Circuit.chis (the channel applied after the gate).  kind 8 (SWEEP) is no gate but
    the global bond truncation of Sec. II.D to chi = q, placed at the end of a layer."""
    kind: int
    q: int
    U: np.ndarray
    chan: int


SWEEP = 8


def sweep_op(chi: int) -> Op:
    return Op(SWEEP, chi, np.zeros((1, 1), dtype=np.complex128), -1)


@dataclasses.dataclass
class Circuit:
    n: int
    ops: List[Op]
    chis: List[Tuple[int, np.ndarray]]  # (nq, chi matrix): what the simulator is given
    kraus: List[List[np.ndarray]] = dataclasses.field(default_factory=list)  # the sets chi was built from
    meta: dict = dataclasses.field(default_factory=dict)

    def n_2q(self) -> int:
        return sum(1 for o in self.ops if o.kind == 2)


class _Chans(list):
    """chi matrices plus the Kraus sets they were synthesised from."""

    def __init__(self):
        super().__init__()
        self.kraus = []


def _add_chan(chis, nq, kraus) -> int:
    chis.append((nq, kraus_to_chi(kraus)))
    chis.kraus.append([np.asarray(K, dtype=np.complex128) for K in kraus])
    return len(chis) - 1


def _circuit(n, ops, chis, meta) -> "Circuit":
    return Circuit(n, ops, list(chis), list(chis.kraus), meta)


def ghz_ansatz(n: int = 6, depth: int = 3, seed: int = MASTER_SEED + 1) -> Circuit:
    """Plain n-qubit GHZ-preparation ansatz: per layer Ry(theta) on every qubit then a CZ
    ladder on (i, i+1).  Each 1q gate carries AD(2e-3) o DEP(1e-3) o Ry(eps), eps ~ N(0, 0.02);
    each CZ carries DEP2(1e-2) o ZZ(phi), phi ~ N(0, 0.01)."""
    rng = np.random.default_rng(seed)
    ops, chis = [], _Chans()
    for _ in range(depth):
        for q in range(n):
            th = rng.uniform(-math.pi, math.pi)
            eps = rng.normal(0.0, 0.02)
            k = compose(amplitude_damping(2e-3), compose(depolarizing_1q(1e-3), unitary_channel(ry(eps))))
            ops.append(Op(1, q, ry(th), _add_chan(chis, 1, k)))
        for q in range(n - 1):
            phi = rng.normal(0.0, 0.01)
            k = compose(depolarizing_2q(1e-2), unitary_channel(zz_phase(phi)))
            ops.append(Op(2, q, cz(), _add_chan(chis, 2, k)))
    return _circuit(n, ops, chis, {"name": f"ghz_ansatz_n{n}_d{depth}"})


def hea_channels(n: int, rng, scale: float = 1.0, record: dict = None) -> Tuple[list, list, list]:
    """Per-qubit 1q channels AD(g) o DEP(p1) and per-pair 2q channels DEP2(p2) o ZZ(phi), with
    p1 ~ U(5e-4, 2e-3), g ~ U(1e-3, 4e-3), p2 ~ U(5e-3, 2e-2), phi ~ N(0, 0.01), all strengths
    multiplied by `scale`; the drawn values are appended to `record` when one is given."""
    chis = _Chans()
    c1 = []
    for _ in range(n):
        p1 = scale * rng.uniform(5e-4, 2e-3)
        g = scale * rng.uniform(1e-3, 4e-3)
        if record is not None:
            record.setdefault("p1", []).append(p1)
            record.setdefault("gamma", []).append(g)
        c1.append(_add_chan(chis, 1, compose(amplitude_damping(g), depolarizing_1q(p1))))
    c2 = []
    for _ in range(n - 1):
        p2 = scale * rng.uniform(5e-3, 2e-2)
        phi = scale * rng.normal(0.0, 0.01)
        if record is not None:
            record.setdefault("p2", []).append(p2)
            record.setdefault("phi", []).append(phi)
        c2.append(_add_chan(chis, 2, compose(depolarizing_2q(p2), unitary_channel(zz_phase(phi)))))
    return chis, c1, c2


def hea_layer_ops(n: int, layer: int, rng, c1, c2) -> List[Op]:
    """One hardware-efficient layer: Rz.Ry.Rz per qubit, then CZ on bonds of parity layer % 2."""
    ops = []
    for q in range(n):
        a, b, c = rng.uniform(-math.pi, math.pi, size=3)
        ops.append(Op(1, q, rz(c) @ ry(b) @ rz(a), c1[q]))
    for q in range(layer % 2, n - 1, 2):
        ops.append(Op(2, q, cz(), c2[q]))
    return ops


def hea(n: int = 20, depth: int = 10, seed: int = MASTER_SEED + 2) -> Circuit:
    rng = np.random.default_rng(seed)
    chis, c1, c2 = hea_channels(n, rng)
    ops = []
    for layer in range(depth):
        ops += hea_layer_ops(n, layer, rng, c1, c2)
    return _circuit(n, ops, chis, {"name": f"hea_n{n}_d{depth}"})


def random_regular3(n: int, rng) -> List[Tuple[int, int]]:
    """Uniform-ish random simple 3-regular graph by the configuration model with rejection."""
    assert n % 2 == 0 and n >= 4
    while True:
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        edges = set()
        ok = True
        for a, b in pairs:
            a, b = int(a), int(b)
            if a == b or (min(a, b), max(a, b)) in edges:
                ok = False
                break
            edges.add((min(a, b), max(a, b)))
        if ok:
            return sorted(edges)


def qaoa_maxcut(n: int, p: int, edges, gammas, betas, rng, chis=None, c1=None, c2=None, cswap=None,
                scale: float = 1.0) -> Circuit:
    """Noisy QAOA for MaxCut on a 1D chain: H layer, then per layer a full odd-even
    transposition SWAP network (n rounds) in which every adjacent pair that is a graph edge
    receives the cost gate fused with its SWAP, followed by the mixer on every qubit.
    meta['perm'][i] is the logical vertex sitting at chain position i at the end."""
    record = {}
    if chis is None:
        chis, c1, c2 = hea_channels(n, rng, scale, record)
        cswap = []
        for q in range(n - 1):
            p2 = scale * rng.uniform(5e-3, 2e-2)
            phi = scale * rng.normal(0.0, 0.01)
            cswap.append(_add_chan(chis, 2, compose(depolarizing_2q(2 * p2), unitary_channel(zz_phase(phi)))))
    eset = set((min(a, b), max(a, b)) for a, b in edges)
    ops = [Op(1, q, hadamard(), c1[q]) for q in range(n)]
    roles = [("h", -1)] * n  # per op: its kind and layer, so the angles can be replaced later
    pos = list(range(n))  # pos[i] = logical vertex at chain position i
    fused_cache = {}
    for layer in range(p):
        g, b = gammas[layer], betas[layer]
        for rnd in range(n):
            for q in range(rnd % 2, n - 1, 2):
                u, v = pos[q], pos[q + 1]
                if (min(u, v), max(u, v)) in eset:
                    key = (layer, q)
                    # cost gate with its 2q channel, then SWAP with the SWAP channel, as one update
                    U = swap() @ qaoa_cost(g)
                    ck = fused_cache.get(key)
                    if ck is None:
                        kc = chis.kraus[c2[q]]
                        ks = chis.kraus[cswap[q]]
                        sw = swap()
                        moved = [sw @ K @ sw.conj().T for K in kc]
                        ck = _add_chan(chis, 2, compose(ks, moved))
                        fused_cache[key] = ck
                    ops.append(Op(2, q, U, ck))
                    roles.append(("cost", layer))
                else:
                    ops.append(Op(2, q, swap(), cswap[q]))
                    roles.append(("swap", layer))
                pos[q], pos[q + 1] = pos[q + 1], pos[q]
        for q in range(n):
            ops.append(Op(1, q, qaoa_mixer(b), c1[q]))
            roles.append(("mix", layer))
    return _circuit(n, ops, chis, {"name": f"qaoa_n{n}_p{p}", "edges": sorted(eset), "perm": pos,
                                   "gammas": list(gammas), "betas": list(betas), "noise": record,
                                   "roles": roles})


def qaoa_with_angles(template: Circuit, gammas, betas) -> Circuit:
    """The QAOA circuit `template` (from qaoa_maxcut) with other angles: the same gate positions and
    channels, the cost gates (fused with their SWAP) and mixers rebuilt for gammas, betas."""
    ops = []
    for op, (role, layer) in zip(template.ops, template.meta["roles"]):
        if role == "cost":
            ops.append(Op(2, op.q, swap() @ qaoa_cost(gammas[layer]), op.chan))
        elif role == "mix":
            ops.append(Op(1, op.q, qaoa_mixer(betas[layer]), op.chan))
        else:
            ops.append(op)
    meta = dict(template.meta)
    meta["gammas"], meta["betas"] = list(gammas), list(betas)
    return Circuit(template.n, ops, template.chis, template.kraus, meta)


def qaoa_batch(count: int, seed: int = MASTER_SEED + 3, n_choices=tuple(range(8, 25, 2)), p_max: int = 4):
    """Batched noisy QAOA MaxCut instances: n ~ U{8,10,..,24} (3-regular graphs need even n),
    p ~ U{1..4}, gamma_k, beta_k ~ U(0, pi)."""
    ss = np.random.SeedSequence(seed)
    out = []
    for child in ss.spawn(count):
        rng = np.random.default_rng(child)
        n = int(rng.choice(n_choices))
        p = int(rng.integers(1, p_max + 1))
        edges = random_regular3(n, rng)
        gam = rng.uniform(0, math.pi, size=p)
        bet = rng.uniform(0, math.pi, size=p)
        out.append(qaoa_maxcut(n, p, edges, gam, bet, rng))
    return out


def cnot() -> np.ndarray:
    """CNOT with the first qubit as control (basis index 2 p_q + p_{q+1})."""
    m = np.eye(4, dtype=np.complex128)
    m[2:, 2:] = PX
    return m


def random_rot_cnot(n: int, m: int, rng, chans=None, sweep_chi: int = 0) -> Circuit:
    """The random 1D circuits of the truncation study (Sec. IV.C, Fig. 13a): a layer of random
    R in {RX, RY, RZ} with angles U(0, 2 pi] on every qubit, then a layer of CNOTs on the bonds of
    parity layer % 2, repeated m - 1 times, and a final rotation layer.  Channels as the HEA workload
    (one realisation per circuit, or the given (chis, c1, c2)).  With sweep_chi > 0 every CNOT layer
    is followed by the global bond truncation to sweep_chi (the schedule of Sec. II.D)."""
    chis, c1, c2 = chans if chans is not None else hea_channels(n, rng)
    rots = (rx, ry, rz)
    ops = []

    def rot_layer():
        for q in range(n):
            r = rots[int(rng.integers(0, 3))]
            ops.append(Op(1, q, r(2 * math.pi - rng.uniform(0, 2 * math.pi)), c1[q]))

    for layer in range(m - 1):
        rot_layer()
        for q in range(layer % 2, n - 1, 2):
            ops.append(Op(2, q, cnot(), c2[q]))
        if sweep_chi > 0:
            ops.append(sweep_op(sweep_chi))
    rot_layer()
    return _circuit(n, ops, chis, {"name": f"random_rot_cnot_n{n}_m{m}"})


def crosstalk_sweep(n: int = 40, depth: int = 20, seed: int = MASTER_SEED + 4) -> Circuit:
    """Random 1D circuit with simultaneous CZ layers and crosstalk: per layer a random
    R in {RX, RY, RZ} per qubit with angle U(0, 2 pi], CZ on bonds of parity layer % 2, then a
    crosstalk channel (ZZ phase ~ N(0, 0.03) with DEP2(2e-3)) on every idle bond next to an
    active pair, once per adjacent active pair.  A final 1q layer closes the circuit."""
    rng = np.random.default_rng(seed)
    chis, c1, c2 = hea_channels(n, rng)
    ops = []
    rots = (rx, ry, rz)

    def one_q_layer():
        for q in range(n):
            r = rots[int(rng.integers(0, 3))]
            t = 2 * math.pi - rng.uniform(0, 2 * math.pi)
            ops.append(Op(1, q, r(t), c1[q]))

    eye4 = np.eye(4, dtype=np.complex128)
    for layer in range(depth):
        one_q_layer()
        active = list(range(layer % 2, n - 1, 2))
        for q in active:
            ops.append(Op(2, q, cz(), c2[q]))
        for q in active:
            for nb in (q - 1, q + 1):
                if 0 <= nb < n - 1 and nb not in active:
                    phi = rng.normal(0.0, 0.03)
                    ck = _add_chan(chis, 2, compose(depolarizing_2q(2e-3), unitary_channel(zz_phase(phi))))
                    ops.append(Op(2, nb, eye4, ck))
    one_q_layer()
    return _circuit(n, ops, chis, {"name": f"crosstalk_n{n}_d{depth}"})


# Gate and coherence times of the unified-model workload.  The paper gives none; these are typical
# superconducting-qubit figures (seconds).
UNIFIED_TIMES = {"t1q": 50e-9, "t2q": 300e-9, "T1": 30e-6, "T2": 20e-6}


def unified_noise_circuit(n: int, depth: int, rng, model: str = "unified", p1: float = 1e-3, p2: float = 1e-2,
                          p_prep: float = 5e-3, e01: float = 1e-2, e10: float = 3e-2, times=None) -> Circuit:
    """The noisy circuit models of Sec. II.B (Fig. 1): state-preparation error on every qubit, then per
    layer Ry Rz on every qubit and CNOTs on the bonds of parity layer % 2, then readout error on every
    qubit.  A 1q gate is followed by DEP(p1) o TRC(t1q).  A CNOT is followed by TRC(t2q) on both
    qubits and, in the unified model (Fig. 1b), DEP(p2) on the target qubit only; in the general model
    (Fig. 1c) DEP(p2) acts on both qubits.  SPAM channels ride on identity gates."""
    if model not in ("unified", "general"):
        raise ValueError(model)
    tm = dict(UNIFIED_TIMES, **(times or {}))
    chis = _Chans()
    trc1 = thermal_relaxation(tm["t1q"], tm["T1"], tm["T2"])
    trc2 = thermal_relaxation(tm["t2q"], tm["T1"], tm["T2"])
    c_prep = _add_chan(chis, 1, state_prep_error(p_prep))
    c_meas = _add_chan(chis, 1, readout_error(e01, e10))
    c1 = _add_chan(chis, 1, compose(depolarizing_1q(p1), trc1))
    dep2 = on_qubit(depolarizing_1q(p2), 1) if model == "unified" else both_qubits(depolarizing_1q(p2),
                                                                                    depolarizing_1q(p2))
    c2 = _add_chan(chis, 2, compose(dep2, both_qubits(trc2, trc2)))
    ops = [Op(1, q, I2.copy(), c_prep) for q in range(n)]
    for layer in range(depth):
        for q in range(n):
            ops.append(Op(1, q, ry(rng.uniform(-math.pi, math.pi)) @ rz(rng.uniform(-math.pi, math.pi)), c1))
        for q in range(layer % 2, n - 1, 2):
            ops.append(Op(2, q, cnot(), c2))
    ops += [Op(1, q, I2.copy(), c_meas) for q in range(n)]
    return _circuit(n, ops, chis, {"name": f"{model}_noise_n{n}_d{depth}", "times": tm})


def random_unitary(d: int, rng) -> np.ndarray:
    z = (rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))) / math.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def random_channel_kraus(nq: int, rank: int, rng) -> List[np.ndarray]:
    """A random CPTP map of the given Kraus rank (isometry columns split into Kraus blocks)."""
    d = 2 ** nq
    V = random_unitary(d * rank, rng)[:, :d]
    return [V[k * d:(k + 1) * d, :] for k in range(rank)]


def random_circuit(n: int, n_ops: int, rng, rank1: int = 3, rank2: int = 6, p2q: float = 0.5, p3q: float = 0.0,
                   rank3: int = 6) -> Circuit:
    """Unstructured random noisy circuit: random unitaries with random CPTP channels (with
    probability p3q a three-qubit gate and channel)."""
    ops, chis = [], _Chans()
    for _ in range(n_ops):
        if n > 2 and rng.uniform() < p3q:
            q = int(rng.integers(0, n - 2))
            ch = _add_chan(chis, 3, random_channel_kraus(3, rank3, rng))
            ops.append(Op(3, q, random_unitary(8, rng), ch))
        elif n > 1 and rng.uniform() < p2q:
            q = int(rng.integers(0, n - 1))
            ch = _add_chan(chis, 2, random_channel_kraus(2, rank2, rng))
            ops.append(Op(2, q, random_unitary(4, rng), ch))
        else:
            q = int(rng.integers(0, n))
            ch = _add_chan(chis, 1, random_channel_kraus(1, rank1, rng))
            ops.append(Op(1, q, random_unitary(2, rng), ch))
    return _circuit(n, ops, chis, {"name": f"random_n{n}_{n_ops}"})


def random_right_canonical_sites(n: int, chi: int, kappa: int, rng, centre_scale: float = 1.0):
    """A random MPDO state with every bond at its cap: site 0 is a random tensor of unit norm and
    every other site is a random right isometry (its (l) x (p, n, r) matrix has orthonormal rows),
    so the orthogonality centre is site 0.  Bonds are min(chi, 2*kappa*bond_left, ...) shaped like a
    saturated chain; the Kraus legs all have dimension kappa."""
    bonds = [1] * (n + 1)
    for q in range(1, n):
        bonds[q] = min(chi, (2 * kappa) ** min(q, n - q))
    sites = []
    for q in range(n):
        dl, dr = bonds[q], bonds[q + 1]
        if q == 0:
            A = rng.normal(size=(dl, 2, kappa, dr)) + 1j * rng.normal(size=(dl, 2, kappa, dr))
            A *= centre_scale / np.linalg.norm(A)
        else:
            U = random_unitary(2 * kappa * dr, rng)
            A = U[:dl, :].reshape(dl, 2, kappa, dr)
        sites.append(np.ascontiguousarray(A, dtype=np.complex128))
    return sites


def surrogate_features(circ, p_max: int = 4) -> np.ndarray:
    """16 inputs of the screening surrogate: gamma_1..4 and beta_1..4 (zero-padded to p_max = 4,
    divided by pi) and the means and spreads of p1, p2, gamma, phi over the chain (divided by the
    middle of their ranges)."""
    g = np.zeros(p_max)
    b = np.zeros(p_max)
    gm, bt = circ.meta["gammas"], circ.meta["betas"]
    g[:len(gm)] = np.asarray(gm) / math.pi
    b[:len(bt)] = np.asarray(bt) / math.pi
    rec = circ.meta["noise"]
    ref = {"p1": 1.25e-3, "p2": 1.25e-2, "gamma": 2.5e-3, "phi": 1e-2}
    means = [np.mean(rec[k]) / ref[k] for k in ("p1", "p2", "gamma", "phi")]
    spreads = [np.std(rec[k]) / ref[k] for k in ("p1", "p2", "gamma", "phi")]
    return np.concatenate([g, b, means, spreads]).astype(np.float32)
