"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Tolerances (tests/tolerances.py): 1e-10 in FP64 and 1e-6 in the complex64 modes (MIXED, FP32) on
every normalised readout and density-matrix entry, plus the oracle's allowance for truncations that
cut inside a near-degenerate eigenvalue cluster (relative gap below 1e-9 / 1e-5; other cuts add
nothing).  The raw trace is an n-fold product of contractions and is compared relatively (1e-10 /
1e-5); the cumulative discarded weights against the bound derived there from the Gram error.
"""
import numpy as np
import pytest

from oracle import channels as OC
from oracle import dense as OD
from oracle import mpdo as OM
from paper_2508_07610_gb300 import mpdo as G
from paper_2508_07610_gb300 import workloads as W
from tolerances import MODES, allowance, discarded_limit, readout_limit

pytestmark = pytest.mark.gpu

TRACE_TOL = {"fp64": 1e-10, "mixed": 1e-5, "fp32": 1e-5}
MODES_READOUT = {k: v[0] for k, v in MODES.items()}


def _oracle_from_gpu(st: G.MPDO, chain: int = 0) -> OM.MPDO:
    o = OM.MPDO(st.n, st.chi_max, st.kappa_max)
    o.sites = st.sites(chain)
    return o


def _check_state(st, orc, prec, n, chain=0, dense=True, label=""):
    lim = readout_limit(orc, prec)
    errs = {}
    if dense:
        rho_g = _oracle_from_gpu(st, chain).dense()
        rho_o = orc.dense()
        errs["rho"] = float(np.max(np.abs(rho_g / np.trace(rho_g) - rho_o / np.trace(rho_o))))
    errs["zz"] = float(np.max(np.abs(st.zz_map()[chain] - orc.zz_map())))
    errs["ghz"] = abs(st.ghz_fidelity()[chain] - orc.ghz_fidelity())
    tr = abs(st.trace()[chain] - orc.trace()) / max(1e-300, orc.trace())
    disc = st.discarded()[chain]
    derr = {"disc_chi": abs(disc[0] - orc.discarded_chi), "disc_kappa": abs(disc[1] - orc.discarded_kappa)}
    dlim = {"disc_chi": discarded_limit(orc, prec, "chi"), "disc_kappa": discarded_limit(orc, prec, "kappa")}
    print(f"parity {label} {prec}: limit {lim:.2e} (allowance {allowance(orc, prec):.2e}) trace_rel={tr:.2e} "
          + " ".join(f"{k}={v:.2e}" for k, v in errs.items())
          + " " + " ".join(f"{k}={v:.2e}/{dlim[k]:.1e}" for k, v in derr.items()))
    for k, v in errs.items():
        assert v < lim, (k, v, lim)
    assert tr < TRACE_TOL[prec] + allowance(orc, prec), ("trace", tr)
    for k, v in derr.items():
        assert v < dlim[k], (k, v, dlim[k])


# ------------------------------------------------------------------ chi -> Kraus (FP64 on the GPU)
@pytest.mark.parametrize("nq,rank,seed", [(1, 1, 0), (1, 2, 1), (1, 4, 2), (2, 1, 3), (2, 5, 4), (2, 16, 5)])
def test_chi_to_kraus_matches_oracle(nq, rank, seed):
    rng = np.random.default_rng(seed)
    chi = W.kraus_to_chi(W.random_channel_kraus(nq, rank, rng))
    st = G.MPDO(2, 2, 2)
    cs = st.channels(nq, [chi])
    kg = cs.kraus(0)
    ko = OC.chi_to_kraus(chi, nq)
    assert cs.ranks[0] == len(ko) == rank
    assert np.max(np.abs(OC.superop(list(kg)) - OC.superop(ko))) < 1e-12
    assert OC.is_trace_preserving(list(kg), 1e-12)
    # descending weight order (the pruning order of Sec. III)
    w = [np.linalg.norm(K) ** 2 for K in kg]
    assert all(w[i] >= w[i + 1] - 1e-12 for i in range(len(w) - 1))


def test_chi_to_kraus_printed_depolarizing_and_set():
    st = G.MPDO(2, 2, 2)
    ps = [0.0, 1e-3, 0.1, 0.5]
    chis = [np.diag([1 - 3 * p / 4, p / 4, p / 4, p / 4]).astype(complex) for p in ps]
    cs = st.channels(1, chis)
    assert list(cs.ranks) == [1, 4, 4, 4]
    for i, p in enumerate(ps):
        k = list(cs.kraus(i))
        assert np.max(np.abs(OC.superop(k) - OC.superop(W.depolarizing_1q(p)))) < 1e-13


def test_invalid_process_matrices_are_rejected():
    st = G.MPDO(2, 2, 2)
    good = W.kraus_to_chi(W.depolarizing_1q(0.1))
    with pytest.raises(G.MPDOError) as e:
        st.channels(1, [good * 1.1])
    assert e.value.status == 4
    bad = good.copy()
    bad[0, 1] += 0.1
    with pytest.raises(G.MPDOError) as e:
        st.channels(1, [bad])
    assert e.value.status == 1
    with pytest.raises(G.MPDOError) as e:
        st.channels(1, [np.diag([1.2, -0.2, 0, 0]).astype(complex)])
    assert e.value.status == 3
    with pytest.raises(G.MPDOError) as e:
        st.channels(1, [np.full((4, 4), np.nan, complex)])
    assert e.value.status == 1


# ------------------------------------------------------------------ whole circuits
@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_ghz_ansatz_n6(prec):
    circ = W.ghz_ansatz()  # n = 6, depth 3, chi_max = 16, kappa_max = 4
    st = G.run_circuit(circ, 16, 4, prec)
    orc = OM.run_circuit(circ, 16, 4)
    _check_state(st, orc, prec, 6, label="ghz_ansatz_n6")
    # Tr rho^2 / (Tr rho)^2: two normalised factors, each within the readout bound
    assert abs(st.purity()[0] - orc.purity()) < readout_limit(orc, prec, 2.0)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("n,nops,chi,kap,seed", [(4, 14, 64, 32, 0), (5, 20, 3, 2, 1), (6, 24, 5, 3, 2),
                                                  (7, 30, 4, 2, 3), (3, 12, 1, 1, 4), (2, 10, 2, 5, 5)])
def test_random_circuits(prec, n, nops, chi, kap, seed):
    rng = np.random.default_rng(1000 + seed)
    circ = W.random_circuit(n, nops, rng, rank1=3, rank2=6)
    st = G.run_circuit(circ, chi, kap, prec)
    orc = OM.run_circuit(circ, chi, kap)
    _check_state(st, orc, prec, n, label=f"random n{n} chi{chi} kappa{kap}")


def test_single_qubit_chain():
    rng = np.random.default_rng(9)
    circ = W.random_circuit(1, 6, rng, rank1=4, p2q=0.0)
    st = G.run_circuit(circ, 4, 3, "fp64")
    orc = OM.run_circuit(circ, 4, 3)
    rho_g = _oracle_from_gpu(st).dense()
    assert np.max(np.abs(rho_g / np.trace(rho_g) - orc.dense() / orc.trace())) < 1e-12


def test_exact_when_caps_cover_ranks():
    circ = W.ghz_ansatz(n=4, depth=1)
    st = G.run_circuit(circ, 64, 32, "fp64")
    rho = OD.run_circuit(circ)
    rho_g = _oracle_from_gpu(st).dense()
    assert np.max(np.abs(rho_g - rho)) < 1e-11
    d = st.discarded()[0]
    assert d[0] < 1e-13 and d[1] < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("chi,kap", [(1, 1), (1, 4), (16, 1), (2, 2)])
def test_smallest_caps(prec, chi, kap):
    """The degenerate caps: chi = 1 keeps a product state, kappa = 1 keeps one Kraus operator per site
    (a pure-state trajectory of largest weight); both still follow the oracle."""
    circ = W.ghz_ansatz(n=5, depth=2)
    st = G.run_circuit(circ, chi, kap, prec)
    orc = OM.run_circuit(circ, chi, kap)
    bonds, kraus = st.dims()
    assert max(bonds) <= chi and max(kraus) <= kap
    _check_state(st, orc, prec, 5, label=f"caps chi={chi} kappa={kap}")


def test_readouts_match_dense_definitions():
    circ = W.ghz_ansatz(n=5, depth=2)
    st = G.run_circuit(circ, 8, 4, "fp64")
    rho = _oracle_from_gpu(st).dense()
    tr = np.trace(rho).real
    assert abs(st.trace()[0] - tr) < 1e-11
    edges = [(0, 1), (1, 4), (2, 3), (0, 3)]
    assert abs(st.maxcut(edges)[0] - OD.maxcut_expectation(rho, 5, edges)) < 1e-11
    assert abs(st.purity()[0] - OD.purity(rho)) < 1e-11
    assert abs(st.ghz_fidelity()[0] - OD.ghz_fidelity(rho, 5)) < 1e-11
    assert abs(st.zz(3, 1)[0] - OD.expect_zz(rho, 5, 1, 3)) < 1e-11


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_bitstring_distribution_matches_oracle(prec):
    """<z| rho |z> / Tr rho for all 32 bitstrings of a truncated n = 5 state against the diagonal of the
    oracle's reconstructed rho (same truncations), and the Jensen-Shannon divergence between the two."""
    circ = W.ghz_ansatz(n=5, depth=2)
    st = G.run_circuit(circ, 8, 4, prec)
    orc = OM.run_circuit(circ, 8, 4)
    rho = orc.dense()
    p_o = OD.probabilities(rho / np.trace(rho))
    p_g = st.probabilities()[0]
    lim = readout_limit(orc, prec)
    assert np.max(np.abs(p_g - p_o)) < lim
    assert abs(p_g.sum() - 1) < lim
    assert G.jsd(p_g, p_o) < 10 * lim
    # a single bitstring through the C ABI, and argument checks
    assert abs(st.probability([0] * 5)[0] - p_o[0]) < lim
    with pytest.raises(G.MPDOError):
        st.probability([0, 1, 2, 0, 0])
    with pytest.raises(G.MPDOError):
        st.probability([0, 1])


# ------------------------------------------------------------------ batches
def test_batch_with_per_chain_gates_and_channels():
    torch = pytest.importorskip("torch")
    B, n = 3, 4
    rng = np.random.default_rng(77)
    circs = [W.random_circuit(n, 0, rng) for _ in range(B)]
    # one shared sequence of positions, different matrices and channels per chain
    layout = [(1, 0), (1, 1), (2, 0), (1, 2), (2, 2), (2, 1), (1, 3), (2, 0), (1, 1)]
    orcs = [OM.MPDO(n, 4, 3) for _ in range(B)]
    st = G.MPDO(n, 4, 3, "fp64", batch=B, stream=torch.cuda.current_stream().cuda_stream)
    keep = []
    for kind, q in layout:
        Us = [W.random_unitary(2 ** kind, rng) for _ in range(B)]
        chans = [W.kraus_to_chi(W.random_channel_kraus(kind, 3 if kind == 1 else 5, rng)) for _ in range(B)]
        cs = st.channels(kind, chans)
        U_dev = torch.tensor(np.stack(Us), dtype=torch.complex128, device="cuda")
        G.bounds_register(U_dev.data_ptr(), U_dev.numel() * U_dev.element_size())  # no-op in release
        keep += [cs, U_dev]
        (st.apply_1q_batch if kind == 1 else st.apply_2q_batch)(q, U_dev.data_ptr(), cs)
        for b in range(B):
            kr = OC.chi_to_kraus(chans[b], kind)
            (orcs[b].apply_1q if kind == 1 else orcs[b].apply_2q)(q, Us[b], kr)
    st.sync()
    zz = st.zz_map()
    for b in range(B):
        rho_g = _oracle_from_gpu(st, b).dense()
        rho_o = orcs[b].dense()
        assert np.max(np.abs(rho_g / np.trace(rho_g) - rho_o / np.trace(rho_o))) < 1e-10
        assert np.max(np.abs(zz[b] - orcs[b].zz_map())) < 1e-10


def test_batch_channel_index_array():
    torch = pytest.importorskip("torch")
    B, n = 4, 3
    rng = np.random.default_rng(5)
    chans = [W.kraus_to_chi(W.random_channel_kraus(2, r, rng)) for r in (2, 5)]
    idx = [1, 0, 0, 1]
    st = G.MPDO(n, 4, 2, "fp64", batch=B, stream=torch.cuda.current_stream().cuda_stream)
    cs = st.channels(2, chans)
    U = W.random_unitary(4, rng)
    U_dev = torch.tensor(np.stack([U] * B), dtype=torch.complex128, device="cuda")
    idx_dev = torch.tensor(idx, dtype=torch.int32, device="cuda")
    for t in (U_dev, idx_dev):
        G.bounds_register(t.data_ptr(), t.numel() * t.element_size())  # no-op in the release library
    st.apply_2q_batch(0, U_dev.data_ptr(), cs, idx_dev.data_ptr())
    st.apply_2q_batch(1, U_dev.data_ptr(), cs, idx_dev.data_ptr())
    st.sync()
    for b in range(B):
        o = OM.MPDO(n, 4, 2)
        kr = OC.chi_to_kraus(chans[idx[b]], 2)
        o.apply_2q(0, U, kr)
        o.apply_2q(1, U, kr)
        rho_g = _oracle_from_gpu(st, b).dense()
        assert np.max(np.abs(rho_g / np.trace(rho_g) - o.dense() / o.trace())) < 1e-10


# ------------------------------------------------------------------ explicit truncation, checkpoint, graphs
def test_truncate_kraus_explicit():
    rng = np.random.default_rng(21)
    circ = W.random_circuit(4, 16, rng, rank1=4, rank2=8)
    st = G.run_circuit(circ, 8, 6, "fp64")
    orc = OM.run_circuit(circ, 8, 6)
    w = st.truncate_kraus(2, 2)[0]
    wo = orc.truncate_kraus(2, 2)
    assert abs(w - wo) < 1e-10
    rho_g = _oracle_from_gpu(st).dense()
    assert np.max(np.abs(rho_g / np.trace(rho_g) - orc.dense() / orc.trace())) < 1e-10


def test_checkpoint_round_trip(tmp_path):
    circ = W.ghz_ansatz(n=5, depth=2)
    st = G.run_circuit(circ, 8, 3, "fp64")
    path = str(tmp_path / "state.ckpt")
    st.save(path)
    st2 = G.MPDO.load(path)
    assert st2.dims() == st.dims()
    assert np.max(np.abs(st2.zz_map() - st.zz_map())) < 1e-14
    assert np.max(np.abs(st2.discarded() - st.discarded())) < 1e-15
    # the loaded state continues like the original
    ch = st.channels(2, [W.kraus_to_chi(W.depolarizing_2q(0.02))])
    ch2 = st2.channels(2, [W.kraus_to_chi(W.depolarizing_2q(0.02))])
    st.apply_2q(1, W.cz(), ch)
    st2.apply_2q(1, W.cz(), ch2)
    assert np.max(np.abs(st2.zz_map() - st.zz_map())) < 1e-13


def test_graph_capture_replays_circuit():
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    circ = W.ghz_ansatz(n=5, depth=2)
    st = G.MPDO(5, 8, 3, "fp64", stream=s.cuda_stream)
    chans = {c: st.channels(nq, [chi]) for c, (nq, chi) in enumerate(circ.chis)}
    ref = G.run_circuit(circ, 8, 3, "fp64")
    st.capture_begin()
    st.reset()
    for op in circ.ops:
        (st.apply_1q if op.kind == 1 else st.apply_2q)(op.q, op.U, chans[op.chan])
    g = st.capture_end()
    for _ in range(2):
        g.launch()
        st.sync()
        assert np.max(np.abs(st.zz_map() - ref.zz_map())) < 1e-13
        assert np.max(np.abs(st.discarded() - ref.discarded())) < 1e-14


@pytest.mark.parametrize("seed", range(3))
def test_neighbour_truncation_matches_centre_moves(seed):
    """With neighbour truncation on, 1q gates next to the centre truncate through the centre's
    environment; the oracle moves the centre.  The states must agree."""
    rng = np.random.default_rng(500 + seed)
    n = 6
    circ = W.random_circuit(n, 40, rng, rank1=4, rank2=6, p2q=0.4)
    st = G.MPDO(n, 6, 3, "fp64")
    st.set_neighbour_truncation(True)
    chans = {}
    for op in circ.ops:
        ch = chans.get(op.chan)
        if ch is None:
            ch = chans[op.chan] = st.channels(op.kind, [circ.chis[op.chan][1]])
        (st.apply_1q if op.kind == 1 else st.apply_2q)(op.q, op.U, ch)
    orc = OM.run_circuit(circ, 6, 3)
    _check_state(st, orc, "fp64", n, label=f"neighbour truncation seed {seed}")


def test_neighbour_truncation_layer_pattern():
    """The benchmark's sweep pattern (pairs left to right, then right to left, far site through the
    centre) on a 7-qubit chain, against the oracle."""
    rng = np.random.default_rng(31)
    n = 7
    st = G.MPDO(n, 8, 4, "fp64")
    orc = OM.MPDO(n, 8, 4)
    keep = []

    def gate(kind, q, neighbour):
        U = W.random_unitary(2 ** kind, rng)
        chi = W.kraus_to_chi(W.random_channel_kraus(kind, 3 if kind == 1 else 5, rng))
        ch = st.channels(kind, [chi])
        keep.append(ch)
        st.set_neighbour_truncation(neighbour)
        (st.apply_1q if kind == 1 else st.apply_2q)(q, U, ch)
        (orc.apply_1q if kind == 1 else orc.apply_2q)(q, U, OC.chi_to_kraus(chi, kind))

    for layer in range(4):
        if layer % 2 == 0:
            for q in range(0, n - 1, 2):
                gate(1, q, False)
                gate(1, q + 1, True)
                gate(2, q, False)
            gate(1, n - 1, False)
        else:
            for q in range(n - 2, 0, -2):
                gate(1, q + 1, False)
                gate(1, q, True)
                gate(2, q, False)
            gate(1, 0, False)
    _check_state(st, orc, "fp64", n, label="neighbour layer pattern")


# ------------------------------------------------------------------ truncation order (Sec. II.D schedules)
@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("case", ["ghz", "random5", "random6"])
def test_kraus_first_order_matches_oracle(prec, case):
    """MPDO_TRUNC_KRAUS_FIRST: the merged tensor's new Kraus leg is truncated before the bond split, on
    the GPU through the Gram of the reduced pair (Theta is never formed), in the oracle by an explicit
    SVD of the merged tensor."""
    if case == "ghz":
        circ, chi, kap = W.ghz_ansatz(), 16, 4
    else:
        n = int(case[-1])
        rng = np.random.default_rng(700 + n)
        circ, chi, kap = W.random_circuit(n, 24, rng, rank1=3, rank2=6), 5, 3
    st = G.run_circuit(circ, chi, kap, prec, trunc_order="kraus_first")
    orc = OM.run_circuit(circ, chi, kap, trunc_order="kraus_first")
    _check_state(st, orc, prec, circ.n, label=f"kraus_first {case}")


def test_kraus_first_equals_split_first_without_bond_cuts():
    rng = np.random.default_rng(91)
    circ = W.random_circuit(4, 16, rng, rank1=3, rank2=6)
    a = G.run_circuit(circ, 64, 3, "fp64", trunc_order="split_first")
    b = G.run_circuit(circ, 64, 3, "fp64", trunc_order="kraus_first")
    ra, rb = _oracle_from_gpu(a).dense(), _oracle_from_gpu(b).dense()
    assert np.max(np.abs(ra / np.trace(ra) - rb / np.trace(rb))) < 1e-12
    assert abs(a.discarded()[0, 1] - b.discarded()[0, 1]) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("n,m,chi,kap,seed", [(5, 6, 3, 4, 12), (6, 8, 4, 4, 15), (6, 6, 2, 2, 2), (6, 8, 1, 4, 3)])
def test_global_bond_truncation_matches_oracle(prec, n, m, chi, kap, seed):
    """The paper's schedule of Sec. II.D on the random RX/RY/RZ + CNOT circuits of Fig. 13a: per-gate
    splits keep every rank (cap 64), and after each CNOT layer a QR sweep into canonical form is
    followed by the right-to-left truncation of every bond to chi; Kraus legs are truncated per gate."""
    rng = np.random.default_rng(900 + seed)
    circ = W.random_rot_cnot(n, m, rng, sweep_chi=chi)
    st = G.run_circuit(circ, 64, kap, prec)
    orc = OM.run_circuit(circ, 64, kap)
    assert orc.discarded_chi > 1e-3
    assert max(orc.bond_dims()) <= chi and max(st.dims()[0]) <= chi
    _check_state(st, orc, prec, n, label=f"global sweep n={n} m={m} chi={chi} kappa={kap}")


def test_global_bond_truncation_exact_when_chi_covers_ranks():
    rng = np.random.default_rng(77)
    circ = W.random_circuit(4, 12, rng, rank1=2, rank2=3)  # Kraus ranks up to 12: kappa_max = 32 cuts nothing
    st = G.run_circuit(circ, 64, 32, "fp64")
    before = _oracle_from_gpu(st).dense()
    w = st.truncate_bonds(64)[0]
    after = _oracle_from_gpu(st).dense()
    assert abs(w) < 1e-13
    assert np.max(np.abs(after - before)) < 1e-12
    assert np.max(np.abs(after - OD.run_circuit(circ))) < 1e-12


def test_global_bond_truncation_rejects_zero_chi():
    st = G.MPDO(3, 4, 2)
    with pytest.raises(G.MPDOError):
        st.truncate_bonds(0)


# ------------------------------------------------------------------ the noise models of Sec. II.B (Fig. 1)
@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("model", ["unified", "general"])
def test_noise_models_of_fig1_match_oracle(prec, model):
    """State-preparation error, thermal relaxation after every gate, depolarizing on the CNOT's target
    only (unified) or on both qubits (general), readout error before measurement."""
    circ = W.unified_noise_circuit(6, 4, np.random.default_rng(1000), model=model)
    st = G.run_circuit(circ, 16, 4, prec)
    orc = OM.run_circuit(circ, 16, 4)
    assert orc.discarded_kappa > 0
    _check_state(st, orc, prec, circ.n, label=f"{model} noise model")


def test_spam_distribution_closed_form():
    """With no gates between them, preparation and readout errors give a product distribution with
    P(read 1) = p (1 - e10) + (1 - p) e01 on every qubit."""
    n, p, e01, e10 = 3, 0.1, 0.02, 0.07
    chis = [(1, W.kraus_to_chi(W.state_prep_error(p))), (1, W.kraus_to_chi(W.readout_error(e01, e10)))]
    ops = [W.Op(1, q, np.eye(2), 0) for q in range(n)] + [W.Op(1, q, np.eye(2), 1) for q in range(n)]
    st = G.run_circuit(W.Circuit(n, ops, chis), 4, 4, "fp64")
    p1 = p * (1 - e10) + (1 - p) * e01
    for z in range(2 ** n):
        bits = [(z >> (n - 1 - i)) & 1 for i in range(n)]
        ref = np.prod([p1 if b else 1 - p1 for b in bits])
        assert abs(st.probability(bits)[0] - ref) < 1e-12


# ------------------------------------------------------------------ three-qubit channels (Fig. 13b)
def _three_qubit_circuit(n, layers, rng):
    """Random gates with physical noise: AD o DEP on 1q gates, DEP2 o ZZ on 2q gates, and the
    three-qubit crosstalk channel on random three-qubit gates."""
    chis = [(1, W.kraus_to_chi(W.compose(W.amplitude_damping(3e-3), W.depolarizing_1q(2e-3)))),
            (2, W.kraus_to_chi(W.compose(W.depolarizing_2q(1e-2), W.unitary_channel(W.zz_phase(0.02))))),
            (3, W.kraus_to_chi(W.crosstalk_3q(1e-2, 0.02, 0.05, 2e-3)))]
    ops = []
    for layer in range(layers):
        ops += [W.Op(1, q, W.random_unitary(2, rng), 0) for q in range(n)]
        ops += [W.Op(3, q, W.random_unitary(8, rng), 2) for q in range(layer % 3, n - 2, 3)]
        ops += [W.Op(2, q, W.random_unitary(4, rng), 1) for q in range((layer + 1) % 2, n - 1, 4)]
    return W.Circuit(n, ops, chis)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("n,layers,chi,kap,seed", [(5, 4, 8, 4, 0), (6, 4, 6, 3, 1)])
def test_three_qubit_channels_match_oracle(prec, n, layers, chi, kap, seed):
    circ = _three_qubit_circuit(n, layers, np.random.default_rng(1200 + seed))
    st = G.run_circuit(circ, chi, kap, prec)
    orc = OM.run_circuit(circ, chi, kap)
    assert orc.discarded_chi > 1e-6 and orc.discarded_kappa > 1e-6
    _check_state(st, orc, prec, n, label=f"three-qubit channels n={n} chi={chi} kappa={kap}")


def test_three_qubit_channels_exact_when_caps_cover_ranks():
    rng = np.random.default_rng(600)
    circ = W.random_circuit(4, 8, rng, rank1=1, rank2=1, p3q=0.5, rank3=2)
    assert sum(op.kind == 3 for op in circ.ops) >= 3
    st = G.run_circuit(circ, 32, 8, "fp64")
    rho = _oracle_from_gpu(st).dense()
    assert np.max(np.abs(rho - OD.run_circuit(circ))) < 1e-12
    assert np.max(np.abs(st.discarded()[0][:2])) < 1e-13


def test_crosstalk_channel_on_cnot_layers():
    """CNOT layers whose gates carry the three-qubit crosstalk channel onto their right neighbour."""
    rng = np.random.default_rng(77)
    n = 6
    ops, chis = [], []
    chis.append((1, W.kraus_to_chi(W.depolarizing_1q(1e-3))))
    chis.append((3, W.kraus_to_chi(W.crosstalk_3q(1e-2, 0.02, 0.05, 2e-3))))
    for layer in range(4):
        for q in range(n):
            ops.append(W.Op(1, q, W.ry(rng.uniform(-np.pi, np.pi)), 0))
        for q in range(layer % 2, n - 2, 3):
            ops.append(W.Op(3, q, np.kron(W.cnot(), np.eye(2)), 1))
    circ = W.Circuit(n, ops, chis)
    for prec in ("fp64", "mixed"):
        st = G.run_circuit(circ, 8, 4, prec)
        orc = OM.run_circuit(circ, 8, 4)
        _check_state(st, orc, prec, n, label=f"crosstalk 3q {prec}")


def test_three_qubit_update_rejects_large_caps():
    st = G.MPDO(4, 64, 8)
    ch = st.channels(3, [W.kraus_to_chi(W.crosstalk_3q(1e-2, 0.02, 0.05, 2e-3))])
    with pytest.raises(G.MPDOError):
        st.apply_3q(0, np.eye(8), ch)


# ------------------------------------------------------------------ scale of the state
@pytest.mark.parametrize("prec,scale", [("fp64", 1e-60), ("mixed", 1e-12), ("fp32", 1e-12)])
def test_tiny_norm_state_truncates_like_a_unit_one(prec, scale):
    """Nothing is renormalised, so after many lossy truncations the state's norm can be tiny.  The
    truncations depend only on ratios: a state scaled by `scale` must give the same normalised readouts
    and discarded weights as the unscaled oracle run, and its trace scaled by scale^2."""
    rng = np.random.default_rng(1300)
    circ = W.random_circuit(5, 20, rng, rank1=3, rank2=5)
    st = G.MPDO(5, 4, 3, prec)
    site = np.zeros((1, 2, 1, 1), dtype=np.complex128)
    site[0, 0, 0, 0] = scale
    st.set_site(0, site)
    chans = {}
    for op in circ.ops:
        ch = chans.get(op.chan)
        if ch is None:
            ch = chans[op.chan] = st.channels(op.kind, [circ.chis[op.chan][1]])
        (st.apply_1q if op.kind == 1 else st.apply_2q)(op.q, op.U, ch)
    orc = OM.run_circuit(circ, 4, 3)
    assert orc.discarded_chi > 1e-6 and orc.discarded_kappa > 1e-6
    lim = readout_limit(orc, prec)
    rho_g = _oracle_from_gpu(st).dense()
    rho_o = orc.dense()
    assert np.max(np.abs(rho_g / np.trace(rho_g) - rho_o / np.trace(rho_o))) < lim
    assert np.max(np.abs(st.zz_map()[0] - orc.zz_map())) < lim
    assert abs(st.trace()[0] / scale ** 2 - orc.trace()) < TRACE_TOL[prec] * orc.trace() + allowance(orc, prec)
    disc = st.discarded()[0]
    assert abs(disc[0] - orc.discarded_chi) < discarded_limit(orc, prec, "chi")
    assert abs(disc[1] - orc.discarded_kappa) < discarded_limit(orc, prec, "kappa")


def test_deep_lossy_qaoa_instance_stays_finite():
    """A 24-qubit p = 4 QAOA instance whose truncations discard about 3 % per update: its norm decays
    to about 1e-18, which once put the eigensolvers' absolute safeguards out of scale."""
    circs = W.qaoa_batch(4096, seed=W.MASTER_SEED + 3)
    c = circs[3187]
    assert c.n == 24 and len(c.ops) > 1000
    traces = {}
    for prec in ("mixed", "fp64"):
        st = G.run_circuit(c, 32, 8, prec)
        traces[prec] = st.trace()[0]
        pos = {v: i for i, v in enumerate(c.meta["perm"])}
        mc = st.maxcut([(pos[u], pos[v]) for u, v in c.meta["edges"]])[0]
        assert np.isfinite(mc) and 0 <= mc <= len(c.meta["edges"])
        disc = st.discarded()[0]
        assert 0 < disc[0] < 2 * len(c.ops) and 0 < disc[1] < 2 * len(c.ops)
    assert 0 < traces["fp64"] < 1e-6 and 0 < traces["mixed"] < 1e-6


@pytest.mark.parametrize("prec", ["mixed", "fp32", "fp64"])
def test_trace_far_below_the_fp32_range(prec):
    """kappa_max = 1 after strong damping and depolarizing keeps about half of the weight per 1q gate,
    so 100 layers take Tr rho to about 1e-53: complex64 sites would underflow without the per-chain
    power-of-two scale, which the TRACE readout multiplies back in.  Every cut is well separated."""
    rng = np.random.default_rng(1400)
    n = 4
    chis = [(1, W.kraus_to_chi(W.compose(W.amplitude_damping(0.5), W.depolarizing_1q(0.6)))),
            (2, W.kraus_to_chi([np.eye(4)]))]
    ops = []
    for layer in range(100):
        ops += [W.Op(1, q, W.random_unitary(2, rng), 0) for q in range(n)]
        ops += [W.Op(2, q, W.random_unitary(4, rng), 1) for q in range(layer % 2, n - 1, 2)]
    circ = W.Circuit(n, ops, chis)
    st = G.run_circuit(circ, 16, 1, prec)
    orc = OM.run_circuit(circ, 16, 1)
    assert orc.trace() < 1e-45 and allowance(orc, prec) == 0
    # the trace is a product of 400 truncations' kept weights: relative error about 400 times the
    # per-truncation bound
    assert abs(st.trace()[0] / orc.trace() - 1) < 400 * TRACE_TOL[prec]
    zz = st.zz_map()[0]
    assert np.max(np.abs(zz - orc.zz_map())) < MODES_READOUT[prec]
