"""Pins for the CPU MPDO reference: exact agreement with the dense simulator when nothing is
truncated, the Eckart-Young identity of Sec. II.D for every truncation, canonical-form
invariants, and the readouts against their dense definitions."""
import numpy as np
import pytest

from oracle import channels as C
from oracle import dense as D
from oracle import mpdo as M
from paper_2508_07610_gb300 import workloads as W


@pytest.mark.parametrize("seed", range(5))
def test_no_truncation_matches_dense(seed):
    rng = np.random.default_rng(seed)
    n = 4
    circ = W.random_circuit(n, 12, rng, rank1=3, rank2=5)
    rho = D.run_circuit(circ)
    st = M.run_circuit(circ, chi_max=64, kappa_max=4096)
    assert st.discarded_chi < 1e-24 and st.discarded_kappa < 1e-24
    assert np.max(np.abs(st.dense() - rho)) < 1e-12
    assert abs(st.trace() - 1) < 1e-12
    for i in range(n):
        for j in range(i + 1, n):
            assert abs(st.expect_zz(i, j) - D.expect_zz(rho, n, i, j)) < 1e-12
    assert abs(st.ghz_fidelity() - D.ghz_fidelity(rho, n)) < 1e-12
    assert abs(st.purity() - D.purity(rho)) < 1e-12


def test_ghz_ansatz_small_no_truncation():
    circ = W.ghz_ansatz(n=4, depth=2)
    rho = D.run_circuit(circ)
    st = M.run_circuit(circ, chi_max=64, kappa_max=4096)
    assert np.max(np.abs(st.dense() - rho)) < 1e-12
    assert abs(st.ghz_fidelity() - D.ghz_fidelity(rho, 4)) < 1e-12


def test_eckart_young_kraus_truncation():
    rng = np.random.default_rng(11)
    st = M.MPDO(3, 16, 3)
    st.auto_truncate = False
    circ = W.random_circuit(3, 8, rng, rank1=4, rank2=8)
    kr = [C.chi_to_kraus(chi, nq) for nq, chi in circ.chis]
    for op in circ.ops:
        (st.apply_1q if op.kind == 1 else st.apply_2q)(op.q, op.U, kr[op.chan])
    q = 1
    st.move_centre(q)
    A = st.sites[q].copy()
    full = np.sum(np.abs(A) ** 2)
    w = st.truncate_kraus(q, kappa=2)
    B = st.sites[q]
    # ||T - T'||_F^2 / ||T||_F^2 with T' = T V V^dag, computed from the kept tensor T V
    dl, _, dn, dr = A.shape
    Tm = A.transpose(0, 1, 3, 2).reshape(-1, dn)
    Bm = B.transpose(0, 1, 3, 2).reshape(-1, B.shape[2])
    V = np.linalg.lstsq(Tm, Bm, rcond=None)[0]
    err = np.sum(np.abs(Tm - Bm @ V.conj().T) ** 2) / full
    assert w > 1e-6
    assert abs(err - w) < 1e-12
    # and it is the best rank-2 approximation: no other rank-2 projector does better
    for _ in range(20):
        Z = np.linalg.qr(rng.normal(size=(dn, 2)) + 1j * rng.normal(size=(dn, 2)))[0]
        assert np.sum(np.abs(Tm - Tm @ Z @ Z.conj().T) ** 2) / full >= w - 1e-12


def test_bond_truncation_weight_matches_state_error():
    # With the centre on the pair, the discarded bond weight equals the squared distance between
    # the purified states before and after the split (Eckart-Young on the two-site matrix).
    rng = np.random.default_rng(5)
    n = 4
    circ = W.random_circuit(n, 10, rng, rank1=2, rank2=4)
    kr = [C.chi_to_kraus(chi, nq) for nq, chi in circ.chis]
    big = M.MPDO(n, 64, 4096)
    small = M.MPDO(n, 64, 4096)
    for op in circ.ops:
        for st in (big, small):
            (st.apply_1q if op.kind == 1 else st.apply_2q)(op.q, op.U, kr[op.chan])
    small.chi_max = 3
    U = W.random_unitary(4, rng)
    kr2 = W.random_channel_kraus(2, 3, rng)
    big.auto_truncate = small.auto_truncate = False
    big.apply_2q(1, U, kr2)
    small.apply_2q(1, U, kr2)
    w = small.log[-1][4]
    assert w > 1e-8
    # the kept part is orthogonal to the dropped part, so Tr rho_small = (1 - w) Tr rho_big
    assert abs(small.trace() - (1 - w) * big.trace()) < 1e-12


def test_canonical_form_after_moves():
    rng = np.random.default_rng(8)
    circ = W.random_circuit(5, 14, rng)
    st = M.run_circuit(circ, 8, 4)
    for c in (0, 4, 2):
        st.move_centre(c)
        for q in range(c):
            A = st.sites[q]
            m = A.reshape(-1, A.shape[3])
            assert np.allclose(m.conj().T @ m, np.eye(m.shape[1]), atol=1e-12)
        for q in range(c + 1, 5):
            A = st.sites[q]
            m = A.reshape(A.shape[0], -1)
            assert np.allclose(m @ m.conj().T, np.eye(m.shape[0]), atol=1e-12)
        # with the centre at c, Tr rho is the squared norm of the centre tensor
        assert abs(st.trace() - np.sum(np.abs(st.sites[c]) ** 2)) < 1e-12


def test_truncated_state_is_valid_density_matrix():
    circ = W.ghz_ansatz(n=6, depth=3)
    st = M.run_circuit(circ, 4, 2)
    rho = st.dense()
    rho = rho / np.trace(rho)
    assert np.max(np.abs(rho - rho.conj().T)) < 1e-13
    assert np.linalg.eigvalsh(rho).min() > -1e-13
    assert st.discarded_chi > 0 and st.discarded_kappa > 0


def test_readouts_against_dense_under_truncation():
    circ = W.ghz_ansatz(n=6, depth=3)
    st = M.run_circuit(circ, 6, 3)
    rho = st.dense()
    assert abs(st.ghz_fidelity() - D.ghz_fidelity(rho, 6)) < 1e-12
    assert abs(st.purity() - D.purity(rho)) < 1e-12
    edges = [(0, 1), (1, 2), (2, 5), (0, 4)]
    assert abs(st.maxcut(edges) - D.maxcut_expectation(rho, 6, edges)) < 1e-12
    zz = st.zz_map()
    for i in range(6):
        for j in range(6):
            if i != j:
                assert abs(zz[i, j] - D.expect_zz(rho, 6, i, j)) < 1e-12


def test_truncation_converges_with_caps():
    circ = W.ghz_ansatz(n=4, depth=2)
    rho = D.run_circuit(circ)
    f_exact = D.ghz_fidelity(rho, 4)
    errs = []
    for chi, kap in [(2, 1), (4, 2), (8, 4), (64, 4096)]:
        errs.append(abs(M.run_circuit(circ, chi, kap).ghz_fidelity() - f_exact))
    assert errs[-1] < 1e-12
    assert errs[0] > errs[-1]


# ------------------------------------------------------------------ the parity allowance at degenerate cuts
def _readouts(st):
    return np.concatenate([st.zz_map().ravel(), [st.ghz_fidelity(), st.purity()]])


def _perturbed_spread(circ, chi, kap, eps, seeds=6):
    """Largest readout change over runs whose every truncated matrix is perturbed by eps (relative)."""
    base = M.run_circuit(circ, chi, kap)
    r0 = _readouts(base)
    d = max(float(np.max(np.abs(_readouts(M.run_circuit(circ, chi, kap, perturb=(eps, np.random.default_rng(s))))
                                - r0))) for s in range(seeds))
    return base, d


def _degenerate_cut_circuit():
    """DEP2(p) on |00>: the Kraus-leg Gram has eigenvalues (1 - 3p/4, p/4, p/4, p/4) (Sec. II.A's Kraus
    set), so kappa = 2 cuts inside an exactly threefold cluster; later entangling gates make the choice
    of the kept direction visible in the readouts."""
    rng = np.random.default_rng(7)
    chis = [(2, W.kraus_to_chi(W.depolarizing_2q(0.05))), (2, W.kraus_to_chi([np.eye(4)]))]
    ops = [W.Op(2, 0, np.eye(4, dtype=np.complex128), 0)]
    ops += [W.Op(2, q, W.random_unitary(4, rng), 1) for q in (1, 0, 1)]
    return W.Circuit(3, ops, chis)


def test_cut_allowance_bounds_a_degenerate_cut():
    circ = _degenerate_cut_circuit()
    for eps in (1e-13, 1e-7):  # FP64-like and complex64-like rounding
        base, d = _perturbed_spread(circ, 8, 2, eps)
        gaps = [g for g, _, _ in base.cuts]
        assert min(gaps) < 1e-12                       # the cut is exactly degenerate
        a = base.cut_allowance(1e-9)
        assert a == base.cut_allowance(1e-5) > 0
        assert d > 1e-3                                # the choice of subspace moves the readouts ...
        assert d <= a                                  # ... by no more than the allowance
        assert a < 10 * d                              # and the allowance is not vacuous (4 x p/4 / Tr rho)


@pytest.mark.parametrize("seed", range(3))
def test_cut_allowance_is_zero_for_separated_cuts(seed):
    rng = np.random.default_rng(1000 + seed)
    circ = W.random_circuit(5, 20, rng, rank1=3, rank2=6)
    base, d = _perturbed_spread(circ, 3, 2, 1e-13, seeds=3)
    assert base.min_gap > 1e-3
    assert base.cut_allowance(1e-5) == 0.0 and base.cut_allowance(1e-9) == 0.0
    # rounding-level perturbations move the readouts only to first order in eps / gap
    assert d < 1e-10
    assert d < base.min_gap and d * base.min_gap / 1e-13 < 1.0


# ------------------------------------------------------------------ truncation order (Sec. II.D schedules)
@pytest.mark.parametrize("seed", range(3))
def test_kraus_first_equals_split_first_when_the_bond_is_not_cut(seed):
    """With chi_max at least every bond's rank the split is exact, and the Kraus leg of site q+1 after
    the split has the same Gram (ancilla density) as the merged tensor's leg: both orders keep the
    same subspace and give the same state."""
    rng = np.random.default_rng(300 + seed)
    circ = W.random_circuit(4, 14, rng, rank1=3, rank2=6)
    a = M.run_circuit(circ, 4096, 3, trunc_order="split_first")
    b = M.run_circuit(circ, 4096, 3, trunc_order="kraus_first")
    assert a.discarded_chi < 1e-24 and b.discarded_chi < 1e-24
    assert a.discarded_kappa > 1e-6
    assert abs(a.discarded_kappa - b.discarded_kappa) < 1e-12
    assert np.max(np.abs(a.dense() - b.dense())) < 1e-12


def test_kraus_first_exact_when_caps_cover_ranks():
    rng = np.random.default_rng(17)
    circ = W.random_circuit(4, 12, rng, rank1=3, rank2=5)
    st = M.run_circuit(circ, 64, 4096, trunc_order="kraus_first")
    assert st.discarded_chi < 1e-24 and st.discarded_kappa < 1e-24
    assert np.max(np.abs(st.dense() - D.run_circuit(circ))) < 1e-12


def test_kraus_first_under_truncation_is_a_valid_state_close_to_split_first():
    circ = W.ghz_ansatz(n=6, depth=3)
    exact = D.run_circuit(circ)
    a = M.run_circuit(circ, 6, 2)
    b = M.run_circuit(circ, 6, 2, trunc_order="kraus_first")
    rho = b.dense() / b.trace()
    assert np.max(np.abs(rho - rho.conj().T)) < 1e-13
    assert np.linalg.eigvalsh(rho).min() > -1e-13
    assert b.discarded_chi > 0 and b.discarded_kappa > 0
    # both schedules approximate the same exact state about equally well
    ea = abs(a.ghz_fidelity() - D.ghz_fidelity(exact, 6))
    eb = abs(b.ghz_fidelity() - D.ghz_fidelity(exact, 6))
    assert eb < 10 * ea + 1e-3 and ea < 10 * eb + 1e-3
    # every kappa cut of kraus_first happens inside the two-qubit update (no separate truncation of q+1)
    assert sum(1 for e in b.log if e[0] == "kappa") == sum(1 for e in a.log if e[0] == "kappa")


# ------------------------------------------------------------------ global bond truncation (Sec. II.D, Fig. 3b)
def _purified(sites):
    """psi[(p_0, n_0), (p_1, n_1), ...] contracted from the site tensors by plain einsums."""
    psi = np.ones((1, 1), dtype=np.complex128)  # [left block, bond]
    for A in sites:
        dl, _, dn, dr = A.shape
        psi = np.einsum("xl,lpnr->xpnr", psi, A).reshape(-1, dr)
    return psi[:, 0]


def _rho_of_purified(psi, n, dns):
    """rho = sum over every Kraus index of psi psi^dag, psi indexed [(p_0, n_0), ..., (p_{n-1}, n_{n-1})]."""
    T = psi.reshape([x for dn in dns for x in (2, dn)])
    phys = list(range(0, 2 * n, 2))
    kr = list(range(1, 2 * n, 2))
    T = T.transpose(phys + kr).reshape(2 ** n, -1)
    return T @ T.conj().T


def _noisy_state(n, seed, rank1=3, rank2=6, ops=14):
    rng = np.random.default_rng(seed)
    circ = W.random_circuit(n, ops, rng, rank1=rank1, rank2=rank2)
    return M.run_circuit(circ, 4096, 4096), circ


def test_global_bond_truncation_exact_when_chi_covers_ranks():
    st, circ = _noisy_state(4, 40)
    rho = st.dense()
    w = st.truncate_bonds(max(st.bond_dims()))
    assert w < 1e-24
    assert st.centre == 0
    assert np.max(np.abs(st.dense() - rho)) < 1e-12
    assert np.max(np.abs(rho - D.run_circuit(circ))) < 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_global_bond_truncation_is_sequential_eckart_young(seed):
    """The sweep keeps, at every cut from the right end to the left, the best rank-chi approximation
    of the purified state across that cut (Eckart-Young applied to the whole state vector, cut by
    cut, in the sweep's order); its discarded weights are those of the dropped Schmidt values."""
    n = 4
    st, _ = _noisy_state(n, 50 + seed)
    dns = st.kraus_dims()
    psi = _purified(st.sites)
    chi = 2
    ref_w = []
    for c in range(n - 1, 0, -1):
        left = int(np.prod([2 * d for d in dns[:c]]))
        Psi = psi.reshape(left, -1)
        Um, s, Vh = np.linalg.svd(Psi, full_matrices=False)
        nz = int(np.sum(s > 1e-13 * s[0]))
        k = min(chi, nz)
        ref_w.append(float(np.sum(s[k:] ** 2) / np.sum(s ** 2)))
        psi = ((Um[:, :k] * s[:k]) @ Vh[:k]).reshape(-1)
    assert max(ref_w) > 1e-4
    st.truncate_bonds(chi)
    got_w = [e[4] for e in st.log if e[0] == "chi"][-(n - 1):]
    assert np.allclose(got_w, ref_w, atol=1e-12)
    assert max(st.bond_dims()) <= chi
    assert np.max(np.abs(st.dense() - _rho_of_purified(psi, n, dns))) < 1e-12


def test_global_bond_truncation_leaves_right_isometries():
    st, _ = _noisy_state(5, 60)
    st.truncate_bonds(3)
    for c in range(1, st.n):
        A = st.sites[c]
        Am = A.reshape(A.shape[0], -1)
        assert np.max(np.abs(Am @ Am.conj().T - np.eye(A.shape[0]))) < 1e-12


# ------------------------------------------------------------------ three-qubit channels (Fig. 13b)
@pytest.mark.parametrize("seed", [504, 506, 507])
def test_three_qubit_channels_match_dense_without_truncation(seed):
    rng = np.random.default_rng(seed)
    circ = W.random_circuit(4, 10, rng, rank1=2, rank2=3, p3q=0.4, rank3=4)
    assert any(op.kind == 3 for op in circ.ops)
    st = M.run_circuit(circ, 4096, 4096)
    assert st.discarded_chi < 1e-24 and st.discarded_kappa < 1e-24
    assert np.max(np.abs(st.dense() - D.run_circuit(circ))) < 1e-12


def test_three_qubit_update_of_a_two_qubit_channel_equals_the_two_qubit_update():
    """A channel acting as identity on the third qubit gives the state of the two-qubit update."""
    rng = np.random.default_rng(41)
    base = W.random_circuit(4, 8, rng, rank1=2, rank2=3)
    kr2 = W.random_channel_kraus(2, 3, rng)
    U2 = W.random_unitary(4, rng)
    a = M.run_circuit(base, 4096, 4096)
    b = M.run_circuit(base, 4096, 4096)
    a.apply_2q(1, U2, kr2)
    b.apply_3q(1, np.kron(U2, np.eye(2)), [np.kron(K, np.eye(2)) for K in kr2])
    assert np.max(np.abs(a.dense() - b.dense())) < 1e-12


def test_three_qubit_split_weights_match_state_error():
    """Each of the two splits is an Eckart-Young truncation: with the centre on the first site the
    discarded weights add up to the squared distance of the purified states."""
    rng = np.random.default_rng(43)
    st = M.MPDO(4, 2, 4096)
    st.auto_truncate = False
    circ = W.random_circuit(4, 10, rng, rank1=2, rank2=3)
    kr = [C.chi_to_kraus(chi, nq) for nq, chi in circ.chis]
    for op in circ.ops:
        (st.apply_1q if op.kind == 1 else st.apply_2q)(op.q, op.U, kr[op.chan])
    exact = M.MPDO(4, 4096, 4096)
    exact.sites = [A.copy() for A in st.sites]
    exact.centre = st.centre
    U = W.random_unitary(8, rng)
    k3 = W.random_channel_kraus(3, 3, rng)
    exact.auto_truncate = False
    exact.apply_3q(0, U, k3)
    st.apply_3q(0, U, k3)
    w1, w2 = st.log[-2][4], st.log[-1][4]
    assert w1 > 1e-6 and w2 > 1e-6
    # both splits keep at most chi_max, and the truncated state stays a valid density matrix
    assert max(st.bond_dims()) <= 2
    rho = st.dense() / st.trace()
    assert np.max(np.abs(rho - rho.conj().T)) < 1e-13 and np.linalg.eigvalsh(rho).min() > -1e-13
    # Eckart-Young on the first split: the kept weight is the top-chi Schmidt weight of the exact state
    ex = exact.dense()
    assert abs(st.trace() - exact.trace() * (1 - w1) * (1 - w2)) < 1e-12 * exact.trace()


@pytest.mark.parametrize("order", ["split_first", "kraus_first"])
def test_trace_never_grows_op_by_op(order):
    """The premise of the library's trace guard: the channels are trace preserving and every
    truncation (Kraus leg, bond split, three-site splits, the global bond sweep) only removes weight,
    so Tr rho is non-increasing op by op, and it strictly drops at a cut that discards weight."""
    rng = np.random.default_rng(404)
    circ = W.random_circuit(6, 40, rng, rank1=3, rank2=6, p3q=0.2)
    ops = list(circ.ops)
    ops.insert(20, W.sweep_op(2))
    kraus = [C.chi_to_kraus(chi, nq) for nq, chi in circ.chis]
    st = M.MPDO(6, 4, 2, trunc_order=order)
    prev, drops = st.trace(), 0
    for op in ops:
        before = st.discarded_chi + st.discarded_kappa
        if op.kind == 8:
            st.truncate_bonds(op.q)
        else:
            (st.apply_1q, st.apply_2q, st.apply_3q)[op.kind - 1](op.q, op.U, kraus[op.chan])
        tr = st.trace()
        assert tr <= prev * (1 + 1e-12), (op.kind, tr, prev)
        if st.discarded_chi + st.discarded_kappa > before + 1e-9:
            assert tr < prev
            drops += 1
        prev = tr
    assert drops > 10
