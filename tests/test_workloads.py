"""Host-side checks of the seeded input generators (no method arithmetic lives there, but the circuits
must have the structure the workloads state): 3-regular graphs, the SWAP-network routing of QAOA, the
crosstalk layer structure, channel validity, reproducibility and the surrogate features."""
import math

import numpy as np
import pytest

from paper_2508_07610_gb300 import workloads as W


@pytest.mark.parametrize("n", [4, 8, 14, 24])
def test_random_regular3_is_simple_and_cubic(n):
    rng = np.random.default_rng(n)
    edges = W.random_regular3(n, rng)
    assert len(edges) == 3 * n // 2
    assert len(set(edges)) == len(edges)
    deg = np.zeros(n, dtype=int)
    for a, b in edges:
        assert a != b and 0 <= a < n and 0 <= b < n
        deg[a] += 1
        deg[b] += 1
    assert np.all(deg == 3)


@pytest.mark.parametrize("n,p", [(4, 1), (8, 2), (10, 3)])
def test_qaoa_swap_network_meets_every_edge_once_per_layer(n, p):
    """Each layer is n rounds of odd-even transpositions (a full reversal of the chain), so every pair
    of vertices is adjacent exactly once; the cost gate is applied exactly at the graph's edges."""
    rng = np.random.default_rng(100 + n)
    edges = W.random_regular3(n, rng)
    g = rng.uniform(0.1, 1.0, size=p)
    b = rng.uniform(0.1, 1.0, size=p)
    c = W.qaoa_maxcut(n, p, edges, g, b, rng)
    ops = c.ops
    assert [op.kind for op in ops[:n]] == [1] * n  # the H layer
    k = n
    pos = list(range(n))
    eset = {tuple(sorted(e)) for e in edges}
    for layer in range(p):
        met = []
        for rnd in range(n):
            for q in range(rnd % 2, n - 1, 2):
                op = ops[k]
                k += 1
                assert op.kind == 2 and op.q == q
                pair = tuple(sorted((pos[q], pos[q + 1])))
                is_cost = not np.allclose(op.U, W.swap())
                assert is_cost == (pair in eset)
                if is_cost:
                    met.append(pair)
                    assert np.allclose(op.U, W.swap() @ W.qaoa_cost(g[layer]))
                pos[q], pos[q + 1] = pos[q + 1], pos[q]
        assert sorted(met) == sorted(eset)  # every edge exactly once
        for q in range(n):
            assert ops[k].kind == 1 and np.allclose(ops[k].U, W.qaoa_mixer(b[layer]))
            k += 1
    assert k == len(ops)
    assert c.meta["perm"] == pos


def test_crosstalk_layers():
    n, depth = 10, 4
    c = W.crosstalk_sweep(n=n, depth=depth)
    k = 0
    for layer in range(depth):
        assert all(op.kind == 1 for op in c.ops[k:k + n])
        k += n
        active = list(range(layer % 2, n - 1, 2))
        for q in active:
            assert c.ops[k].kind == 2 and c.ops[k].q == q and np.allclose(c.ops[k].U, W.cz())
            k += 1
        idle = [nb for q in active for nb in (q - 1, q + 1) if 0 <= nb < n - 1 and nb not in active]
        for nb in idle:
            assert c.ops[k].kind == 2 and c.ops[k].q == nb and np.allclose(c.ops[k].U, np.eye(4))
            k += 1
    assert all(op.kind == 1 for op in c.ops[k:])
    assert len(c.ops) - k == n


@pytest.mark.parametrize("maker", [lambda: W.ghz_ansatz(), lambda: W.hea(n=6, depth=3), lambda: W.crosstalk_sweep(6, 3),
                                   lambda: W.qaoa_batch(3, n_choices=(6,), p_max=2)[1],
                                   lambda: W.unified_noise_circuit(4, 2, np.random.default_rng(0)),
                                   lambda: W.unified_noise_circuit(4, 2, np.random.default_rng(0), model="general")])
def test_channels_are_valid_process_matrices(maker):
    c = maker()
    for nq, chi in c.chis:
        d = 4 ** nq
        assert chi.shape == (d, d)
        assert np.allclose(chi, chi.conj().T, atol=1e-14)
        assert abs(np.trace(chi) - 1) < 1e-12
        assert np.linalg.eigvalsh(chi).min() > -1e-12


def test_generators_are_reproducible():
    a, b = W.hea(n=6, depth=2), W.hea(n=6, depth=2)
    assert all(np.array_equal(x.U, y.U) and x.q == y.q for x, y in zip(a.ops, b.ops))
    assert all(np.array_equal(x[1], y[1]) for x, y in zip(a.chis, b.chis))
    q1, q2 = W.qaoa_batch(4, seed=5), W.qaoa_batch(4, seed=5)
    assert [c.n for c in q1] == [c.n for c in q2]
    assert all(c1.meta["edges"] == c2.meta["edges"] for c1, c2 in zip(q1, q2))


def test_surrogate_features_pad_to_four_layers():
    rng = np.random.default_rng(3)
    edges = W.random_regular3(8, rng)
    c = W.qaoa_maxcut(8, 2, edges, [0.5, 1.0], [0.25, 2.0], rng)
    f = W.surrogate_features(c)
    assert f.shape == (16,) and f.dtype == np.float32
    assert np.allclose(f[:4], np.array([0.5, 1.0, 0, 0]) / math.pi, atol=1e-7)
    assert np.allclose(f[4:8], np.array([0.25, 2.0, 0, 0]) / math.pi, atol=1e-7)
    assert np.all(f[8:11] > 0)  # mean p1, p2, gamma (phi's mean has either sign)
    assert np.all(f[12:16] >= 0)  # spreads


# ------------------------------------------------------------------ Sec. II.B channel generators
def _apply(kraus, rho):
    return sum(K @ rho @ K.conj().T for K in kraus)


def test_thermal_relaxation_closed_form():
    """Population of |1> decays as exp(-t/T1), coherences as exp(-t/T2); trace preserving."""
    t, T1, T2 = 0.7, 2.0, 1.5
    K = W.thermal_relaxation(t, T1, T2)
    assert np.allclose(sum(k.conj().T @ k for k in K), np.eye(2), atol=1e-14)
    out = _apply(K, np.array([[0, 0], [0, 1]], dtype=complex))
    assert abs(out[1, 1] - math.exp(-t / T1)) < 1e-14 and abs(out[0, 0] - (1 - math.exp(-t / T1))) < 1e-14
    plus = np.full((2, 2), 0.5, dtype=complex)
    out = _apply(K, plus)
    assert abs(out[0, 1] - 0.5 * math.exp(-t / T2)) < 1e-14
    # T2 = 2 T1: no pure dephasing, the channel is amplitude damping alone
    assert abs(W.phase_damping(1.0)[1]).max() == 0
    with pytest.raises(ValueError):
        W.thermal_relaxation(1.0, 1.0, 2.5)


def test_spam_channels_closed_form():
    e01, e10, p = 0.02, 0.07, 0.1
    R = W.readout_error(e01, e10)
    assert np.allclose(sum(k.conj().T @ k for k in R), np.eye(2), atol=1e-15)
    for pop1 in (0.0, 0.3, 1.0):
        rho = np.array([[1 - pop1, 0.2], [0.2, pop1]], dtype=complex)
        out = _apply(R, rho)
        assert abs(out[1, 1] - (pop1 * (1 - e10) + (1 - pop1) * e01)) < 1e-15
        assert abs(out[0, 1]) < 1e-15  # a measurement leaves no coherence
    out = _apply(W.state_prep_error(p), np.array([[1, 0], [0, 0]], dtype=complex))
    assert abs(out[1, 1] - p) < 1e-15


def test_unified_model_depolarizes_only_the_target():
    """Fig. 1b: the two-qubit channel's depolarizing part acts on the target (second) qubit only."""
    from oracle import channels as OC
    p = 0.2
    sup = OC.superop(W.on_qubit(W.depolarizing_1q(p), 1))
    ref = OC.superop([np.kron(np.eye(2), K) for K in W.depolarizing_1q(p)])
    assert np.allclose(sup, ref, atol=1e-15)
    rho = np.zeros((4, 4), dtype=complex)
    rho[0, 0] = 1  # |00>: control untouched, target mixed towards I/2
    out = _apply(W.on_qubit(W.depolarizing_1q(p), 1), rho)
    assert abs(out[0, 0] - (1 - p / 2)) < 1e-15 and abs(out[1, 1] - p / 2) < 1e-15 and abs(out[2, 2]) < 1e-15
    c = W.unified_noise_circuit(3, 2, np.random.default_rng(1))
    assert [o.kind for o in c.ops[:3]] == [1, 1, 1] and [o.kind for o in c.ops[-3:]] == [1, 1, 1]
