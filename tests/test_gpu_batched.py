"""The batched runtime (heterogeneous noisy QAOA MaxCut instances grouped by gate-position signature,
one CUDA graph per group) against the CPU oracle run instance by instance."""
import numpy as np
import pytest

from oracle import mpdo as OM
from paper_2508_07610_gb300 import batched as BR
from paper_2508_07610_gb300 import workloads as W
from tolerances import discarded_limit, readout_limit

pytestmark = pytest.mark.gpu


def _oracle_maxcut(c, chi, kap):
    o = OM.run_circuit(c, chi, kap)
    pos = {v: i for i, v in enumerate(c.meta["perm"])}
    return o.maxcut([(pos[u], pos[v]) for u, v in c.meta["edges"]]), o


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_qaoa_matches_oracle(prec):
    torch = pytest.importorskip("torch")
    circs = W.qaoa_batch(8, seed=W.MASTER_SEED + 33, n_choices=(4, 6), p_max=2)
    chi, kap = 8, 4
    run = BR.BatchedRun(circs, chi, kap, prec, stream=torch.cuda.Stream().cuda_stream, torch=torch)
    assert 1 < len(run.groups) < len(circs)  # some instances share a group, some do not
    run.run(graphs=True)
    mc = run.maxcut()
    disc = run.discarded()
    for i, c in enumerate(circs):
        ref, o = _oracle_maxcut(c, chi, kap)
        # <H_MaxCut> = sum over |E| edges of (1 - <Z Z>) / 2: |E| / 2 readouts of norm 1
        lim = readout_limit(o, prec, len(c.meta["edges"]) / 2)
        assert abs(mc[i] - ref) < lim, (i, mc[i], ref, lim)
        assert abs(disc[i, 0] - o.discarded_chi) < discarded_limit(o, prec, "chi")
        assert abs(disc[i, 1] - o.discarded_kappa) < discarded_limit(o, prec, "kappa")
    # replaying the graphs reproduces the result exactly
    run.run(graphs=True)
    assert np.array_equal(run.maxcut(), mc)


def test_ideal_qaoa_on_the_4_cycle_prefers_the_optimal_cut():
    """Noise-free QAOA p = 2 on the 4-cycle of Fig. 12 (vertices on a chain, edge 3-0 routed by the
    SWAP network): a coarse grid search finds angles whose <C> beats the |E|/2 of random guessing."""
    torch = pytest.importorskip("torch")
    edges = [(0, 1), (1, 2), (2, 3), (0, 3)]
    rng = np.random.default_rng(0)
    ideal1 = W.kraus_to_chi([np.eye(2)])
    ideal2 = W.kraus_to_chi([np.eye(4)])
    circs = []
    grid = [(g, b) for g in np.linspace(0.2, 1.4, 4) for b in np.linspace(0.2, 1.4, 4)]
    for g, b in grid:
        c = W.qaoa_maxcut(4, 2, edges, [g, g], [b, b], rng)
        c.chis = [(nq, ideal1 if nq == 1 else ideal2) for nq, _ in c.chis]
        circs.append(c)
    run = BR.BatchedRun(circs, 16, 1, "fp64", stream=torch.cuda.Stream().cuda_stream, torch=torch)
    assert len(run.groups) == 1
    run.run()
    mc = run.maxcut()
    assert mc.max() > 3.0 and mc.max() <= 4.0 + 1e-12
    for i in (0, int(np.argmax(mc))):
        ref, _ = _oracle_maxcut(circs[i], 16, 1)
        assert abs(mc[i] - ref) < 1e-10


def test_batched_qaoa_up_to_n12_mixed_matches_oracle():
    """Config-3 shaped instances (n in {8, 10, 12}, p in {1, 2}) through the batch ABI in MIXED, each
    against the oracle at the per-result bound."""
    torch = pytest.importorskip("torch")
    circs = W.qaoa_batch(16, seed=W.MASTER_SEED + 34, n_choices=(8, 10, 12), p_max=2)
    chi, kap = 16, 4
    run = BR.BatchedRun(circs, chi, kap, "mixed", torch=torch)
    run.run()
    mc = run.maxcut()
    worst = 0.0
    for i, c in enumerate(circs):
        ref, o = _oracle_maxcut(c, chi, kap)
        lim = readout_limit(o, "mixed", len(c.meta["edges"]) / 2)
        worst = max(worst, abs(mc[i] - ref))
        assert abs(mc[i] - ref) < lim, (i, c.n, mc[i], ref, lim)
    print(f"batched QAOA n<=12 mixed: largest |MaxCut - oracle| {worst:.2e} over {len(circs)} instances")


def test_autotuner_persists_and_reuses_schedules(tmp_path):
    """A group of 130 instances is timed over its schedules once; the choice is written to the JSON
    tuning file and a second batch built from the file takes it without timing; both give the same
    results."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    edges = W.random_regular3(4, rng)
    circs = [W.qaoa_maxcut(4, 1, edges, rng.uniform(0, np.pi, 1), rng.uniform(0, np.pi, 1), rng) for _ in range(130)]
    path = str(tmp_path / "tuning.json")
    a = BR.BatchedRun(circs, 8, 4, "mixed", torch=torch, tuning=path)
    (nq, chains, handles, tc, ms), = a.groups
    assert chains == 130 and handles in (1, 2, 4) and ms > 0
    text = open(path).read()
    assert '"key": "n=4' in text and f'"handles": {handles}' in text
    b = BR.BatchedRun(circs, 8, 4, "mixed", torch=torch, tuning=path)
    (nq2, chains2, handles2, tc2, ms2), = b.groups
    assert (nq2, chains2, handles2, tc2) == (nq, chains, handles, tc) and abs(ms2 - ms) < 1e-3
    a.run()
    b.run()
    assert np.max(np.abs(a.maxcut() - b.maxcut())) < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_global_bond_schedule_matches_oracle(prec):
    """Random RX/RY/RZ + CNOT circuits with the global bond truncation after every CNOT layer
    (MPDO_OP_TRUNCATE_BONDS ops) through the batch runtime, against the oracle's truncate_bonds."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(W.MASTER_SEED + 61)
    circs = [W.random_rot_cnot(6, 6, rng, sweep_chi=2) for _ in range(6)]
    cap, kap = 64, 2
    run = BR.BatchedRun(circs, cap, kap, prec, stream=torch.cuda.Stream().cuda_stream, torch=torch)
    run.run()
    ghz = run.ghz()
    disc = run.discarded()
    for i, c in enumerate(circs):
        o = OM.run_circuit(c, cap, kap)
        assert max(o.bond_dims()) <= 2 and o.discarded_chi > 1e-6
        assert abs(ghz[i] - o.ghz_fidelity()) < readout_limit(o, prec), (i, ghz[i], o.ghz_fidelity())
        assert abs(disc[i, 0] - o.discarded_chi) < discarded_limit(o, prec, "chi")
        assert abs(disc[i, 1] - o.discarded_kappa) < discarded_limit(o, prec, "kappa")
