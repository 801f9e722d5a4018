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
