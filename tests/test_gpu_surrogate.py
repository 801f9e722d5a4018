"""GPU surrogate (BF16 operands, FP32 accumulation) against the FP64 MLP reference, its training, and
the screened variational loop against the same loop without the surrogate."""
import math

import numpy as np
import pytest

from oracle import mlp as OM
from paper_2508_07610_gb300 import surrogate as S
from paper_2508_07610_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return pytest.importorskip("torch")


def test_forward_gradients_and_adamw_match_fp64(torch):
    model = S.Surrogate(torch, max_batch=1024, seed=3)
    dims = model.dims
    rng = np.random.default_rng(0)
    p = model.params().astype(np.float64)
    X = rng.normal(size=(512, 16)).astype(np.float32)
    T = rng.normal(scale=0.3, size=(512, 2)).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    # forward: BF16 weights/activations, FP32 accumulation -> about 1e-2 relative
    y = model.forward(Xd).cpu().numpy()
    y_ref = OM.forward(p, dims, X.astype(np.float64))
    rel = np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)
    assert rel < 2e-2, rel
    # gradients
    loss = model.gradients(Xd, Td)
    loss_ref, g_ref = OM.loss_and_grad(p, dims, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - loss_ref) < 2e-2 * loss_ref
    g = model.grads().astype(np.float64)
    for w, b, i, o in OM.layout(dims)[0]:
        for lo, hi in ((w, w + i * o), (b, b + o)):
            rel = np.linalg.norm(g[lo:hi] - g_ref[lo:hi]) / max(np.linalg.norm(g_ref[lo:hi]), 1e-30)
            assert rel < 3e-2, (lo, rel)
    # one AdamW step from the GPU's own gradients, in FP32 master precision
    opt = OM.AdamW(dims, lr=1e-3, wd=1e-2)
    p_ref = opt.step(p, g)
    model.adamw(1e-3, wd=1e-2)
    assert np.max(np.abs(model.params() - p_ref)) < 1e-6


def _bf16(x):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_forward_matches_bf16_rounded_reference(torch):
    """The forward pass (hidden layers on the tensor cores) against an FP64 evaluation that rounds the
    weights, the input and every hidden activation to BF16 as the kernels do: only the FP32 summation
    order differs, so the outputs agree far more closely than with the unrounded FP64 model; a
    layout or descriptor mistake in the tensor-core path would show as an O(1) difference."""
    model = S.Surrogate(torch, max_batch=4096, seed=9)
    dims = model.dims
    p = model.params().astype(np.float64)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(1000, 16)).astype(np.float32)  # 1000 rows: a ragged last 128-row tile
    layers, _ = OM.layout(dims)
    a = _bf16(X)
    for li, (w, b, i, o) in enumerate(layers):
        W = _bf16(p[w:w + i * o].reshape(o, i))
        z = a @ W.T + p[b:b + o]
        if li + 1 < len(layers):
            a = _bf16(OM.gelu(z))
        else:
            a = z
    y = model.forward(torch.tensor(X, device="cuda")).cpu().numpy()
    rel = np.linalg.norm(y - a) / np.linalg.norm(a)
    assert rel < 2e-3, rel
    assert model.sync() is None


def test_training_fits_a_smooth_function(torch):
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, size=(8192, 16)).astype(np.float32)
    T = np.stack([np.sin(X[:, 0] * 2) * 0.5 + 0.1 * X[:, 3], np.cos(X[:, 1]) * X[:, 2]], axis=1).astype(np.float32)
    model = S.Surrogate(torch, max_batch=4096, seed=5)
    losses = model.train(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), epochs=30, batch=1024,
                         lr=2e-3)
    assert losses[-1] < 0.05 * losses[0], losses[::5]


def test_screened_loop_beats_the_loop_without_the_surrogate(torch):
    """Train on MPDO-generated samples of noisy p = 1 QAOA on one fixed 8-vertex 3-regular graph (angles
    and noise strength varied), then with the
    same MPDO budget (64 re-scored candidates) the surrogate-screened search must find a better
    <H_MaxCut> than scoring 64 unscreened candidates."""
    rng = np.random.default_rng(W.MASTER_SEED + 5)
    n = 8
    edges = W.random_regular3(n, rng)
    chi, kap, prec = 16, 4, "mixed"
    train = S.sample_circuits(4096, n, edges, rng, p_choices=(1,))
    Y = S.mpdo_targets(train, chi, kap, prec, torch)
    X = S.features(train)
    model = S.Surrogate(torch, max_batch=4096, seed=11)
    Xd, Yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    losses = model.train(Xd, Yd, epochs=400, batch=256, lr=2e-3)
    assert losses[-1] < 0.1 * losses[0]
    # held-out error of the surrogate
    test = S.sample_circuits(256, n, edges, rng, p_choices=(1,))
    Yt = S.mpdo_targets(test, chi, kap, prec, torch)
    pt = model.forward(torch.tensor(S.features(test), device="cuda")).cpu().numpy()
    rmse = float(np.sqrt(np.mean((pt[:, 0] - Yt[:, 0]) ** 2)))
    print(f"surrogate held-out RMSE of <H_MaxCut>/|E|: {rmse:.4f}, final training loss {losses[-1]:.2e}")
    assert rmse < 0.05
    # screening: candidates at one noise setting, p = 1
    cand = []
    crng = np.random.default_rng(99)
    for _ in range(2048):
        g = crng.uniform(0, math.pi, size=1)
        b = crng.uniform(0, math.pi, size=1)
        cand.append(W.qaoa_maxcut(n, 1, edges, g, b, np.random.default_rng(7), scale=1.0))
    best_i, best_screened, err, fell_back = S.screen(model, cand, chi, kap, prec, torch, top=64, tol=0.05)
    unscreened = S.mpdo_targets(cand[:64], chi, kap, prec, torch)[:, 0]
    print(f"screened best {best_screened:.4f} (surrogate error {err:.3f}, fallback {fell_back}) "
          f"vs unscreened best {unscreened.max():.4f}")
    assert not fell_back
    assert best_screened > unscreened.max()
