"""Learned surrogate for the noisy-QAOA variational loop (binding of include/surrogate.h) and the
screening loop around it.

The surrogate maps 16 features (QAOA angles padded to p = 4, and the means and spreads of the
channel strengths) to the predicted <H_MaxCut>/|E| and GHZ fidelity of the noisy circuit.  It is
trained on samples the batched MPDO produces, screens many candidate angle sets at once, and the
MPDO re-scores the best few; when the surrogate's error on those exceeds the threshold the loop
falls back to the MPDO alone.
"""
from __future__ import annotations

import ctypes as C
import math
from typing import List, Optional

import numpy as np

from . import batched as BR
from . import mpdo as G
from . import workloads as W

IN_DIM, HIDDEN, N_HIDDEN, OUT_DIM = 16, 256, 3, 2


def _lib():
    L = G.lib()
    if getattr(L, "_surr_ready", False):
        return L
    vp, fp, dp, i32 = C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_double), C.c_int
    sig = {
        "surr_create": [i32, i32, i32, i32, i32, C.c_ulonglong, vp, C.POINTER(vp)],
        "surr_free": [vp],
        "surr_get_params": [vp, fp],
        "surr_set_params": [vp, fp],
        "surr_forward": [vp, vp, i32, vp],
        "surr_gradients": [vp, vp, vp, i32, dp],
        "surr_get_grads": [vp, fp],
        "surr_adamw": [vp, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float],
        "surr_train_step": [vp, vp, vp, i32, C.c_float, C.c_float, dp],
        "surr_sync": [vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.surr_num_params.argtypes = [vp]
    L.surr_num_params.restype = C.c_longlong
    L._surr_ready = True
    return L


def _check(st, where):
    if st != 0:
        raise RuntimeError(f"{where}: surrogate status {st}")


class Surrogate:
    def __init__(self, torch, max_batch: int = 65536, seed: int = 1, dims=(IN_DIM, HIDDEN, N_HIDDEN, OUT_DIM),
                 stream: int = 0):
        L = _lib()
        self.torch = torch
        self.in_dim, self.hidden, self.n_hidden, self.out_dim = dims
        self.max_batch = max_batch
        h = C.c_void_p()
        _check(L.surr_create(self.in_dim, self.hidden, self.n_hidden, self.out_dim, max_batch, seed,
                             C.c_void_p(stream or None), C.byref(h)), "surr_create")
        self.h = h
        self.n_params = int(L.surr_num_params(h))
        self.dims = [self.in_dim] + [self.hidden] * self.n_hidden + [self.out_dim]

    def free(self):
        if getattr(self, "h", None):
            _lib().surr_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def sync(self):
        """Wait for the handle's stream; raises if a tensor-core launch gave up waiting."""
        _check(_lib().surr_sync(self.h), "surr_sync")

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(_lib().surr_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float))), "surr_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(_lib().surr_set_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float))), "surr_set_params")

    def grads(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(_lib().surr_get_grads(self.h, out.ctypes.data_as(C.POINTER(C.c_float))), "surr_get_grads")
        return out

    def forward(self, X):
        """X: torch float32 CUDA tensor (batch x 16) -> torch float32 CUDA tensor (batch x 2)."""
        t = self.torch
        Y = t.empty((X.shape[0], self.out_dim), dtype=t.float32, device=X.device)
        for s in range(0, X.shape[0], self.max_batch):
            e = min(X.shape[0], s + self.max_batch)
            _check(_lib().surr_forward(self.h, C.c_void_p(X[s:e].data_ptr()), e - s, C.c_void_p(Y[s:e].data_ptr())),
                   "surr_forward")
        return Y

    def gradients(self, X, T) -> float:
        loss = C.c_double()
        _check(_lib().surr_gradients(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()), X.shape[0],
                                     C.byref(loss)), "surr_gradients")
        return loss.value

    def adamw(self, lr, b1=0.9, b2=0.999, eps=1e-8, wd=1e-2):
        _check(_lib().surr_adamw(self.h, lr, b1, b2, eps, wd), "surr_adamw")

    def train(self, X, T, epochs: int = 200, batch: int = 4096, lr: float = 1e-3, wd: float = 1e-2,
              seed: int = 0) -> List[float]:
        """AdamW with a cosine learning-rate schedule over shuffled minibatches; returns the epoch losses."""
        t = self.torch
        g = t.Generator(device="cpu").manual_seed(seed)
        n = X.shape[0]
        steps = epochs * max(1, n // batch)
        losses, k = [], 0
        for ep in range(epochs):
            perm = t.randperm(n, generator=g).to(X.device)
            tot = 0.0
            nb = max(1, n // batch)
            for bi in range(nb):
                idx = perm[bi * batch:(bi + 1) * batch]
                xb, tb = X[idx].contiguous(), T[idx].contiguous()
                lr_k = lr * 0.5 * (1 + math.cos(math.pi * k / steps))
                loss = C.c_double()
                _check(_lib().surr_train_step(self.h, C.c_void_p(xb.data_ptr()), C.c_void_p(tb.data_ptr()),
                                              xb.shape[0], lr_k, wd, C.byref(loss)), "surr_train_step")
                tot += loss.value
                k += 1
            losses.append(tot / nb)
        return losses


# ------------------------------------------------------------------------- data from the MPDO
def sample_circuits(count: int, n: int, edges, rng, p_choices=(1, 2, 3, 4), scale_range=(0.5, 2.0)):
    """Noisy QAOA circuits on one fixed graph: p ~ U(p_choices), angles ~ U(0, pi), per-sample noise
    strength scale ~ U(scale_range)."""
    out = []
    for _ in range(count):
        p = int(rng.choice(p_choices))
        g = rng.uniform(0, math.pi, size=p)
        b = rng.uniform(0, math.pi, size=p)
        s = rng.uniform(*scale_range)
        out.append(W.qaoa_maxcut(n, p, edges, g, b, rng, scale=s))
    return out


def mpdo_targets(circs, chi: int, kappa: int, prec: str, torch) -> np.ndarray:
    """<H_MaxCut>/|E| and GHZ fidelity of every circuit, from the batched MPDO."""
    run = BR.BatchedRun(circs, chi, kappa, prec, torch=torch)
    run.run()
    mc = run.maxcut()
    ghz = run.ghz()
    run.free()
    ne = np.array([len(c.meta["edges"]) for c in circs])
    return np.stack([mc / ne, ghz], axis=1).astype(np.float32)


def features(circs) -> np.ndarray:
    return np.stack([W.surrogate_features(c) for c in circs])


def angle_features(template, gammas: np.ndarray, betas: np.ndarray, p_max: int = 4) -> np.ndarray:
    """Features of many candidate angle sets (rows of gammas, betas) that share the channels of one
    QAOA circuit `template`: the angles padded to p_max and divided by pi, then the template's
    noise descriptors (W.surrogate_features layout)."""
    base = W.surrogate_features(template, p_max)
    N, p = gammas.shape
    X = np.tile(base, (N, 1))
    X[:, :p_max] = 0.0
    X[:, p_max:2 * p_max] = 0.0
    X[:, :p] = gammas / math.pi
    X[:, p_max:p_max + p] = betas / math.pi
    return X.astype(np.float32)


def mpdo_scores(template, gammas, betas, chi, kappa, prec, torch) -> np.ndarray:
    """<H_MaxCut>/|E| of the candidates (rows of gammas, betas) on the template's channels, by the
    batched MPDO."""
    circs = [W.qaoa_with_angles(template, g, b) for g, b in zip(gammas, betas)]
    return mpdo_targets(circs, chi, kappa, prec, torch)[:, 0]


def screen(model: Surrogate, X: np.ndarray, score, top: int = 64, tol: float = 1e-2):
    """One screened step of the variational loop.  The surrogate ranks all candidates (rows of the
    feature matrix X) by predicted <H_MaxCut>/|E|; score(indices) evaluates the `top` best with the
    MPDO.  The answer is the best MPDO-scored candidate.  When the surrogate's root-mean-square error
    on the scored set exceeds tol its ranking is not trusted (fallback): the loop should score
    candidates with the MPDO alone from then on; the MPDO evaluations already made are kept, so the
    budget is the same either way.  Returns (best index, its MPDO score, surrogate error, fell back)."""
    t = model.torch
    pred = model.forward(t.tensor(X, device="cuda"))[:, 0].cpu().numpy()
    order = np.argsort(-pred)[:top]
    scored = np.asarray(score(order))
    err = float(np.sqrt(np.mean((scored - pred[order]) ** 2)))
    b = int(np.argmax(scored))
    return int(order[b]), float(scored[b]), err, err > tol


def generate_training_set(count: int, n: int, edges, seed: int, chi: int, kappa: int, prec: str, torch,
                          p_choices=(1, 2, 3, 4), scale_range=(0.5, 2.0), chunk: int = 4096,
                          checkpoint: Optional[str] = None):
    """`count` (features, targets) pairs from the batched MPDO, generated in chunks of `chunk` samples.
    Chunk c draws its circuits from its own seed (seed, c), so the set does not depend on how it was
    split.  With a checkpoint path every finished chunk is saved there (NumPy .npz) and a later call
    resumes after the last saved chunk."""
    Xs, Ys = [], []
    if checkpoint:
        try:
            with np.load(checkpoint) as f:
                Xs = [f["X"][i:i + chunk] for i in range(0, f["X"].shape[0], chunk)]
                Ys = [f["Y"][i:i + chunk] for i in range(0, f["Y"].shape[0], chunk)]
        except (FileNotFoundError, OSError, KeyError):
            Xs, Ys = [], []
    # only whole chunks are kept (every chunk is generated in full and the result cut to count)
    Xs = [x for x in Xs if x.shape[0] == chunk]
    Ys = Ys[:len(Xs)]
    done = chunk * len(Xs)
    while done < count:
        c = done // chunk
        m = chunk
        rng = np.random.default_rng([seed, c])
        circs = sample_circuits(m, n, edges, rng, p_choices, scale_range)
        Xs.append(features(circs))
        Ys.append(mpdo_targets(circs, chi, kappa, prec, torch))
        done += m
        if checkpoint:
            np.savez(checkpoint, X=np.concatenate(Xs), Y=np.concatenate(Ys))
    return np.concatenate(Xs)[:count], np.concatenate(Ys)[:count]
