"""Training driver of the learned spectral-radius predictor (sequencing of library kernels).

Every step of training runs in libue.so: features (ue_rho_features), BF16 tensor-core forward
(ue_mlp_forward), per-mesh max aggregation (ue_seg_argmax), loss gradient (ue_rho_loss),
backward on the argmax rows (ue_mlp_backward) and Adam (ue_adam).  This module only
allocates the device tensors (through PyTorch) and calls them in order.  Labels come from the
library's FP64 power iteration (ue_geometry_build with UE_DT_POWER), the "complex time" method
of the paper's Section 2.

``python -m paper_1812_01448_gb300.learned --out paper_1812_01448_gb300/rho_mlp.npy`` trains
the shipped weights (seeded corpus, seeded initialisation).
"""
from __future__ import annotations

import argparse
import math
import os

import numpy as np

from . import _native as N
from .api import Mesh, adam, mlp_backward, mlp_forward, rho_loss, seg_argmax

H, D = 64, 12
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rho_mlp.npy")


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded He initialisation (host).  The network is a correction on top of log sqrt(K_jj):
    w3 starts small and b3 at log 1.25, a typical rho / sqrt(max K_jj)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, D)) * math.sqrt(2.0 / D)
    W2 = rng.standard_normal((H, H)) * math.sqrt(2.0 / H)
    w3 = rng.standard_normal(H) * math.sqrt(1.0 / H) * 0.01
    p = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, [math.log(1.25)]])
    return p.astype(np.float32)


def load_weights(path: str = WEIGHTS) -> np.ndarray:
    p = np.load(path).astype(np.float32)
    if p.shape != (N.UE_MLP_PARAMS,):
        raise ValueError("bad weight file")
    return p


def build_corpus(meshes, stream=None, power_iters: int = 200):
    """Features, base terms, segment offsets and log rho_PI labels of a list of MeshArrays."""
    import torch
    Xs, Ls, offs, labels = [], [], [0], []
    for ms in meshes:
        m = Mesh(ms.xy, ms.tris)
        m.geometry_build(stream=stream, power_iters=power_iters)
        _, rho, _ = m.get_dt()
        X = torch.empty((m.n_tris, D), dtype=torch.float32, device="cuda")
        L = torch.empty(m.n_tris, dtype=torch.float32, device="cuda")
        m.rho_features(X, L, stream)
        m.close()
        Xs.append(X)
        Ls.append(L)
        offs.append(offs[-1] + X.shape[0])
        labels.append(math.log(rho))
    return dict(X=torch.cat(Xs), base=torch.cat(Ls),
                off=torch.tensor(offs, dtype=torch.int64, device="cuda"),
                target=torch.tensor(labels, dtype=torch.float32, device="cuda"))


def train(corpus, epochs: int = 2000, lr: float = 3e-3, seed: int = 0, bf16: bool = True,
          stream=None, params0: np.ndarray | None = None):
    """Adam on the mean over meshes of (log rho_hat - log rho_PI)^2.  Returns (params, losses)."""
    import torch
    X, base, off, target = corpus["X"], corpus["base"], corpus["off"], corpus["target"]
    M = target.shape[0]
    p = torch.from_numpy(params0 if params0 is not None else init_params(seed)).cuda()
    m1 = torch.zeros_like(p)
    m2 = torch.zeros_like(p)
    g = torch.zeros_like(p)
    z = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    best = torch.empty(M, dtype=torch.float32, device="cuda")
    arg = torch.empty(M, dtype=torch.int64, device="cuda")
    dz = torch.empty(M, dtype=torch.float32, device="cuda")
    loss = torch.empty(M, dtype=torch.float32, device="cuda")
    work = torch.empty((M, N.UE_MLP_PARAMS), dtype=torch.float32, device="cuda")
    hist = []
    for t in range(1, epochs + 1):
        mlp_forward(p, X, z, bf16, stream)
        seg_argmax(z, base, off, best, arg, stream)
        rho_loss(best, target, dz, loss, stream)
        mlp_backward(p, X, arg, dz, g, work, bf16, stream)
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * (t - 1) / epochs))   # cosine decay
        adam(p, g, m1, m2, t, lr=lr_t, stream=stream)
        if t % 50 == 0 or t == epochs:
            hist.append(float(loss.mean()))
    return p.cpu().numpy(), hist


def main(argv=None):
    import multiprocessing as mp

    import meshgen
    ap = argparse.ArgumentParser()
    ap.add_argument("--meshes", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--seed", type=int, default=1005)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--workers", type=int, default=0, help="mesh generator processes (0: all cores)")
    a = ap.parse_args(argv)
    import time
    t0 = time.perf_counter()
    specs = meshgen.learned_specs(a.meshes, seed=a.seed)
    # the pool is started (spawn) before the first GPU call; the meshes stream from it into
    # the corpus, which keeps only their features on the device
    workers = a.workers or min(32, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(workers) as pool:
        import torch
        torch.cuda.set_device(0)
        corpus = build_corpus(pool.imap(meshgen.learned_mesh, specs, chunksize=4))
    t1 = time.perf_counter()
    p, hist = train(corpus, epochs=a.epochs, seed=a.seed)
    t2 = time.perf_counter()
    np.save(a.out, p)
    print(f"trained on {a.meshes} meshes, {corpus['X'].shape[0]} triangles; "
          f"loss {hist[0]:.4g} -> {hist[-1]:.4g}; rms log error {math.sqrt(hist[-1]):.4f}; "
          f"corpus {t1 - t0:.0f} s ({workers} generator processes), training {t2 - t1:.0f} s")


if __name__ == "__main__":
    main()
