"""Training and use of the learned surrogate of the spreading kernel (host orchestration only: the
features, the tensor-core convolutions, the loss, the gradients and the Adam update all run in
libfdirw through the C ABI).

Recipe: training structures are seeded sphere packings (porosity U[0.3, 0.5], per-sphere log10
diffusivity ratio U[3, 8]); their FD kernels (window R = 8, n_sub substeps at the stability limit) are
the targets; the network starts from a delta-kernel prior (the source marker routed to the head so that
z = 0 at the source and ln(1e-9) elsewhere) plus N(0, 0.02) noise, and is trained with Adam on the
generalised Kullback-Leibler divergence sum (y - k ln y + k ln k - k), y = exp(z), whose gradient y - k
penalises predicted mass wherever the FD kernel has less (the gate checks the total mass).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import fdirw, synth

EPS = 1e-9
LAYERS, TAPS, C = 4, 27, 16


def init_params(seed: int, noise: float = 0.02) -> np.ndarray:
    """Flat float32 parameter vector (weights [4][27][16 co][16 ci], biases [4][16]) of the delta prior."""
    rng = np.random.default_rng(seed)
    W = rng.normal(0.0, noise, size=(LAYERS, TAPS, C, C))
    b = np.zeros((LAYERS, C))
    centre = 13
    lnv = -np.log(EPS)
    W[0, centre, 0, :] = 0.0
    W[0, centre, 0, 2] = 1.0            # channel 0 <- source marker
    for l in (1, 2):
        W[l, centre, 0, :] = 0.0
        W[l, centre, 0, 0] = 1.0        # channel 0 passed on through the relu layers
    W[3, :, 1:, :] = 0.0                # the head uses output channel 0 only
    W[3, centre, 0, 0] = lnv
    b[3, 0] = -lnv
    return fdirw.pack_params(W, b)


@dataclasses.dataclass
class Sample:
    shape: tuple
    D: np.ndarray
    ctx: fdirw.FDiRW          # context of the structure (its D feeds the features)
    sources: np.ndarray
    targets: "object"         # torch tensor on the device, [n, 17, 17, 17] float64


def training_set(n_structures: int, per_structure: int, seed: int, side: int = 48, n_sub: int = 200,
                 device: int = -1):
    """FD kernels of `per_structure` random sources in each of `n_structures` seeded packings."""
    import torch
    out = []
    rng = np.random.default_rng(seed)
    for j in range(n_structures):
        shape = (side,) * 3
        p = synth.sphere_packing(shape, float(rng.uniform(0.3, 0.5)), seed * 1000 + j)
        D = synth.diffusivity_per_sphere(p)
        dt = fdirw.fdirw_stable_dt(shape, D, device=device)
        ctx = fdirw.FDiRW(shape, D, n_sub * dt, 8, n_sub, "fp32", device=device)
        ctx.kernels()
        src = rng.integers(0, side ** 3, per_structure)
        tg = torch.empty((per_structure, 17, 17, 17), dtype=torch.float64, device=f"cuda:{max(device, 0)}")
        for q0 in range(0, per_structure, 1024):
            tg[q0:q0 + 1024] = torch.from_numpy(ctx.read_kernels(src[q0:q0 + 1024])).to(tg.device)
        out.append(Sample(shape, D, ctx, src, tg))
    return out


def train(net: fdirw.Net, data, epochs: int, batch: int = 256, lr: float = 2e-3, seed: int = 0, log=None):
    """Adam over shuffled batches drawn within each structure; returns the mean loss of every epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        t0 = time.perf_counter()
        losses = []
        order = [(j, q) for j, s in enumerate(data) for q in range(0, len(s.sources), batch)]
        rng.shuffle(order)
        for j, q in order:
            s = data[j]
            perm = np.arange(q, min(q + batch, len(s.sources)))
            losses.append(net.train_step(s.ctx.ctx, s.sources[perm], s.targets[perm[0]:perm[-1] + 1], lr))
        hist.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e} ({time.perf_counter() - t0:.1f} s)")
    return hist


def train_rate(steps: int = 20, batch: int = 256, side: int = 64, seed: int = 20240827, device: int = 0) -> dict:
    """Wall time of `steps` training steps (features, four convolutions, loss, input and weight gradients of
    every layer, Adam; each step reads its loss back) on `batch` random sources of a seeded sphere packing,
    with targets already on the device; three untimed steps first."""
    import torch
    shape = (side,) * 3
    D = synth.diffusivity_per_sphere(synth.sphere_packing(shape, 0.4, seed))
    dt = fdirw.fdirw_stable_dt(shape, D, device=device)
    rng = np.random.default_rng(seed)
    src = rng.integers(0, side ** 3, batch)
    tg = torch.rand((batch, 17 ** 3), dtype=torch.float64, device=f"cuda:{device}",
                    generator=torch.Generator(device=f"cuda:{device}").manual_seed(seed)) * 1e-3
    with fdirw.FDiRW(shape, D, dt, 8, 1, "bf16", device=device) as f:
        net = fdirw.Net(init_params(seed), device=device)
        try:
            for _ in range(3):
                net.train_step(f.ctx, src, tg, 1e-4)
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            for _ in range(steps):
                net.train_step(f.ctx, src, tg, 1e-4)
            torch.cuda.synchronize(device)
            dt_step = (time.perf_counter() - t0) / steps
        finally:
            net.close()
    return {"batch": batch, "steps": steps, "train_step_ms": dt_step * 1e3, "samples_per_s": batch / dt_step}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Timing of the surrogate's training step")
    ap.add_argument("--train-rate", action="store_true", help="time training steps of 256 sources on a 64^3 packing")
    ap.add_argument("--steps", type=int, default=20)
    a = ap.parse_args()
    if a.train_rate:
        print(json.dumps(train_rate(a.steps)))
