"""Training data, training loop and evaluation of the learned warm start.

Orchestration only: the solves, features, targets, standardisation, network
passes and Adam steps all run in the CUDA library (``rhd.Surrogate``); this
module chooses seeds, batch order and learning rate and concatenates buffers.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import rhd, synth


def training_set(sur: rhd.Surrogate, n_cells: int, edges, law, *, v_max: float, tau_max: float,
                 seed: int, device, dt: float = synth.DT, c_v: float = synth.C_V,
                 consts: dict | None = None, chunk: int = 1 << 20):
    """Features and targets of n_cells synthetic cells (the recipe of
    ``synth.make_state``) advanced by the plain FP64 solver at the default
    tolerance."""
    consts = consts or synth.Workload("", {}, edges, law).consts
    xs, ys = [], []
    for c0 in range(0, n_cells, chunk):
        m = min(chunk, n_cells - c0)
        st = synth.make_state(m, edges, law, v_max=v_max, tau_max=tau_max, seed=seed + c0,
                              device=device)
        before = synth.clone_state(st)
        rhd.source_update(st, edges, law, dt=dt, c_v=c_v, consts=consts, precision=rhd.FP64)
        xs.append(sur.features(before, edges, law, dt=dt, c_v=c_v, consts=consts))
        ys.append(sur.targets(before, st, edges, law, dt=dt, c_v=c_v, consts=consts))
        del st, before
    return torch.cat(xs), torch.cat(ys)


def _coprime(n: int, rng) -> int:
    while True:
        a = int(rng.integers(1, max(2, n)))
        if math.gcd(a, n) == 1:
            return a


def train(sur: rhd.Surrogate, x: torch.Tensor, y: torch.Tensor, *, epochs: int = 4,
          batch: int = 4096, lr: float = 2e-3, lr_final: float = 2e-4, seed: int = 0) -> list:
    """Fit the standardisation, then Adam over shuffled batches (each epoch a
    permutation mult * i + add mod n); learning rate decays geometrically from
    lr to lr_final.  Returns the mean batch loss of every epoch."""
    sur.fit_normalization(x, y)
    n = x.shape[0]
    rng = np.random.default_rng(seed)
    steps = max(1, n // batch)
    losses = []
    loss = torch.zeros(1, dtype=torch.float32, device=x.device)
    total = epochs * steps
    k = 0
    for _ in range(epochs):
        mult, add = _coprime(n, rng), int(rng.integers(0, n))
        loss.zero_()
        for s in range(steps):
            a = lr * (lr_final / lr) ** (k / max(1, total - 1))
            sur.train_step(x, y, s * batch, batch, mult, add, a, loss)
            k += 1
        losses.append(float(loss.item()) / steps)
    return losses
