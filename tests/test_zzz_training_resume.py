"""Resuming the learned warm start's training from a checkpoint.

A surrogate loaded from ``rhd_surrogate_checkpoint``'s file (the parameters,
the standardisation, both Adam moments and the step count) takes the same
next Adam steps as the one that wrote it, bit for bit.  The training step is
deterministic: fixed-order reductions, tensor-core GEMMs, and zero-filled
padding.  A file of ``rhd_surrogate_save`` holds the network alone, so
training resumes with a fresh optimiser and the next step differs.  This file
is collected after every other test file.
"""
import pytest
import torch

from paper_2407_18304_gb300 import rhd, surrogate, synth

pytestmark = pytest.mark.gpu


def test_checkpoint_resumes_training_bit_for_bit(tmp_path):
    G, n, B, lr = 16, 4096, 512, 1e-3
    mult, add = 2053, 11  # odd, so the batch permutation mult * i + add mod 4096 is a bijection
    w = synth.preset("mixed_128cube_ng16", n_cells=16, seed=77)
    _, _, vmax, taumax, _ = synth.PRESETS["mixed_128cube_ng16"]
    a = rhd.Surrogate(G, 3)
    x, y = surrogate.training_set(a, n, w.edges, w.law, v_max=vmax, tau_max=taumax, seed=78,
                                  device="cuda")
    a.fit_normalization(x, y)
    for k in range(4):
        a.train_step(x, y, k * B, B, mult, add, lr)
    ck = str(tmp_path / "train_state.bin")
    a.checkpoint(ck)
    b = rhd.Surrogate.load(ck)
    pa, na = a.get_params()
    pb, nb = b.get_params()
    assert torch.equal(pa, pb) and torch.equal(na, nb)
    for k in range(4, 8):
        a.train_step(x, y, k * B, B, mult, add, lr)
        b.train_step(x, y, k * B, B, mult, add, lr)
    torch.cuda.synchronize()
    pa, pb = a.get_params()[0], b.get_params()[0]
    assert torch.equal(pa, pb), float((pa - pb).abs().max())
    # the network alone: Adam restarts (step 1 bias correction, zero moments)
    net = str(tmp_path / "net.bin")
    a.save(net)
    c = rhd.Surrogate.load(net)
    a.train_step(x, y, 0, B, mult, add, lr)
    c.train_step(x, y, 0, B, mult, add, lr)
    torch.cuda.synchronize()
    assert not torch.equal(a.get_params()[0], c.get_params()[0])
    assert a.error_flag() == 0 and b.error_flag() == 0 and c.error_flag() == 0
