"""FP64 reference of the learned warm start's network (plain numpy).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library.

The network (not in the paper; the paper's solver starts from the state at the
beginning of the step): standardised features x (2 N_g + 4) -> 128 -> 128 ->
128 -> N_g + 1 with the tanh form of GELU,
    gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))),
after the three hidden layers and a linear output; loss = mean over rows and
outputs of (y_pred - y)^2 on standardised targets.  The flat parameter vector
is [W1 (128 x n_in), b1, W2 (128 x 128), b2, W3, b3, W4 (n_out x 128), b4],
each W row-major [out][in].  The standardisation vector is
[x_mean, x_sd, y_mean, y_sd].

``bf16=True`` rounds to bfloat16 (round to nearest even) at the points where
the tensor-core path stores BF16 operands: the standardised inputs, every
weight matrix, every hidden activation after GELU, and, in the backward pass,
the output error dY and each dZ before they multiply a matrix (the bias
gradients use the unrounded values).  Everything else is FP64.

Parity status: pinned by central finite differences of the FP64 loss
(gradient), by the zero-weight special case (output = b4 exactly), by a
single-path network evaluated by hand (layout, standardisation and its
inverse), by the loss of a zero output, by the exact-GELU comparison (the tanh
form is within 5e-4 of z Phi(z)), and by hand-checked bfloat16 roundings
(``tests/test_oracle_mlp.py``).
"""
from __future__ import annotations

import math

import numpy as np

H = 128


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def gelu(z):
    k0 = math.sqrt(2.0 / math.pi)
    return 0.5 * z * (1.0 + np.tanh(k0 * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    k0 = math.sqrt(2.0 / math.pi)
    u = k0 * (z + 0.044715 * z ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * k0 * (1.0 + 3.0 * 0.044715 * z * z)


def shapes(n_in: int, n_out: int):
    return [(H, n_in), (H, H), (H, H), (n_out, H)]


def n_params(n_in: int, n_out: int) -> int:
    return sum(o * i + o for o, i in shapes(n_in, n_out))


def unpack(p: np.ndarray, n_in: int, n_out: int):
    """Weights and biases of the four layers from the flat vector."""
    Ws, bs, k = [], [], 0
    for o, i in shapes(n_in, n_out):
        Ws.append(np.asarray(p[k:k + o * i], dtype=np.float64).reshape(o, i))
        k += o * i
        bs.append(np.asarray(p[k:k + o], dtype=np.float64))
        k += o
    return Ws, bs


def standardise(x, y, norm, n_in, n_out):
    norm = np.asarray(norm, dtype=np.float64)
    xm, xs = norm[:n_in], norm[n_in:2 * n_in]
    ym, ys = norm[2 * n_in:2 * n_in + n_out], norm[2 * n_in + n_out:]
    xn = (np.asarray(x, dtype=np.float64) - xm) / xs
    yn = None if y is None else (np.asarray(y, dtype=np.float64) - ym) / ys
    return xn, yn, ym, ys


def forward(p, norm, x, n_in, n_out, bf=False):
    """Standardised outputs and the cache of the forward pass."""
    r = bf16 if bf else (lambda a: a)
    Ws, bs = unpack(p, n_in, n_out)
    xn, _, _, _ = standardise(x, None, norm, n_in, n_out)
    a = r(xn)
    acts, zs = [a], []
    for l in range(3):
        z = a @ r(Ws[l]).T + bs[l]
        zs.append(z)
        a = r(gelu(z))
        acts.append(a)
    out = a @ r(Ws[3]).T + bs[3]
    return out, (acts, zs, Ws)


def predict(p, norm, x, n_in, n_out, bf=False):
    """Raw (de-standardised) outputs."""
    out, _ = forward(p, norm, x, n_in, n_out, bf)
    _, _, ym, ys = standardise(x, None, norm, n_in, n_out)
    return out * ys + ym


def loss(p, norm, x, y, n_in, n_out, bf=False) -> float:
    out, _ = forward(p, norm, x, n_in, n_out, bf)
    _, yn, _, _ = standardise(x, y, norm, n_in, n_out)
    return float(np.mean((out - yn) ** 2))


def loss_grad(p, norm, x, y, n_in, n_out, bf=False):
    """Loss and its gradient with respect to the flat parameters (backprop)."""
    r = bf16 if bf else (lambda a: a)
    out, (acts, zs, Ws) = forward(p, norm, x, n_in, n_out, bf)
    _, yn, _, _ = standardise(x, y, norm, n_in, n_out)
    B = out.shape[0]
    L = float(np.mean((out - yn) ** 2))
    dy = 2.0 * (out - yn) / (B * n_out)
    gW, gb = [None] * 4, [None] * 4
    gb[3] = dy.sum(0)
    gW[3] = r(dy).T @ acts[3]
    dh = r(dy) @ r(Ws[3])
    for l in (2, 1, 0):
        dz = dh * gelu_grad(zs[l])
        gb[l] = dz.sum(0)
        gW[l] = r(dz).T @ acts[l]
        if l > 0:
            dh = r(dz) @ r(Ws[l])
    g = np.concatenate([np.concatenate([gW[l].ravel(), gb[l]]) for l in range(4)])
    return L, g


def init_params(n_in: int, n_out: int, seed: int) -> np.ndarray:
    """Random parameters for tests (uniform, He scale)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (o, i) in enumerate(shapes(n_in, n_out)):
        s = math.sqrt(6.0 / i) * (0.3 if l == 3 else 1.0)
        parts.append(rng.uniform(-s, s, o * i))
        parts.append(rng.uniform(-0.1, 0.1, o))
    return np.concatenate(parts)
