"""Pins of the FP64 reference network (oracle/mlp.py) against things other
than itself: finite differences, exact special cases, the exact GELU and
hand-rounded bfloat16 values."""
import math

import numpy as np
import pytest

from oracle import mlp as M

N_IN, N_OUT = 12, 5


def _norm(rng):
    return np.concatenate([rng.normal(0, 1, N_IN), rng.uniform(0.5, 2.0, N_IN),
                           rng.normal(0, 1, N_OUT), rng.uniform(0.5, 2.0, N_OUT)])


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    p = M.init_params(N_IN, N_OUT, 1)
    norm = _norm(rng)
    x = rng.normal(0, 1.5, (16, N_IN))
    y = rng.normal(0, 1.0, (16, N_OUT))
    L, g = M.loss_grad(p, norm, x, y, N_IN, N_OUT)
    assert abs(L - M.loss(p, norm, x, y, N_IN, N_OUT)) < 1e-15 * max(1.0, L)
    idx = rng.choice(len(p), 60, replace=False)
    # include biases and every layer
    offs = np.cumsum([0] + [o * i + o for o, i in M.shapes(N_IN, N_OUT)])
    idx = np.unique(np.concatenate([idx, offs[:-1], offs[1:] - 1]))
    for k in idx:
        h = 1e-6 * max(1.0, abs(p[k]))
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (M.loss(pp, norm, x, y, N_IN, N_OUT) - M.loss(pm, norm, x, y, N_IN, N_OUT)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-6, np.abs(g).max()), (k, fd, g[k])


def test_zero_weights_give_the_output_bias():
    rng = np.random.default_rng(2)
    p = M.init_params(N_IN, N_OUT, 3)
    Ws, bs = M.unpack(p, N_IN, N_OUT)
    off = sum(o * i + o for o, i in M.shapes(N_IN, N_OUT)[:3])
    p[off:off + N_OUT * M.H] = 0.0  # W4 = 0
    b4 = p[off + N_OUT * M.H:]
    out, _ = M.forward(p, _norm(rng), rng.normal(0, 1, (7, N_IN)), N_IN, N_OUT)
    assert np.array_equal(out, np.broadcast_to(b4, out.shape))


def test_tanh_gelu_is_close_to_the_exact_gelu():
    z = np.linspace(-8, 8, 4001)
    exact = np.array([0.5 * t * (1.0 + math.erf(t / math.sqrt(2.0))) for t in z])
    assert np.max(np.abs(M.gelu(z) - exact)) < 5e-4  # known bound of the tanh form: 4.7e-4
    # its derivative against a difference quotient
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - M.gelu_grad(z))) < 1e-8


@pytest.mark.parametrize("value,expected", [
    (1.0, 1.0),
    (1.0 + 2.0 ** -9, 1.0),                            # below half an ulp (2^-7)
    (1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7),            # above half an ulp
    (1.0 + 2.0 ** -8, 1.0),                            # tie, to the even neighbour
    (1.0 + 2.0 ** -7 + 2.0 ** -8, 1.0 + 2.0 ** -6),    # tie, to the even neighbour
    (-2.5, -2.5),
    (65504.0, 65536.0),                                # 2^16 - 2^5 rounds up to 2^16
])
def test_bf16_rounding(value, expected):
    assert float(M.bf16(np.array([value]))[0]) == expected


def test_single_path_network_by_hand():
    """A network with one live path fixes the parameter layout ([W (out x in)
    row-major, b] per layer), the standardisation of x and the mapping of the
    output back to raw units: input j -> hidden unit 2 -> unit 5 -> unit 7 ->
    every output, the other hidden units carrying only their biases."""
    rng = np.random.default_rng(5)
    norm = _norm(rng)
    xm, xs = norm[:N_IN], norm[N_IN:2 * N_IN]
    ym, ys = norm[2 * N_IN:2 * N_IN + N_OUT], norm[2 * N_IN + N_OUT:]
    shp = M.shapes(N_IN, N_OUT)
    offs = np.cumsum([0] + [o * i + o for o, i in shp])
    p = np.zeros(offs[-1])
    j, w1, w2, w3 = 3, 0.7, -1.3, 0.9
    w4 = rng.normal(0, 1, N_OUT)
    b = [rng.normal(0, 0.2, o) for o, _ in shp]
    for l, (o, i) in enumerate(shp):
        p[offs[l] + o * i:offs[l + 1]] = b[l]
    p[offs[0] + 2 * N_IN + j] = w1                 # W1[2, j]
    p[offs[1] + 5 * M.H + 2] = w2                  # W2[5, 2]
    p[offs[2] + 7 * M.H + 5] = w3                  # W3[7, 5]
    p[offs[3] + np.arange(N_OUT) * M.H + 7] = w4   # W4[k, 7]
    x = rng.normal(0, 1.5, (9, N_IN))
    a1 = M.gelu(w1 * (x[:, j] - xm[j]) / xs[j] + b[0][2])
    a2 = M.gelu(w2 * a1 + b[1][5])
    a3 = M.gelu(w3 * a2 + b[2][7])
    out = a3[:, None] * w4[None, :] + b[3][None, :]
    np.testing.assert_allclose(M.predict(p, norm, x, N_IN, N_OUT), out * ys + ym, rtol=1e-14, atol=1e-14)


def test_loss_is_the_mean_square_of_standardised_errors():
    """With W4 = 0 and b4 = 0 the output is zero, so the loss is the mean over
    rows and outputs of ((y - y_mean)/y_sd)^2."""
    rng = np.random.default_rng(6)
    norm = _norm(rng)
    ym, ys = norm[2 * N_IN:2 * N_IN + N_OUT], norm[2 * N_IN + N_OUT:]
    p = M.init_params(N_IN, N_OUT, 7)
    off = sum(o * i + o for o, i in M.shapes(N_IN, N_OUT)[:3])
    p[off:] = 0.0
    x = rng.normal(0, 1, (11, N_IN))
    y = rng.normal(0, 2, (11, N_OUT))
    expect = sum(((y[r, k] - ym[k]) / ys[k]) ** 2 for r in range(11) for k in range(N_OUT)) / (11 * N_OUT)
    assert M.loss(p, norm, x, y, N_IN, N_OUT) == pytest.approx(expect, rel=1e-14)
    L, _ = M.loss_grad(p, norm, x, y, N_IN, N_OUT)
    assert L == pytest.approx(expect, rel=1e-14)
