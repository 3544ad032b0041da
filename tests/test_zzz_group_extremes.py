"""Parity at the extreme group counts, in both precisions, against the oracle.

The small end is one to three groups, the smallest problems the method has.
One group over [0, inf) in PC mode is the grey problem, and 1-3 groups run
the same one-cell-per-thread kernel as 4 to 16.  The large end is 129 and 256
(RHD_MAX_GROUPS) groups, which run the one-cell-per-thread kernel with
256-wide arrays.  A ragged cell count is used, above one CTA where the oracle
allows.  This file is collected after every other test file, so a failure
here comes after every other test has run.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2407_18304_gb300 import rhd, synth
from parity import MAX_UNCONVERGED, agreed, conservation, converged, errors, run_gpu, run_oracle, select

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
TIGHT = dict(tol=1e-14, tol_outer=1e-15)
FLOOR = 10 * TIGHT["tol"] / FP64_TOL
MIXED_BOUND = 1e-6
MIXED_FLOOR = 10 * 1e-11 / MIXED_BOUND

_CASES = {}


def _case(G):
    """Workload and oracle result for G groups (cached: both precisions
    compare with the same oracle run)."""
    if G not in _CASES:
        if G == 0:  # one PC group over all frequencies
            st = synth.make_state(257, synth.log_edges(1), synth.powerlaw_law(0.0), v_max=1e-2,
                                  tau_max=1e4, seed=501)
            w = synth.Workload("pc_one_group", st, np.array([0.0, math.inf]), synth.powerlaw_law(0.0))
            _CASES[G] = (w, run_oracle(w, mode=O.PC), rhd.PC)
        else:
            n = 257 if G <= 3 else 33
            w = synth.preset("mixed_128cube_ng16", n_cells=n, seed=500 + G, n_groups=G)
            _CASES[G] = (w, run_oracle(w), rhd.PPL_FIXED)
    return _CASES[G]


@pytest.mark.parametrize("G", [0, 1, 2, 3, 129, 256], ids=["1_pc_0_inf", "1", "2", "3", "129", "256"])
@pytest.mark.parametrize("precision", [rhd.FP64, rhd.MIXED], ids=["fp64", "mixed"])
def test_extreme_group_counts(G, precision):
    w, o, mode = _case(G)
    kw = TIGHT if precision == rhd.FP64 else {}
    g = run_gpu(w, precision=precision, mode=mode, **kw)
    st0 = synth.to_numpy(w.state)
    ok = agreed("extreme_group_counts", g, oracle=o)
    floor = FLOOR if precision == rhd.FP64 else MIXED_FLOOR
    e = errors(select(g, ok), select(o, ok), select(st0, ok), w.consts["c"], w.c_v,
               floor=floor)
    print(f"G={w.n_groups} {w.name} precision={precision}",
          " ".join(f"{k}={v:.2e}" for k, v in e.items()))
    ce, cm = conservation(select(g, ok), select(st0, ok), w.consts["c"], w.consts["c_hat"])
    bound = (2 * w.n_groups + 16) * 2.0 ** -53
    assert ce < max(bound, 64 * 2.0 ** -52) and cm < max(bound, 64 * 2.0 ** -52)
    if precision == rhd.FP64:
        for k, v in e.items():
            if not k.endswith("_plain"):
                assert v < FP64_TOL, (k, v)
    else:
        for k in ("T", "egas", "erad"):
            assert e[k] < MIXED_BOUND, (k, e[k])


@pytest.mark.parametrize("preset", ["mixed_128cube_ng16", "full_256cube_ng64"])
@pytest.mark.parametrize("precision", [rhd.FP64, rhd.MIXED], ids=["fp64", "mixed"])
def test_transparent_cells_are_left_unchanged(preset, precision):
    """kappa_0 = 0: no group couples to the gas (tau = 0), so R_g = 0 in
    eq. Rnew, the flux update of eq. fupdate returns F_g^t, and the
    write-back leaves E_g, E_gas and rho v as they were; every third cell is
    transparent, among ordinary cells (one cell per thread at 16 groups, a
    warp per cell at 64)."""
    w = synth.preset(preset, n_cells=301, seed=91)
    st = {k: (None if v is None else v.clone()) for k, v in w.state.items()}
    clear = np.arange(301) % 3 == 0
    st["kappa0"][torch.as_tensor(clear)] = 0.0
    w = synth.Workload(w.name, st, w.edges, w.law)
    g = run_gpu(w, precision=precision)
    s0 = synth.to_numpy(st)
    assert np.all(g["status"][clear] == 0), np.bincount(g["status"][clear])
    # E_g = E_g^t + 0 and E_gas = E_gas^t - (c/c_hat) 0 exactly; F_g = F_g^t up to the
    # rounding of x (1/x) in the flux update's shared reciprocal (one ulp)
    for k in ("egas", "erad", "frad"):
        np.testing.assert_allclose(g[k][..., clear], s0[k][..., clear], rtol=4 * 2.0 ** -52, atol=0,
                                   err_msg=k)
    # rho v changes by those flux roundings over (c c_hat): measured on the cell's
    # total momentum, gas plus radiation
    c, c_hat = w.consts["c"], w.consts["c_hat"]
    ms = np.abs(s0["mom"]) + np.abs(s0["frad"]).sum(1) / (c * c_hat)
    dm = np.abs(g["mom"] - s0["mom"])
    assert np.all(dm[:, clear] <= 4 * w.n_groups * 2.0 ** -52 * ms[:, clear])
    # the oracle agrees on the transparent cells
    o = run_oracle(w)
    np.testing.assert_allclose(o["erad"][:, clear], s0["erad"][:, clear], rtol=1e-14, atol=0)
