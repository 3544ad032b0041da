"""Parity of the free-slope PPL mode (Appendix A, RHD_PPL_FREE) with the
oracle, through the C ABI.  The starting radiation spectra are Planck spectra
at a radiation temperature of their own, multiplied group by group by seeded
factors in [0.5, 2], so the fitted indices of E_nu differ from those of B_nu
and change sign between neighbouring groups (minmod takes all its branches).
Same measures and tolerance as the fixed-slope FP64 parity tests."""
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


def _workload(preset, n, G=None, seed=41):
    w = synth.preset(preset, n_cells=n, n_groups=G)
    g = torch.Generator().manual_seed(seed)
    f = torch.exp(np.log(2.0) * (2.0 * torch.rand(w.state["erad"].shape, generator=g,
                                                  dtype=torch.float64) - 1.0))
    w.state["erad"] = w.state["erad"] * f
    w.state["frad"] = w.state["frad"] * f[None]
    return w


def _check(w, g, o, name):
    st0 = synth.to_numpy(w.state)
    ok = agreed("_check", g, oracle=o)
    g, o, st0 = select(g, ok), select(o, ok), select(st0, ok)
    e = errors(g, o, st0, w.consts["c"], w.c_v, floor=FLOOR)
    print(name, " ".join(f"{k}={v:.2e}" for k, v in e.items()))
    ce, cm = conservation(g, st0, w.consts["c"], w.consts["c_hat"])
    assert ce < 64 * 2.0 ** -52 and cm < 64 * 2.0 ** -52
    for k, v in e.items():
        if not k.endswith("_plain"):
            assert v < FP64_TOL, (k, v)


@pytest.mark.parametrize("preset,n,G", [("tiny", 700, None), ("mixed_128cube_ng16", 1200, None),
                                        ("mixed_128cube_ng16", 300, 33),
                                        ("full_256cube_ng64", 200, None),
                                        ("mixed_128cube_ng16", 100, 100)])
def test_free_slopes_match_oracle(preset, n, G):
    w = _workload(preset, n, G)
    g = run_gpu(w, mode=rhd.PPL_FREE, **TIGHT)
    o = run_oracle(w, mode=O.PPL_FREE)
    _check(w, g, o, f"{preset} G={w.n_groups}")


@pytest.mark.parametrize("variant", ["src_theta_half", "temp_exponent", "mixed_precision"])
def test_free_slope_variants(variant):
    w = _workload("mixed_128cube_ng16", 600, seed=43)
    kw, ko = {}, {}
    if variant == "src_theta_half":
        src = 0.2 * w.state["erad"].flip(0).clone()
        w.state["src"] = src
        kw = ko = dict(theta=0.5)
    elif variant == "temp_exponent":
        kw = ko = dict(temp_exponent=-1.5, T_ref=synth.T_REF)
    else:
        kw = dict(precision=rhd.MIXED)
    g = run_gpu(w, mode=rhd.PPL_FREE, **TIGHT, **kw)
    o = run_oracle(w, mode=O.PPL_FREE, **ko)
    _check(w, g, o, variant)


def test_free_slopes_differ_from_fixed_and_batched_rejects_them():
    w = _workload("mixed_128cube_ng16", 256)
    a = run_gpu(w, mode=rhd.PPL_FREE, **TIGHT)
    b = run_gpu(w, mode=rhd.PPL_FIXED, **TIGHT)
    assert np.max(np.abs(a["erad"] - b["erad"]) / np.abs(b["erad"])) > 1e-6
    ctx = rhd.Context()
    st = {k: (None if v is None else v.cuda().clone()) for k, v in w.state.items()}
    spec = rhd.GridSpec(st, w.edges, w.law, dt=w.dt, c_v=w.c_v, consts=w.consts,
                        mode=rhd.PPL_FREE)
    with pytest.raises(rhd.RhdError):
        ctx.update([spec])
    torch.cuda.synchronize()
    ctx.close()
