"""Parity at the full size of the headline workload, in the configuration the
benchmark times.

The workload is 256^3 cells x 64 groups (35.2 GB of FP64 state), built from
the same preset and seed as the benchmark; the learned warm start is trained
with the benchmark's recipe (2^21 solver-labelled cells, 4 epochs).  Each
form is one call over all cells on one stream, as the benchmark launches it:
the mixed form from the warm start (the headline) and the plain FP64 form
(its comparison).  The oracle cannot solve 16.8M cells, so it solves a sample
of them (the first and last cell and 510 spread over the grid) one by one
from their inputs, read before the call; properties that hold at any size
(energy and momentum conservation, the fraction of cells at an iteration
cap) are checked over the whole grid on the device.
"""
import numpy as np
import pytest
import torch

from paper_2407_18304_gb300 import rhd, surrogate, synth
from parity import MAX_UNCONVERGED, agreed, converged, errors, run_oracle, select

pytestmark = pytest.mark.gpu

WORKLOAD = "full_256cube_ng64"
N_SAMPLE = 512
MIXED_BOUND = 1e-6
DEFAULT_FLOOR = 10 * 1e-11 / MIXED_BOUND


@pytest.fixture(scope="module")
def full():
    dev = torch.device("cuda", 0)
    w = synth.preset(WORKLOAD, device=dev)
    n = w.n_cells
    assert n == 256 ** 3 and w.n_groups == 64
    rng = np.random.default_rng(2407)
    idx = np.unique(np.concatenate([[0, n - 1], rng.choice(np.arange(1, n - 1), N_SAMPLE - 2,
                                                           replace=False)]))
    tidx = torch.as_tensor(idx, device=dev)
    sample = {k: (None if v is None else v.cpu()) for k, v in synth.take_cells(w.state, tidx).items()}
    ws = synth.Workload("sample", sample, w.edges, w.law, dt=w.dt, c_v=w.c_v, consts=dict(w.consts))
    o = run_oracle(ws)
    yield w, tidx, ws, o
    del w
    torch.cuda.empty_cache()


def _conservation_bound(G):
    """Worst-case rounding of the write-back and of the G-term sums on both
    sides (unit round-off 2^-53 per addition, relative to the summed
    magnitudes)."""
    return (2 * G + 16) * 2.0 ** -53


def _whole_grid(w, st, status):
    """Relative change of total energy and momentum per cell (max over the
    grid) and the fraction of cells at an iteration cap."""
    s0 = w.state
    c, c_hat = w.consts["c"], w.consts["c_hat"]
    r = c / c_hat
    l1 = lambda x, d: torch.linalg.vector_norm(x, ord=1, dim=d)
    src = 0.0 if s0.get("src") is None else s0["src"].sum(0)
    e0 = s0["egas"] + r * (s0["erad"].sum(0) + src)
    e1 = st["egas"] + r * st["erad"].sum(0)
    es = s0["egas"].abs() + r * (l1(s0["erad"], 0) + l1(st["erad"], 0))
    m0 = s0["mom"] + s0["frad"].sum(1) / (c * c_hat)
    m1 = st["mom"] + st["frad"].sum(1) / (c * c_hat)
    ms = s0["mom"].abs() + (l1(s0["frad"], 1) + l1(st["frad"], 1)) / (c * c_hat)
    ce = float(((e1 - e0).abs() / es).max())
    cm = float(((m1 - m0).abs() / ms).max())
    capped = float((status >= rhd.STATUS_MAXITER).float().mean())
    return ce, cm, capped


def _solve(w, precision, sur=None):
    st = synth.clone_state(w.state)
    n = w.n_cells
    status = torch.full((n,), 255, dtype=torch.uint8, device=st["rho"].device)
    iters = torch.zeros(n, dtype=torch.uint8, device=st["rho"].device)
    args = dict(dt=w.dt, c_v=w.c_v, consts=w.consts, precision=precision, status=status,
                iters=iters, stream=torch.cuda.current_stream(), flags=0)
    if sur is None:
        rhd.source_update(st, w.edges, w.law, **args)
    else:
        sur.source_update(st, w.edges, w.law, **args)
    torch.cuda.synchronize()
    return st, status, iters


def _sampled(st, status, iters, tidx):
    g = synth.to_numpy(synth.take_cells(st, tidx))
    g["status"] = status[tidx].cpu().numpy().astype(np.int32)
    g["iters"] = iters[tidx].cpu().numpy().astype(np.int32)
    return g


def test_headline_mixed_with_warm_start_at_full_size(full):
    w, tidx, ws, o = full
    _, _, vmax, taumax, _ = synth.PRESETS[WORKLOAD]
    sur = rhd.Surrogate(w.n_groups, 1)
    x, y = surrogate.training_set(sur, 1 << 21, w.edges, w.law, v_max=vmax, tau_max=taumax,
                                  seed=9_000_000, device=w.state["rho"].device)
    surrogate.train(sur, x, y, epochs=4, batch=8192, seed=0)
    del x, y
    st, status, iters = _solve(w, rhd.MIXED, sur)
    assert sur.error_flag() == 0
    assert int((status == 255).sum()) == 0
    ce, cm, capped = _whole_grid(w, st, status)
    print(f"whole grid: energy {ce:.2e}, momentum {cm:.2e}, capped {capped:.2e}, "
          f"fallback {float((status == rhd.STATUS_FALLBACK).float().mean()):.2e}, "
          f"mean Newton iterations {float(iters.float().mean()):.2f}")
    assert ce < _conservation_bound(w.n_groups) and cm < _conservation_bound(w.n_groups)
    assert capped <= MAX_UNCONVERGED
    g = _sampled(st, status, iters, tidx)
    del st
    torch.cuda.empty_cache()
    st0 = synth.to_numpy(ws.state)
    ok = agreed("mixed+surrogate at full size", g, oracle=o, fallback_ok=True)
    e = errors(select(g, ok), select(o, ok), select(st0, ok), w.consts["c"], w.c_v,
               floor=DEFAULT_FLOOR)
    print("sampled mixed+surrogate", " ".join(f"{k}={v:.2e}" for k, v in e.items()))
    assert e["T"] < MIXED_BOUND
    assert e["erad"] < MIXED_BOUND and e["egas"] < MIXED_BOUND


def test_fp64_form_at_full_size(full):
    """The benchmark's comparison form at the default tolerances: energies
    agree with the oracle's root on the scale the stopping test controls."""
    w, tidx, ws, o = full
    st, status, iters = _solve(w, rhd.FP64)
    assert int((status == 255).sum()) == 0
    ce, cm, capped = _whole_grid(w, st, status)
    print(f"whole grid: energy {ce:.2e}, momentum {cm:.2e}, capped {capped:.2e}, "
          f"mean Newton iterations {float(iters.float().mean()):.2f}")
    assert ce < _conservation_bound(w.n_groups) and cm < _conservation_bound(w.n_groups)
    assert capped <= MAX_UNCONVERGED
    g = _sampled(st, status, iters, tidx)
    del st
    torch.cuda.empty_cache()
    st0 = synth.to_numpy(ws.state)
    ok = agreed("fp64_form_at_full_size", g, oracle=o)
    g, oo, st0 = select(g, ok), select(o, ok), select(st0, ok)
    c = w.consts["c"]
    etot = st0["egas"] + st0["erad"].sum(0)
    d_egas = np.abs(g["egas"] - oo["egas"]) / etot
    d_erad = np.abs(g["erad"] - oo["erad"]).sum(0) / etot
    d_frad = np.linalg.norm(g["frad"] - oo["frad"], axis=0).sum(0) / (c * etot)
    print("sampled fp64", d_egas.max(), d_erad.max(), d_frad.max())
    assert d_egas.max() < 1e-10 and d_erad.max() < 1e-10 and d_frad.max() < 1e-10
