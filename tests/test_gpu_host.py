"""rhd_source_update_host: the state in host memory, streamed through the GPU
in chunks with the copies overlapped with the solve.  Cells are independent,
so every chunking must give the device entry's results bit for bit."""
import numpy as np
import pytest
import torch

from paper_2407_18304_gb300 import rhd, synth

pytestmark = pytest.mark.gpu


def _pinned(st):
    return {k: (None if v is None else v.cpu().pin_memory()) for k, v in st.items()}


@pytest.mark.parametrize("precision,with_src,chunk,use_sur", [
    (rhd.FP64, False, 1000, False), (rhd.MIXED, True, 777, False), (rhd.MIXED, False, 0, True),
    (rhd.FP64, True, 4096, True)])
def test_host_entry_equals_device_entry(precision, with_src, chunk, use_sur):
    n = 2 * 1000 + 537
    w = synth.preset("mixed_128cube_ng16", n_cells=n, seed=61, n_groups=40, device="cuda")
    if with_src:
        w.state["src"] = 0.2 * w.state["erad"].flip(0).contiguous()
    sur = rhd.Surrogate(w.n_groups, 5) if use_sur else None
    kw = dict(dt=w.dt, c_v=w.c_v, consts=w.consts, precision=precision)
    dev = synth.clone_state(w.state)
    s_dev = torch.empty(n, dtype=torch.uint8, device="cuda")
    i_dev = torch.empty(n, dtype=torch.uint8, device="cuda")
    if use_sur:
        sur.source_update(dev, w.edges, w.law, status=s_dev, iters=i_dev, **kw)
    else:
        rhd.source_update(dev, w.edges, w.law, status=s_dev, iters=i_dev, **kw)
    torch.cuda.synchronize()
    host = _pinned(w.state)
    s_h = torch.empty(n, dtype=torch.uint8).pin_memory()
    i_h = torch.empty(n, dtype=torch.uint8).pin_memory()
    rhd.source_update_host(host, w.edges, w.law, status=s_h, iters=i_h, surrogate=sur,
                           chunk_cells=chunk, **kw)
    for k in ("mom", "egas", "erad", "frad"):
        assert torch.equal(host[k], dev[k].cpu()), k
    for k in ("rho", "kappa0"):
        assert torch.equal(host[k], w.state[k].cpu()), k  # inputs untouched
    assert torch.equal(s_h, s_dev.cpu()) and torch.equal(i_h, i_dev.cpu())
    assert int((s_h <= rhd.STATUS_FALLBACK).sum()) == n


def test_host_entry_group_stride_and_errors():
    """A host grid with group stride > n_cells (the first n cells of a larger
    array) and the argument checks of the device entry."""
    w = synth.preset("tiny", n_cells=900, seed=3, device="cuda")
    n = 700
    kw = dict(dt=w.dt, c_v=w.c_v, consts=w.consts, precision=rhd.FP64)
    dev = synth.clone_state(w.state)
    sub = {k: (v[..., :n].contiguous() if v is not None and v.shape[-1] == 900 else v)
           for k, v in dev.items()}
    rhd.source_update(sub, w.edges, w.law, **kw)
    host = _pinned(w.state)
    st = rhd._state(host, w.n_groups, n, 900, c_v=w.c_v, consts=w.consts, theta=1.0,
                    precision=rhd.FP64, closure=rhd.M1, tol=0.0, tol_outer=0.0, max_newton=0,
                    max_outer=0, status=None, iters=None, flags=0, device="cpu")
    e = np.ascontiguousarray(w.edges, dtype=np.float64)
    gr = rhd.Groups(len(e) - 1, rhd._dp(e))
    lw, keep = rhd.make_law(w.law)
    assert rhd.lib().rhd_source_update_host(st, gr, lw, w.dt, n, None, 256) == 0
    torch.cuda.synchronize()
    assert torch.equal(host["erad"][:, :n], sub["erad"].cpu())
    assert torch.equal(host["erad"][:, n:], w.state["erad"][:, n:].cpu())  # beyond n_cells untouched
    assert rhd.lib().rhd_source_update_host(st, gr, lw, w.dt, n, None, -1) == -1
    bad = np.ascontiguousarray(w.edges[::-1], dtype=np.float64)
    gb = rhd.Groups(len(bad) - 1, rhd._dp(bad))
    assert rhd.lib().rhd_source_update_host(st, gb, lw, w.dt, n, None, 0) == -2
