"""rhd_source_update_noalloc: the mixed form for callers that cannot let a
library allocate device memory (a host whose memory pool owns all of HBM, a
latency-bound loop where a first-call cudaMalloc would synchronize the device,
a run that must not fail for lack of memory midway).  It keeps the FP32
iterate and the correction step in the library's fixed 64 MiB device array
instead of a cudaMalloc'd workspace, and must give the same result as rhd_source_update with
precision = RHD_MIXED, call after call (the array keeps the previous call's
contents).  This file is collected last, so a failure here comes after every
other test has run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2407_18304_gb300 import rhd, synth

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the parity tests' per-output relative bound


def _state(w):
    return {k: (None if v is None else v.to("cuda").clone()) for k, v in w.state.items()}


def _run(fn, w, **kw):
    st = _state(w)
    n = st["rho"].shape[0]
    status = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    fn(st, w.edges, w.law, dt=w.dt, c_v=w.c_v, consts=w.consts, status=status, **kw)
    torch.cuda.synchronize()
    out = synth.to_numpy(st)
    out["status"] = status.cpu().numpy()
    return out


def _close(a, b):
    for k in ("egas", "erad", "frad", "mom"):
        np.testing.assert_allclose(a[k], b[k], rtol=TOL, atol=0, err_msg=k)
    np.testing.assert_array_equal(a["status"], b["status"])


def _bytes(n, G):
    """The array a call of n cells at G groups needs (the documented limit)."""
    return n * (32 * G + 34) + 1024


def _largest(G):
    return (rhd.NOALLOC_BYTES - 1024) // (32 * G + 34)


@pytest.mark.parametrize("preset,n", [("mixed_128cube_ng16", 3001), ("full_256cube_ng64", 30000)])
def test_noalloc_matches_the_allocating_entry_point_twice(preset, n):
    w = synth.preset(preset, n_cells=n, seed=2024)
    assert _bytes(n, w.n_groups) <= rhd.NOALLOC_BYTES
    ref = _run(rhd.source_update, w, precision=rhd.MIXED)
    assert (ref["status"] == 0).mean() > 0.99
    for _ in range(2):  # the second call finds the first call's contents in the array
        out = _run(rhd.source_update_noalloc, w)
        _close(out, ref)


def test_noalloc_takes_exactly_the_largest_call_that_fits():
    """At 64 groups: the largest cell count the array holds runs and matches
    the allocating entry; one cell more is refused."""
    n = _largest(64)
    assert n == 32232 and _bytes(n, 64) <= rhd.NOALLOC_BYTES < _bytes(n + 1, 64)
    w = synth.preset("full_256cube_ng64", n_cells=n, seed=77)
    _close(_run(rhd.source_update_noalloc, w), _run(rhd.source_update, w, precision=rhd.MIXED))
    w1 = synth.preset("full_256cube_ng64", n_cells=n + 1, seed=77)
    with pytest.raises(rhd.RhdError) as ei:
        _run(rhd.source_update_noalloc, w1)
    assert ei.value.code == -6


def test_noalloc_rejects_calls_beyond_its_array():
    w = synth.preset("full_256cube_ng64", n_cells=70000, seed=1)
    assert _bytes(70000, 64) > rhd.NOALLOC_BYTES
    st = _state(w)
    before = st["erad"].clone()
    with pytest.raises(rhd.RhdError) as ei:
        rhd.source_update_noalloc(st, w.edges, w.law, dt=w.dt, c_v=w.c_v, consts=w.consts)
    assert ei.value.code == -6
    torch.cuda.synchronize()
    assert torch.equal(st["erad"], before)  # nothing was launched
