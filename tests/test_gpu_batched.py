"""The batched path (many uneven grids in one persistent launch, replayed as a
CUDA graph) against the FP64 oracle and against the one-grid entry point.

Each grid has its own cell count, group count (4..64), opacity law, dt, theta
and reduced speed of light; every cell must come out as the one-grid call
gives it (same per-cell algorithm), and so as the oracle gives it within the
parity bounds of the one-grid tests.
"""
import numpy as np
import pytest
import torch

from paper_2407_18304_gb300 import rhd, synth
from parity import MAX_UNCONVERGED, agreed, conservation, converged, errors, run_gpu, run_oracle, select

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
TIGHT = dict(tol=1e-14, tol_outer=1e-15)
FLOOR = 10 * TIGHT["tol"] / FP64_TOL
MIXED_BOUND = 1e-6
DEFAULT_FLOOR = 10 * 1e-11 / MIXED_BOUND


def _grids(n_grids=6, seed=31, max_side=8):
    ws = synth.batched_grids(n_grids=n_grids, seed=seed, side_lo=3, side_hi=12, max_side=max_side)
    rng = np.random.default_rng(seed)
    extra = []
    for w in ws:
        w.dt = synth.DT * float(np.exp(rng.uniform(np.log(0.3), np.log(3.0))))
        extra.append(dict(theta=float(rng.choice([1.0, 0.5])),
                          c_hat=float(w.consts["c"] * rng.choice([1.0, 0.3]))))
    return ws, extra


def _specs(ws, extra, precision, states, tight, flags=0):
    specs, outs = [], []
    for w, x, st in zip(ws, extra, states):
        n = st["rho"].shape[0]
        status = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
        iters = torch.zeros(n, dtype=torch.uint8, device="cuda")
        consts = dict(w.consts, c_hat=x["c_hat"])
        specs.append(rhd.GridSpec(st, w.edges, w.law, dt=w.dt, c_v=w.c_v, consts=consts,
                                  theta=x["theta"], precision=precision, status=status,
                                  iters=iters, flags=flags, **(TIGHT if tight else {})))
        outs.append((status, iters))
    return specs, outs


def _to_dev(ws):
    return [{k: (None if v is None else v.cuda().clone()) for k, v in w.state.items()} for w in ws]


def _collect(states, outs):
    res = []
    for st, (status, iters) in zip(states, outs):
        r = synth.to_numpy(st)
        r["status"] = status.cpu().numpy().astype(np.int32)
        r["iters"] = iters.cpu().numpy().astype(np.int32)
        res.append(r)
    return res


def run_batched(ws, extra, precision, tight=False, ctx=None, states=None, flags=0):
    ctx = ctx or rhd.Context()
    states = states if states is not None else _to_dev(ws)
    specs, outs = _specs(ws, extra, precision, states, tight, flags)
    ctx.update(specs)
    torch.cuda.synchronize()
    return _collect(states, outs)


def _check_parity(ws, extra, got, ref, tol, floor, label):
    for w, x, g, o in zip(ws, extra, got, ref):
        st0 = synth.to_numpy(w.state)
        ok = agreed(f"{label} {w.name}", g, oracle=o)
        gs, os_, s0 = select(g, ok), select(o, ok), select(st0, ok)
        e = errors(gs, os_, s0, w.consts["c"], w.c_v, floor=floor)
        print(label, w.name, len(w.edges) - 1, s0["rho"].shape[0],
              " ".join(f"{k}={v:.2e}" for k, v in e.items()))
        ce, cm = conservation(gs, s0, w.consts["c"], x["c_hat"])
        assert ce < 64 * 2.0 ** -52 and cm < 64 * 2.0 ** -52
        for k in ("T", "egas", "erad"):
            assert e[k] < tol, (label, w.name, k, e[k])
        if tol == FP64_TOL:
            for k, v in e.items():
                if not k.endswith("_plain"):
                    assert v < tol, (label, w.name, k, v)


def test_batched_fp64_matches_oracle_and_single_grid():
    # the flux test makes every group flux converge (the paper's outer test
    # sees F_g only through v.F), so the fluxes too can be held to 1e-10
    ws, extra = _grids()
    got = run_batched(ws, extra, rhd.FP64, tight=True, flags=rhd.FLUX_TEST)
    orc = [run_oracle(w, theta=x["theta"], c_hat=x["c_hat"]) for w, x in zip(ws, extra)]
    _check_parity(ws, extra, got, orc, FP64_TOL, FLOOR, "batched-fp64 vs oracle")
    one = [run_gpu(w, theta=x["theta"], c_hat=x["c_hat"], flags=rhd.FLUX_TEST, **TIGHT)
           for w, x in zip(ws, extra)]
    _check_parity(ws, extra, got, one, FP64_TOL, FLOOR, "batched-fp64 vs one-grid")
    same = np.mean([np.array_equal(g[k], o[k]) for g, o in zip(got, one)
                    for k in ("egas", "erad", "frad", "mom")])
    print("bit-identical arrays (batched vs one-grid):", same)


def test_batched_mixed_matches_oracle_and_single_grid():
    ws, extra = _grids(seed=32)
    got = run_batched(ws, extra, rhd.MIXED)
    orc = [run_oracle(w, theta=x["theta"], c_hat=x["c_hat"]) for w, x in zip(ws, extra)]
    _check_parity(ws, extra, got, orc, MIXED_BOUND, DEFAULT_FLOOR, "batched-mixed vs oracle")
    one = [run_gpu(w, precision=rhd.MIXED, theta=x["theta"], c_hat=x["c_hat"])
           for w, x in zip(ws, extra)]
    _check_parity(ws, extra, got, one, MIXED_BOUND, DEFAULT_FLOOR, "batched-mixed vs one-grid")
    same = np.mean([np.array_equal(g[k], o[k]) for g, o in zip(got, one)
                    for k in ("egas", "erad", "frad", "mom")])
    print("bit-identical arrays (batched vs one-grid):", same)
    # at the default mappings (the one-grid call's) the same device functions
    # take every cell through the same phases
    assert same == 1.0


def _bucket_grids(seed=36):
    """Two small grids in each bucket (4 and 16, 24 and 32, 40 and 64 groups),
    moving cells, breakpoints on the group edges, own law and cell count each."""
    rng = np.random.default_rng(seed)
    ws = [synth.preset("mixed_128cube_ng16", n_cells=int(rng.integers(60, 200)), seed=seed + G,
                       n_groups=G) for G in (4, 16, 24, 32, 40, 64)]
    extra = [dict(theta=1.0, c_hat=w.consts["c_hat"]) for w in ws]
    return ws, extra


def _configs(precision):
    """Mapping configurations that together take every mapping each bucket
    offers (the passes', and in the mixed form the correction step's)."""
    per_bucket = []
    for b in range(rhd.BATCH_BUCKETS):
        cs = rhd.CORRECTION_MAPPINGS[b] if precision == rhd.MIXED else rhd.CORRECTION_MAPPINGS[b][:1]
        per_bucket.append([(p, c) for p in rhd.PASS_MAPPINGS[b] for c in cs])
    n = max(len(x) for x in per_bucket)
    return [[x[k % len(x)] for x in per_bucket] for k in range(n)]


@pytest.mark.parametrize("precision", [rhd.MIXED, rhd.FP64], ids=["mixed", "fp64"])
def test_every_mapping_of_every_bucket_matches_the_oracle(precision):
    ws, extra = _bucket_grids()
    orc = [run_oracle(w) for w in ws]
    fp64 = precision == rhd.FP64
    for cfg in _configs(precision):
        ctx = rhd.Context()
        for b, (p, c) in enumerate(cfg):
            ctx.set_mapping(b, p, c)
        assert ctx.mappings == cfg
        got = run_batched(ws, extra, precision, tight=fp64, ctx=ctx,
                          flags=rhd.FLUX_TEST if fp64 else 0)
        _check_parity(ws, extra, got, orc, FP64_TOL if fp64 else MIXED_BOUND,
                      FLOOR if fp64 else DEFAULT_FLOOR, f"mapping {cfg}")


def test_set_mapping_rejects_what_a_bucket_does_not_offer():
    ctx = rhd.Context()
    default = [(0, 8), (0, 16), (0, 32)]  # passes 0: the one-grid call's, by precision
    assert ctx.mappings == default
    for b, p, c in [(0, 16, 8), (0, 1, 16), (1, 2, 8), (1, 1, 32), (2, 8, 32), (2, 1, 8),
                    (3, 1, 8), (-1, 1, 8)]:
        with pytest.raises(rhd.RhdError) as e:
            ctx.set_mapping(b, p, c)
        assert e.value.code == -1
    with pytest.raises(rhd.RhdError):
        ctx.mapping(3)
    assert ctx.mappings == default


def test_graph_replay_is_bit_exact_and_recaptures_on_a_new_batch():
    ws, extra = _grids(n_grids=5, seed=33, max_side=10)
    ctx = rhd.Context()
    first = run_batched(ws, extra, rhd.MIXED, ctx=ctx)
    again = run_batched(ws, extra, rhd.MIXED, ctx=ctx)  # replay of the captured graph
    for a, b in zip(first, again):
        for k in ("egas", "erad", "frad", "mom", "status", "iters"):
            np.testing.assert_array_equal(a[k], b[k])
    sub = run_batched(ws[:3], extra[:3], rhd.MIXED, ctx=ctx)  # new shape: captured again
    for a, b in zip(first[:3], sub):
        for k in ("egas", "erad", "frad", "mom", "status"):
            np.testing.assert_array_equal(a[k], b[k])


def test_autotune_leaves_the_state_unchanged_and_keeps_valid_choices():
    ws, extra = _grids(n_grids=4, seed=34, max_side=12)
    bws, bex = _bucket_grids(seed=37)
    ws, extra = ws + bws, extra + bex  # every bucket has grids
    ctx = rhd.Context()
    assert ctx.shape == (128, 512)
    states = _to_dev(ws)
    before = [synth.to_numpy(s) for s in states]
    specs, _ = _specs(ws, extra, rhd.MIXED, states, False)
    threads, cpi = ctx.autotune(specs)
    torch.cuda.synchronize()
    assert threads in (64, 128, 256) and cpi in (threads, 4 * threads, 16 * threads)
    picked = ctx.mappings
    print("autotuned mappings", picked, "shape", (threads, cpi))
    for b, (p, c) in enumerate(picked):
        assert p in rhd.PASS_MAPPINGS[b] and c in rhd.CORRECTION_MAPPINGS[b]
    for b, s in zip(before, states):
        a = synth.to_numpy(s)
        for k in ("egas", "erad", "frad", "mom"):
            np.testing.assert_array_equal(a[k], b[k])
    tuned = run_batched(ws, extra, rhd.MIXED, ctx=ctx)
    # the CTA shape moves cells between threads, never the arithmetic of a cell
    same = rhd.Context()
    for b, (p, c) in enumerate(picked):
        same.set_mapping(b, p, c)
    plain = run_batched(ws, extra, rhd.MIXED, ctx=same)
    for a, b in zip(tuned, plain):
        for k in ("egas", "erad", "frad", "mom", "status"):
            np.testing.assert_array_equal(a[k], b[k])
    orc = [run_oracle(w, theta=x["theta"], c_hat=x["c_hat"]) for w, x in zip(ws, extra)]
    _check_parity(ws, extra, tuned, orc, MIXED_BOUND, DEFAULT_FLOOR, "autotuned vs oracle")


def test_empty_grids_invalid_cells_and_errors():
    ws, extra = _grids(n_grids=3, seed=35)
    ws[0] = synth.Workload("empty", synth.take_cells(ws[0].state, slice(0, 0)), ws[0].edges,
                           ws[0].law)
    ws[1].state["rho"][3] = float("nan")
    got = run_batched(ws, extra, rhd.FP64)
    assert got[0]["rho"].shape == (0,)
    assert got[1]["status"][3] == rhd.STATUS_INVALID
    assert (got[1]["status"] != 255).all() and (got[2]["status"] != 255).all()
    ctx = rhd.Context()
    with pytest.raises(rhd.RhdError) as e:
        ctx.update([])
    assert e.value.code == -1
    states = _to_dev(ws)
    specs, _ = _specs(ws, extra, rhd.MIXED, states, False)
    specs[2].c.state.precision = rhd.FP64
    with pytest.raises(rhd.RhdError) as e:
        ctx.update(specs)
    assert e.value.code == -1
    w65 = synth.preset("tiny", n_cells=10, n_groups=65)
    sp = rhd.GridSpec({k: (None if v is None else v.cuda()) for k, v in w65.state.items()},
                      w65.edges, w65.law, dt=w65.dt, c_v=w65.c_v, consts=w65.consts)
    with pytest.raises(rhd.RhdError) as e:
        ctx.update([sp])
    assert e.value.code == -6
    for s, b in zip(states, [synth.to_numpy(s) for s in _to_dev(ws)]):
        np.testing.assert_array_equal(synth.to_numpy(s)["egas"], b["egas"])
