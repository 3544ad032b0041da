"""The operation-counting model of the update (oracle/opcount.py), on the CPU.

The model is a working solver on a counting number type: its counts are
those of an algorithm that demonstrably reaches the root.  Pins:
* its paper inner/outer iteration (Sec. 3) reaches the oracle's root;
* its coupled Newton correction (the mixed form's step) takes an iterate
  1e-6 off the root to the oracle's root in one step, where the paper's tests
  hold on the FP64 residual;
* an inner evaluation costs exactly a G + b operations (eq. matrix's O(N_g)
  elimination: no operation grows faster than the group count);
* the charged cost of the special functions is the stated method's;
* tests/golden/opcounts.json is what the generator writes.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle import opcount as OC
from paper_2407_18304_gb300 import synth
from parity import oracle_groups, run_oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _params(w):
    return O.Params(c=w.consts["c"], c_hat=w.consts["c_hat"], a_rad=w.consts["a_rad"],
                    h=w.consts["h"], k_B=w.consts["k_B"], c_v=w.c_v, dt=w.dt)


@pytest.mark.parametrize("preset", ["tiny", "mixed_128cube_ng16"])
def test_the_paper_iteration_of_the_model_reaches_the_oracle_root(preset):
    w = synth.preset(preset, n_cells=6, seed=3)
    o = run_oracle(w)
    st = synth.to_numpy(w.state)
    for i in range(6):
        cell = OC.make_cell(st, i, _params(w), oracle_groups(w))
        ok, ev = OC.solve_paper(cell, tol=1e-13, tol_outer=1e-14)
        assert ok and len(ev["eval64"]) >= 2
        r = OC.result(cell)
        et = st["egas"][i] + st["erad"][:, i].sum()
        assert np.abs(r["erad"] - o["erad"][:, i]).max() < 1e-10 * et
        assert abs(r["egas"] - o["egas"][i]) < 1e-10 * et
        assert np.abs(r["frad"] - o["frad"][:, :, i]).max() < 1e-10 * w.consts["c"] * et


@pytest.mark.parametrize("preset", ["mixed_128cube_ng16", "full_256cube_ng64"])
def test_one_coupled_newton_step_reaches_the_root_from_fp32_accuracy(preset):
    w = synth.preset(preset, n_cells=3, seed=3)
    o = run_oracle(w)
    st = synth.to_numpy(w.state)
    rng = np.random.default_rng(0)
    for i in range(3):
        cell = OC.make_cell(st, i, _params(w), oracle_groups(w))
        OC.setup(cell)
        et = st["egas"][i] + st["erad"][:, i].sum()
        ms = o["mom"][:, i]
        Eg = o["erad"][:, i]
        cell.Eint = OC.Num((o["egas"][i] - 0.5 * ms @ ms / cell.rho) * (1 + 1e-6 * rng.standard_normal()))
        cell.R = [OC.Num(Eg[g] - cell.E0[g] + 1e-6 * Eg[g] * rng.standard_normal())
                  for g in range(cell.G)]
        cell.F = [[OC.Num(o["frad"][d, g, i] + 1e-6 * w.consts["c"] * Eg[g] * rng.standard_normal())
                   for d in range(3)] for g in range(cell.G)]
        ok0, res = OC.coupled_residual(cell, 1e-11, 1e-13)
        assert not ok0
        OC.coupled_step(cell, res)
        ok1, res = OC.coupled_residual(cell, 1e-11, 1e-13)
        assert ok1
        OC.finish(cell, res)
        r = OC.result(cell)
        assert np.abs(r["erad"] - Eg).max() < 1e-11 * et
        assert abs(r["egas"] - o["egas"][i]) < 1e-11 * et
        assert np.abs(r["frad"] - o["frad"][:, :, i]).max() < 1e-11 * w.consts["c"] * et


def test_an_inner_evaluation_costs_exactly_linear_in_the_group_count():
    counts = {}
    for G in (4, 8, 16):
        w = synth.preset("mixed_128cube_ng16", n_cells=1, seed=5, n_groups=G)
        st = synth.to_numpy(w.state)
        counts[G] = OC.per_event_counts(st, 0, _params(w), oracle_groups(w))["eval64"]
    for k in OC.KINDS:
        d1, d2 = counts[8][k] - counts[4][k], counts[16][k] - counts[8][k]
        assert d2 == 2 * d1, (k, counts[4][k], counts[8][k], counts[16][k])
    # and it is O(N_g) with a per-group cost of a few tens of operations
    per_group = sum(counts[16][k] - counts[8][k] for k in OC.KINDS) / 8
    assert 40 < per_group < 120


def test_the_charged_cost_of_the_edge_terms():
    """One edge: expm1, one reciprocal, a degree-13 Horner polynomial on the
    argument's segment and the prefactors -- counted from the method."""
    t0 = OC.TALLY.snapshot()
    OC.edge_terms(3.0, OC.Num(1.0))
    d = OC.Tally.diff(t0, OC.TALLY.snapshot())["f64"]
    assert d["exp"] == 1 and d["div"] == 1 and d["fma"] == OC.PLANCK_DEGREE and d["sqrt"] == 0
    assert d["add"] == 4 and d["mul"] == 14 and d["cmp"] == 1
    t0 = OC.TALLY.snapshot()
    OC.fma(OC.Num(1.0), 2.0, 3.0)
    assert OC.Tally.diff(t0, OC.TALLY.snapshot())["f64"]["fma"] == 1


def test_the_committed_table_is_what_the_generator_writes():
    path = os.path.join(HERE, "golden", "opcounts.json")
    with open(path) as f:
        committed = f.read()
    assert committed == json.dumps(OC.table(), indent=1, sort_keys=True) + "\n"


def test_the_float_float_step_counts_the_fp64_residual_operations():
    """residdf is the coupled residual of resid64 with its FP64 operations in
    float-float (tallied under "df") and without the tests; stepdf is step32."""
    w = synth.preset("full_256cube_ng64", n_cells=1, seed=5, n_groups=8)
    ev = OC._event_counts(synth.to_numpy(w.state), 0, _params(w), oracle_groups(w))
    assert ev["residdf"]["df"] == ev["resid64"]["f64"]
    assert all(v == 0 for v in ev["residdf"]["f64"].values())
    assert all(v == 0 for v in ev["residdf"]["f32"].values())
    assert sum(ev["resid64"]["f32"].values()) > 0  # the tests, which residdf leaves out
    assert ev["stepdf"] == ev["step32"]
    # a float-float operation costs several FP32 operations, never none
    for k in OC.KINDS:
        assert sum(OC.DF_FP32_OPS[k].values()) >= 2
