"""bench.py's JSON line for the reference arm (the FP64 oracle on the host
cores), run on the CPU: one bounded step, every key the contract names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT, check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in line, k
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["unit"] == "cell-group updates/s" and line["steps"] == 1
    assert line["config"]["workload"] == "full_256cube_ng64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    """Launched as the multi-GPU bench is (torchrun, two ranks, 127.0.0.1),
    rank 0 alone runs the oracle and prints; the other rank exits 0."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                          "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port",
                          str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def test_roofline_numerator_takes_each_kernel_s_events_from_the_counting_model():
    """bench.algorithmic_ops: a kernel's algorithmic slots are its events x N_g x the
    counting model's operations per cell-group for them (tests/golden/opcounts.json);
    the first correction step's float-float operations enter as their FP32 operations."""
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "tests", "golden", "opcounts.json")) as f:
        full = json.load(f)
    t = full["events"]["full_256cube_ng64"]
    w = {"fp64_op_slots": {"div": 9.0, "sqrt": 9.0, "exp": 22.0},
         "fp32_op_slots": {"div": 15.0, "sqrt": 11.0, "exp": 30.0}}
    G, n = 64, 1000
    one = {e: n for e in ("eval32", "outer32", "residdf", "stepdf", "resid64", "step32",
                          "finish64")}
    ops = bench.algorithmic_ops("full_256cube_ng64", one, G, w)
    s64 = lambda c: bench.op_slots(c, w["fp64_op_slots"])
    s32 = lambda c: bench.op_slots(c, w["fp32_op_slots"])
    assert abs(ops["fp32_passes"]["f32"] - n * G * (s32(t["eval32"]["f32"]) + s32(t["outer32"]["f32"]))) < 1e-6
    assert abs(ops["correction"]["f64"] - n * G * sum(s64(t[e]["f64"]) for e in ("resid64", "step32", "finish64"))) < 1e-6
    df = {}
    for kind, cnt in t["residdf"]["df"].items():
        for k, v in full["df_fp32_ops"][kind].items():
            df[k] = df.get(k, 0.0) + cnt * v
    want = n * G * (s32(df) + s32(t["stepdf"]["f32"]))
    assert abs(ops["refine"]["f32"] - want) < 1e-6 * want
    # a float-float residual costs several times the FP64 residual's operation count
    assert ops["refine"]["f32"] > 3 * n * G * s64(t["resid64"]["f64"])
