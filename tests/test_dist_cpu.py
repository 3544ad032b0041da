"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): the
max-over-ranks time, the whole-job unit sum and the per-rank seeds of the
weak-scaling workload.  (The solve itself needs a GPU; the ranks share no
data on the hot path.)"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from paper_2407_18304_gb300 import synth
    t = 1.5 + rank          # this rank's timed seconds
    units = 100.0 * (rank + 1)
    bench.barrier(ws)
    tmax = bench.allmax(t, ws)
    total = bench.allsum(units, ws)
    seed = synth.PRESET_SEED["tiny"] + 1000 * rank  # bench.run_ours's per-rank seed
    w = synth.preset("tiny", n_cells=16, seed=seed)
    out[rank] = (tmax, total, float(w.state["rho"][0]))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_reduce_like_the_bench():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, _free_port(), out), nprocs=ws, start_method="spawn")
    assert out[0][0] == out[1][0] == 2.5            # max over ranks
    assert out[0][1] == out[1][1] == 300.0          # whole-job units
    assert out[0][2] != out[1][2]                   # every rank draws its own grid
