"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2): one
process per rank, each pushing its own electrons (weak scaling, no data-path
collective); only the barrier and the max over ranks of the timed region
cross ranks, and only rank 0 reports."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import sys
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import torch.distributed as dist
    got_ws, got_rank, _ = bench.dist_setup()
    assert dist.get_backend() == "gloo"
    bench.barrier(got_ws)
    ms = 10.0 + 5.0 * rank                      # the slower rank sets the job time
    ms_max = bench.max_over_ranks(got_ws, ms)
    wl = bench.rank_workload(rank, 1000, 3)
    x0 = wl.particles().x
    out[rank] = (got_ws, got_rank, ms_max, float(x0[:8].sum()),
                 bench.aggregate_value(1000, 7, got_ws, ms_max))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_only_timing():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2 and {res[0][1], res[1][1]} == {0, 1}
    assert res[0][2] == res[1][2] == 15.0                # max over ranks
    assert res[0][3] != res[1][3]                        # each rank its own electrons
    assert abs(res[0][4] - 1000 * 7 * 2 / 0.015) < 1e-6  # whole-job units / slowest time


def test_reference_arm_reports_on_rank_zero_only():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    class A:
        cpu_sample, start_step, warmup, steps, gpus = 64, 5, 1, 2, 2
    assert bench.run_reference(A(), 2, 1) is None
    line = bench.run_reference(A(), 2, 0)
    assert line["impl"] == "reference" and line["steps"] == 2 and line["value"] > 0
