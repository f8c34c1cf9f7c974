"""Multi-rank host logic of bench.py on CPU: two gloo ranks.

Each rank runs its own problem (seeds shifted by the rank), the job's time is
the slowest rank's (all_reduce MAX), and the whole-job value counts every
rank's elements; the reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1504_04653_gb300 import workloads as W

    ms = [3.0, 5.0][rank]
    ms_max = bench.max_over_ranks(ms, world, torch.device("cpu"))
    wl = bench.rank_workload(W.WORKLOADS["lmax64"], rank)
    colat = np.linspace(0.01, np.pi - 0.01, 257)
    ninv = wl.ninv(colat)
    class A:  # the reference arm's arguments
        workload, steps, warmup = "lmax64", 1, 0
    ref = bench.reference_arm(A, rank, world) if rank == 1 else "skipped"
    out[rank] = (ms_max, bench.job_value(1000, ms_max, world), wl.seeds[0], float(ninv.sum()), ref)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 5.0  # both ranks see the slowest rank's time
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1000 / 5e-3)
    assert res[1][2] == res[0][2] + 1  # rank r's problem: seeds shifted by r
    assert res[0][3] != res[1][3]  # ... so the N^-1 maps differ
    assert res[1][4] is None  # the reference arm does no work off rank 0


def test_single_rank_is_identity():
    import importlib
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    assert bench.max_over_ranks(4.5, 1, None) == 4.5
    assert bench.job_value(10, 2.0, 1) == pytest.approx(5000.0)
