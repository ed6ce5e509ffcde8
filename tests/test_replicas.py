"""The multi-GPU mode is replicas only: every rank runs its own independent
simulation and the single exchange is the benchmark's whole-job total (units
summed over ranks, timed region of the slowest rank). Checked here with two
gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = [1.5e9, 2.25e9][rank]
    ms = [80.0, 95.0][rank]
    total, slowest = bench.job_totals(units, ms, world)
    out[rank] = (total, slowest)
    dist.destroy_process_group()


def test_job_totals_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (3.75e9, 95.0)


def test_job_totals_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(7.0, 3.0, 1) == (7.0, 3.0)
