"""Multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1) agree on the job time as
the maximum over ranks, solve different seeded right-hand sides, and the whole-job rate counts
every rank's dofs."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank  # rank 1 is the slower one
        total = bench.max_over_ranks(torch, mine, torch.device("cpu"), world)
        out[rank] = (total, bench.rank_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_seeds():
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
    assert all(p.exitcode == 0 for p in procs)
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] != out[1][1]


def test_job_rate_counts_every_rank():
    # 2 ranks x 1,046,529 dofs x 8 steps in 100 ms
    assert bench.job_rate(2, 1046529, 8, 100.0) == pytest.approx(2 * 1046529 * 8 / 0.1 / 1e6)
    assert bench.max_over_ranks(torch, 3.5, torch.device("cpu"), 1) == 3.5
