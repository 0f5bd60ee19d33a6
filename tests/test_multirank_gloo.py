"""Multi-rank host logic of the benchmark on CPU: two gloo ranks, each with its own batch.

Fields are independent, so ranks share no data; the only collective is the maximum of the step
times.  Checked here: every rank's batch has rank 0's shape (samples x sources), the ranks' orientation
draws differ, and the reported step time is the slowest rank's.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2302_10988_gb300 import workloads as W
        wl = bench.rank_workload(W, 6, rank)
        sizes = torch.tensor([s.nx for s in wl.samples], dtype=torch.int64)
        theta = torch.tensor(np.concatenate([s.region_theta for s in wl.samples]))
        all_sizes = [torch.zeros_like(sizes) for _ in range(world)]
        all_theta = [torch.zeros_like(theta) for _ in range(world)]
        dist.all_gather(all_sizes, sizes)
        dist.all_gather(all_theta, theta)
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)
        if rank == 0:
            out.put({"sizes": [s.tolist() for s in all_sizes], "theta": [t.numpy() for t in all_theta],
                     "ms": ms, "nodes": wl.nodes()})
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res["ms"] == 15.0                                     # slowest rank
    assert len(res["sizes"][0]) == len(res["sizes"][1]) == 6      # same batch shape on every rank
    assert not np.allclose(res["theta"][0], res["theta"][1])      # its own orientation draws
