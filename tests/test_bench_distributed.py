"""The multi-process path of bench.py on CPU (gloo, world size 2): every rank
projects its own grids (weak scaling: different seeds per rank, no data-path
collective) and the reported time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + rank, torch.device("cpu"))
        u, v, fl = bench.make_inputs(rank)
        q.put((rank, t, float(u[0, 100, 100]), int(fl.sum())))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_the_grids_and_report_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][1] == out[1][1] == 11.0
    # the two ranks draw different grids
    assert out[0][2] != out[1][2] or out[0][3] != out[1][3]
