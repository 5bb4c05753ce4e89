"""The bench's N>1 path on CPU: two gloo ranks, each an independent replica, agree on the
job time as the maximum over ranks (the only cross-rank step; there is no data-path
collective)."""
from __future__ import annotations

import importlib.util
import os
import socket

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    dist.barrier()
    ms = bench.max_over_ranks(10.0 + 3.5 * rank, world, torch.device("cpu"))
    q.put((rank, ms))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got == {0: 13.5, 1: 13.5}
    assert all(p.exitcode == 0 for p in ps)
