"""The N > 1 path on CPU: world_size-2 gloo ranks shard one graph by edge
range (as bench.py does under torchrun), generate their ranges independently
(here with the CPU oracle), and the gathered result equals the one-rank graph;
the timing reduction takes the maximum over ranks.  No GPU involved."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1905_03525_gb300.sharding import strong_range, weak_range


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, mode, m, q):
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = oracle.Table.variable(0.57, 0.19, 0.19, 0.05, 26, 4096)
    off, cnt = weak_range(rank, m) if mode == "weak" else strong_range(rank, world, m)
    r, c = oracle.generate([t], 26, 1, off, cnt)
    parts = [None] * world
    dist.all_gather_object(parts, (off, r, c))
    elapsed = torch.tensor([0.1 * (rank + 1)], dtype=torch.float64)   # stand-in per-rank time
    dist.all_reduce(elapsed, op=dist.ReduceOp.MAX)
    if rank == 0:
        parts.sort(key=lambda p: p[0])
        q.put((np.concatenate([p[1] for p in parts]), np.concatenate([p[2] for p in parts]), float(elapsed.item())))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode,m", [("weak", 5000), ("strong", 10_001)])
def test_two_gloo_ranks_shard_one_graph(mode, m):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = 2
    procs = [ctx.Process(target=_rank_main, args=(r, world, _free_port_once(mode), mode, m, q))
             for r in range(world)]
    for p in procs:
        p.start()
    rows, cols, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total = m * world if mode == "weak" else m
    r1, c1 = oracle.generate([oracle.Table.variable(0.57, 0.19, 0.19, 0.05, 26, 4096)], 26, 1, 0, total)
    assert np.array_equal(rows, r1) and np.array_equal(cols, c1)
    assert tmax == pytest.approx(0.2)


_PORTS = {}


def _free_port_once(key):
    if key not in _PORTS:
        _PORTS[key] = _free_port()
    return _PORTS[key]


def test_strong_ranges_cover_exactly():
    for world in (1, 2, 3, 8):
        for m in (0, 1, 7, 1000, 2 ** 35 + 3):
            spans = [strong_range(r, world, m) for r in range(world)]
            assert sum(c for _, c in spans) == m
            assert all(spans[i][0] + spans[i][1] == spans[i + 1][0] for i in range(world - 1))
