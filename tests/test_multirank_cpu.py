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


def _partition_rank(rank, world, port, q):
    import oracle
    import paper_1905_03525_gb300 as rm
    from paper_1905_03525_gb300.sharding import row_tiles
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    k, t, m, seed = 14, 3, 40_000, 21
    r0, r1 = row_tiles(rank, world, t)
    # tiles from the library's host code (no device needed), edges from the oracle
    table = rm.rmat_build_table(0.57, 0.19, 0.19, 0.05, k, 1024)
    tiles = rm.rmat_partition_tiles(rm.rmat_partition_create(table, t, m, seed, r0, r1))
    ot = oracle.Table.variable(0.57, 0.19, 0.19, 0.05, k, 1024)
    _, (r, c) = oracle.generate_partitioned(ot, (0.57, 0.19, 0.19, 0.05), k, t, m, seed, r0, r1)
    ok = bool(((r >> np.uint64(k - t)) >= r0).all() and ((r >> np.uint64(k - t)) < r1).all())
    parts = [None] * world
    dist.all_gather_object(parts, (rank, tiles, r, c, ok))
    if rank == 0:
        q.put(parts)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_rows_without_exchange():
    """Partitioned graph (Sec. 3) over two ranks by tile rows: each rank's
    tiles (library host code) and edges (oracle) hold only its rows, and
    together they are exactly the one-rank partitioned graph."""
    import oracle
    from paper_1905_03525_gb300 import build
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts.sort(key=lambda x: x[0])
    assert all(p[4] for p in parts)
    ot = oracle.Table.variable(0.57, 0.19, 0.19, 0.05, 14, 1024)
    full, (r, c) = oracle.generate_partitioned(ot, (0.57, 0.19, 0.19, 0.05), 14, 3, 40_000, 21)
    got = {}
    for _, tiles, _, _, _ in parts:
        for R, C, n, f in zip(tiles["row"], tiles["col"], tiles["count"], tiles["first"]):
            got[int(f)] = (int(R), int(C), int(n))
    want = {int(f): (int(R), int(C), int(n)) for R, C, n, f in zip(full["row"], full["col"], full["count"], full["first"])}
    assert got == want
    # edges: every global edge once, identified by its number within the graph
    by_first = {}
    for _, tiles, rr, cc, _ in parts:
        pos = 0
        for n, f in zip(tiles["count"], tiles["first"]):
            by_first[int(f)] = (rr[pos:pos + int(n)], cc[pos:pos + int(n)])
            pos += int(n)
    rows = np.concatenate([by_first[f][0] for f in sorted(by_first)])
    cols = np.concatenate([by_first[f][1] for f in sorted(by_first)])
    assert np.array_equal(rows, r) and np.array_equal(cols, c)
