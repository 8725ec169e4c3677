"""Full-size parity: every edge of the benchmark workloads against the CPU
oracle, chunk by chunk.

The GPU writes the whole output in the launch configuration that bench.py
times; each chunk is copied back and compared edge for edge with the oracle
computing the same edge range on all host cores (edges are independent, so
the oracle's range split changes nothing).  A mismatch names its chunk.

  - k = 26, m = 2^30, variable table bound 2^12 (the contract workload);
  - one whole 2^30-edge chunk (the last, edges 31 * 2^30 ..) of the k = 34,
    per-level noisy, undirected, u64 workload, with the tuner's group length
    and launch shape;
  - a wave of the batched workload (the first 128 of its 4096 graphs) in one
    persistent launch, tables as the autotuner picks them.
"""
import numpy as np
import pytest

import oracle
import paper_1905_03525_gb300 as rm
from paper_1905_03525_gb300 import autotune
from paper_1905_03525_gb300.workloads import G500, batched_graphs, noisy_levels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHUNK = 1 << 24


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1905_03525_gb300 import build
    build.build()
    yield
    torch.cuda.synchronize()
    rm.rmat_check_device_errors()
    torch.cuda.empty_cache()


def _host_pairs(dev, k, host):
    """Copy a (n, 2) device slice into the pinned staging tensor; (row, col) views."""
    n = dev.shape[0]
    h = host[:n]
    h.copy_(dev)
    a = h.numpy().view(np.uint32 if k <= 32 else np.uint64)
    return a[:, 0], a[:, 1]


def _staging(dtype):
    return torch.empty((CHUNK, 2), dtype=dtype, pin_memory=True)


def _compare_chunks(out, k, tables, seed, e0, host, undirected=False, chunk=CHUNK):
    """(chunk index, first differing edge) of every chunk whose edges differ
    from the oracle's."""
    m = out.shape[0]
    bad = []
    for i, lo in enumerate(range(0, m, chunk)):
        n = min(chunk, m - lo)
        r_g, c_g = _host_pairs(out[lo:lo + n], k, host)
        r_o, c_o = oracle.generate_parallel(tables, k, seed, e0 + lo, n, undirected=undirected)
        if not (np.array_equal(r_g, r_o) and np.array_equal(c_g, c_o)):
            first = int(np.nonzero((r_g != r_o) | (c_g != c_o))[0][0])
            bad.append((i, e0 + lo + first))
    return bad


def test_k26_every_edge_of_2p30():
    """The contract workload: k = 26, m = 2^30 (edge factor 16), Graph 500
    parameters, variable table bound 2^12, seed 1, default launch shape."""
    k, m, seed = 26, 1 << 30, 1
    t = rm.rmat_build_table(*G500, k, 4096)
    out = rm.empty_edges(m, k)
    rm.rmat_generate(t, seed, 0, m, out)
    torch.cuda.synchronize()
    bad = _compare_chunks(out, k, [oracle.Table.variable(*G500, k, 4096)], seed, 0, _staging(out.dtype))
    assert not bad, f"(chunk, first differing edge) against the oracle: {bad[:8]}"
    del out


def test_k34_per_level_last_chunk_every_edge():
    """Edges 31 * 2^30 .. 32 * 2^30 - 1 of the k = 34 workload (u64 pairs,
    undirected, per-level noise +-0.05), group length and launch shape from
    the tuner as the benchmark picks them."""
    k, m, seed = 34, 1 << 30, 34
    P = noisy_levels(k)
    ell = autotune.tune_levels(k, P, rm.RMAT_UNDIRECTED)["ell"]
    t = rm.rmat_build_table_levels(P, k, ell, rm.RMAT_UNDIRECTED)
    autotune.tune_launch(t, sample_edges=1 << 26)
    e0 = 31 << 30
    out = rm.empty_edges(m, k)
    rm.rmat_generate(t, seed, e0, m, out)
    torch.cuda.synchronize()
    bad = _compare_chunks(out, k, oracle.level_groups(P, k, ell), seed, e0, _staging(out.dtype), undirected=True)
    assert not bad, f"l = {ell}: (chunk, first differing edge) against the oracle: {bad[:8]}"
    del out


def test_batched_wave_every_edge():
    """The first 128 graphs of the 4096-graph batched workload (k ~ U{10..24},
    m = round(2^U(12, 26)), Dirichlet parameters), tables of the autotuner's
    kinds and sizes, all in one persistent launch."""
    graphs = batched_graphs(4096)[:128]
    tables, _ = autotune.plan_batch(graphs)
    total = sum(g["m"] for g in graphs)
    arena = torch.empty((total + 64 * len(graphs), 2), dtype=torch.int32, device="cuda")
    b = rm.rmat_batch_create()
    outs, off = [], 0
    for g, t in zip(graphs, tables):
        o = arena[off:off + g["m"]]
        outs.append(o)
        off += (g["m"] + 63) // 64 * 64
        rm.rmat_batch_add(b, t, g["seed"], 0, g["m"], o)
    rm.rmat_batch_launch(b)
    torch.cuda.synchronize()
    bad = []
    host = _staging(arena.dtype)
    for i, (g, t, o) in enumerate(zip(graphs, tables, outs)):
        kind, x = t.spec
        ot = oracle.Table.variable(*g["abcd"], g["k"], x) if kind == "variable" else oracle.Table.fixed([g["abcd"]], x)
        for c, e in _compare_chunks(o, g["k"], [ot], g["seed"], 0, host):
            bad.append((i, t.spec, c, e))
    assert not bad, f"(graph, table, chunk, first differing edge): {bad[:8]}"
    b.free()
    del arena
