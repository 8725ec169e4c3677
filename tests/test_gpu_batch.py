"""GPU parity of the batched persistent launch: every graph of a batch is
byte-identical to the same graph generated alone, and to the oracle."""
import numpy as np
import pytest

import oracle
import paper_1905_03525_gb300 as rm
from paper_1905_03525_gb300.workloads import G500, SKEWED, batched_graphs, noisy_levels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1905_03525_gb300 import build
    build.build()
    yield
    torch.cuda.synchronize()
    rm.rmat_check_device_errors()


def _mixed_jobs():
    """Graphs covering every kernel path: compact/wide entries, shared/global
    tables, u32/u64 output, per-level tables, ragged and tiny sizes."""
    jobs = []
    for i, g in enumerate(batched_graphs(40, seed=77, k_range=(10, 24), log2m_range=(5.0, 15.0))):
        jobs.append((rm.rmat_build_table(*g["abcd"], g["k"], 1 << (8 + i % 6)), g["k"], g["seed"], 0, g["m"]))
    jobs.append((rm.rmat_build_table(*SKEWED, 30, 1 << 14), 30, 5, 3, 20_001))     # wide entries
    jobs.append((rm.rmat_build_table(*G500, 26, 1 << 16), 26, 6, 0, 30_000))       # global table
    jobs.append((rm.rmat_build_table_fixed(*G500, 16, 4), 16, 1, 0, 1 << 16))
    jobs.append((rm.rmat_build_table(*G500, 40, 4096), 40, 7, 1 << 33, 10_000))    # u64
    jobs.append((rm.rmat_build_table_levels(noisy_levels(34), 34, 6, rm.RMAT_UNDIRECTED), 34, 34, 31 << 30, 25_000))
    jobs.append((rm.rmat_build_table(*G500, 26, 4096), 26, 1, 0, 1))
    jobs.append((rm.rmat_build_table(*G500, 26, 4096), 26, 1, 0, 0))               # empty
    return jobs


@pytest.mark.parametrize("shape", [None, (512, 2, 128), (256, 4, 64)])
def test_batch_equals_single_launches(shape):
    jobs = _mixed_jobs()
    b = rm.rmat_batch_create()
    outs = []
    for t, k, seed, e0, m in jobs:
        out = rm.empty_edges(max(m, 1), k)
        out.fill_(-1)
        rm.rmat_batch_add(b, t, seed, e0, m, out)
        outs.append(out)
    if shape:
        rm.rmat_batch_prepare(b, *shape)
    rm.rmat_batch_launch(b)
    torch.cuda.synchronize()
    for (t, k, seed, e0, m), out in zip(jobs, outs):
        if m == 0:
            assert bool((out == -1).all())
            continue
        ref = rm.empty_edges(m, k)
        rm.rmat_generate(t, seed, e0, m, ref)
        torch.cuda.synchronize()
        assert torch.equal(out[:m], ref), (k, m)
    # relaunch (as a CUDA graph replay would) gives the same bytes
    first = [o.clone() for o in outs]
    rm.rmat_batch_launch(b)
    torch.cuda.synchronize()
    assert all(torch.equal(a, c) for a, c in zip(first, outs))


def test_batch_against_oracle():
    gs = batched_graphs(12, seed=5, k_range=(10, 24), log2m_range=(8.0, 14.0))
    b = rm.rmat_batch_create()
    outs, tabs = [], []
    for g in gs:
        t = rm.rmat_build_table(*g["abcd"], g["k"], 2048)
        out = rm.empty_edges(g["m"], g["k"])
        rm.rmat_batch_add(b, t, g["seed"], 0, g["m"], out)
        outs.append(out)
    rm.rmat_batch_launch(b)
    torch.cuda.synchronize()
    for g, out in zip(gs, outs):
        row, col = oracle.generate([oracle.Table.variable(*g["abcd"], g["k"], 2048)], g["k"], g["seed"], 0, g["m"])
        h = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(h[:, 0], row) and np.array_equal(h[:, 1], col)


def test_batch_in_cuda_graph():
    jobs = _mixed_jobs()[:10]
    b = rm.rmat_batch_create()
    outs = []
    for t, k, seed, e0, m in jobs:
        out = rm.empty_edges(m, k)
        rm.rmat_batch_add(b, t, seed, e0, m, out)
        outs.append(out)
    rm.rmat_batch_prepare(b)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rm.rmat_batch_launch(b, s)
    for o in outs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    for (t, k, seed, e0, m), out in zip(jobs, outs):
        ref = rm.empty_edges(m, k)
        rm.rmat_generate(t, seed, e0, m, ref)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_batch_scrambled_graphs_match_single_launches():
    jobs = _mixed_jobs()[:12] + _mixed_jobs()[-5:-2]
    b = rm.rmat_batch_create()
    outs = []
    for i, (t, k, seed, e0, m) in enumerate(jobs):
        rm.rmat_table_set_scramble(t, i % 2 == 0, 1000 + i)
        out = rm.empty_edges(m, k)
        rm.rmat_batch_add(b, t, seed, e0, m, out)
        outs.append(out)
    rm.rmat_batch_launch(b)
    torch.cuda.synchronize()
    for (t, k, seed, e0, m), out in zip(jobs, outs):
        ref = rm.empty_edges(m, k)
        rm.rmat_generate(t, seed, e0, m, ref)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
