"""GPU parity: librmat's kernels against the CPU oracle, bit for bit.

Every case runs through the C ABI (the ctypes binding) on seeded synthetic
inputs and compares every edge; the full-size workloads are compared edge
for edge in test_gpu_fullsize.py.
"""
import numpy as np
import pytest

import oracle
import paper_1905_03525_gb300 as rm
from paper_1905_03525_gb300.workloads import G500, SKEWED, noisy_levels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ASYM = (0.5, 0.2, 0.25, 0.05)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1905_03525_gb300 import build
    build.build()
    yield
    torch.cuda.synchronize()
    rm.rmat_check_device_errors()


def as_u64_pairs(t, k):
    """(count, 2) device tensor -> host (row, col) uint64 arrays."""
    h = t.cpu().numpy()
    if k <= 32:
        h = h.view(np.uint32)
    else:
        h = h.view(np.uint64)
    return h[:, 0].astype(np.uint64), h[:, 1].astype(np.uint64)


def gpu_edges(table, k, seed, e0, count, stream=None):
    out = rm.empty_edges(count, k)
    rm.rmat_generate(table, seed, e0, count, out, stream)
    torch.cuda.synchronize()
    return as_u64_pairs(out, k)


def assert_same(gpu, ref):
    r_g, c_g = gpu
    r_o, c_o = ref
    bad = np.nonzero((r_g != r_o) | (c_g != c_o))[0]
    assert bad.size == 0, f"{bad.size} edges differ; first at {bad[:5]}: gpu {r_g[bad[:3]]},{c_g[bad[:3]]} oracle {r_o[bad[:3]]},{c_o[bad[:3]]}"


# ----------------------------------------------------------- whole outputs --

def test_plain_k16_fixed_l4_full():
    """k = 16, m = 2^20, Graph 500 parameters, fixed l = 4 (256 entries), seed 1."""
    k, m = 16, 1 << 20
    t = rm.rmat_build_table_fixed(*G500, k, 4)
    assert_same(gpu_edges(t, k, 1, 0, m), oracle.generate([oracle.Table.fixed([G500], 4)], k, 1, 0, m))


@pytest.mark.parametrize("count,e0", [(1, 0), (31, 7), (33, 0), (4097, 12345), ((1 << 18) + 37, (1 << 32) - 1000)])
def test_k26_variable_ragged(count, e0):
    k = 26
    t = rm.rmat_build_table(*G500, k, 4096)
    ot = oracle.Table.variable(*G500, k, 4096)
    assert_same(gpu_edges(t, k, 1, e0, count), oracle.generate([ot], k, 1, e0, count))


@pytest.mark.parametrize("params,k,bound", [
    (G500, 26, 256), (ASYM, 20, 1000), (SKEWED, 26, 8192), (SKEWED, 32, 4096),
    (G500, 1, 16), (G500, 32, 4096), (G500, 33, 4096), (SKEWED, 64, 4096), (G500, 40, 5),
    (G500, 26, 1 << 16),   # table larger than shared memory: read from global
    (SKEWED, 30, 1 << 15),  # paths > 13 levels (wide entries), global table
])
def test_variable_tables(params, k, bound):
    m = 50_000
    t = rm.rmat_build_table(*params, k, bound)
    ot = oracle.Table.variable(*params, k, bound)
    assert_same(gpu_edges(t, k, 99, 3, m), oracle.generate([ot], k, 99, 3, m))


@pytest.mark.parametrize("params,k,ell", [(G500, 26, 6), (ASYM, 9, 4), (G500, 34, 5), (ASYM, 12, 12),
                                          (SKEWED, 64, 7), (G500, 3, 5)])
def test_fixed_tables(params, k, ell):
    m = 40_000
    t = rm.rmat_build_table_fixed(*params, k, ell)
    assert_same(gpu_edges(t, k, 5, 0, m), oracle.generate([oracle.Table.fixed([params], ell)], k, 5, 0, m))


@pytest.mark.parametrize("k,ell,undirected", [(34, 6, True), (34, 5, True), (34, 5, False), (20, 3, True),
                                              (7, 12, False), (64, 4, True)])
def test_per_level_tables(k, ell, undirected):
    m = 40_000
    P = noisy_levels(k, seed=7 + k + ell)
    t = rm.rmat_build_table_levels(P, k, ell, rm.RMAT_UNDIRECTED if undirected else 0)
    ref = oracle.generate(oracle.level_groups(P, k, ell), k, 34, 1 << 34, m, undirected=undirected)
    assert_same(gpu_edges(t, k, 34, 1 << 34, m), ref)


def test_undirected_flag_on_single_table():
    k, m = 26, 20_000
    t = rm.rmat_build_table(*G500, k, 4096)
    rm.rmat_table_set_flags(t, rm.RMAT_UNDIRECTED)
    ref = oracle.generate([oracle.Table.variable(*G500, k, 4096)], k, 3, 0, m, undirected=True)
    assert_same(gpu_edges(t, k, 3, 0, m), ref)


@pytest.mark.parametrize("params,k", [(G500, 26), (ASYM, 13), (G500, 40)])
def test_naive_kernel_matches_oracle(params, k):
    m = 30_000
    out = rm.empty_edges(m, k)
    rm.rmat_generate_naive(params, k, 0, 17, 100, m, out)
    torch.cuda.synchronize()
    assert_same(as_u64_pairs(out, k), oracle.generate_naive([params], k, 17, 100, m))


def test_launch_shape_does_not_change_output():
    k, m = 26, (1 << 17) + 5
    t = rm.rmat_build_table(*G500, k, 4096)
    ref = gpu_edges(t, k, 8, 0, m)
    for threads, ctas, tile in [(128, 1, 32), (256, 4, 64), (256, 2, 96), (512, 1, 160), (512, 2, 1024),
                                (1024, 1, 256), (1024, 1, 512)]:
        rm.rmat_set_launch_config(t, threads, ctas, tile)
        assert_same(gpu_edges(t, k, 8, 0, m), ref)


def test_chunking_does_not_change_output():
    k, m = 26, 100_000
    t = rm.rmat_build_table(*G500, k, 4096)
    whole = gpu_edges(t, k, 4, 0, m)
    parts = [gpu_edges(t, k, 4, a, b - a) for a, b in [(0, 1), (1, 33333), (33333, 33334), (33334, m)]]
    r = np.concatenate([p[0] for p in parts])
    c = np.concatenate([p[1] for p in parts])
    assert_same((r, c), whole)


def test_unaligned_output_and_guard_region():
    """An output that is 8- but not 16-byte aligned takes the plain-store path;
    nothing outside [out, out + count) is written."""
    k, m = 26, 10_001
    t = rm.rmat_build_table(*G500, k, 4096)
    buf = torch.full((m + 64, 2), -1, dtype=torch.int32, device="cuda")
    view = buf[1:1 + m]
    assert view.data_ptr() % 16 == 8
    rm.rmat_generate(t, 6, 0, m, view)
    torch.cuda.synchronize()
    assert_same(as_u64_pairs(view, k), oracle.generate([oracle.Table.variable(*G500, k, 4096)], k, 6, 0, m))
    h = buf.cpu()
    assert bool((h[0] == -1).all()) and bool((h[1 + m:] == -1).all())


def test_generate_host_matches_device():
    k, m = 26, (1 << 26) + 11   # crosses the 256 MiB staging chunk
    t = rm.rmat_build_table(*G500, k, 4096)
    dev = rm.empty_edges(m, k)
    rm.rmat_generate(t, 2, 5, m, dev)
    host = rm.empty_edges(m, k, device="cpu", pin_memory=True)
    rm.rmat_generate_host(t, 2, 5, m, host)
    torch.cuda.synchronize()
    assert torch.equal(dev.cpu(), host)


def test_streams_are_honoured():
    k, m = 26, 1 << 20
    t = rm.rmat_build_table(*G500, k, 4096)
    s = torch.cuda.Stream()
    out = rm.empty_edges(m, k)
    with torch.cuda.stream(s):
        rm.rmat_generate(t, 1, 0, m, out, s)
    s.synchronize()
    assert_same(as_u64_pairs(out[:4096], k), oracle.generate([oracle.Table.variable(*G500, k, 4096)], k, 1, 0, 4096))


def test_tables_with_different_shared_memory_needs_interleave():
    """Launch plans are cached per table; the kernel's shared-memory limit is
    per function.  Alternating a large and a small table of the same kernel
    must keep working (and stay exact)."""
    k, m = 26, 70_000
    big = rm.rmat_build_table(*G500, k, 1 << 14)    # ~129 KiB blob, smaller tiles
    small = rm.rmat_build_table(*G500, k, 256)
    refs = {}
    for name, t, bound in [("big", big, 1 << 14), ("small", small, 256), ("big", big, 1 << 14), ("small", small, 256)]:
        got = gpu_edges(t, k, 9, 0, m)
        if name not in refs:
            refs[name] = oracle.generate([oracle.Table.variable(*G500, k, bound)], k, 9, 0, m)
        assert_same(got, refs[name])


@pytest.mark.parametrize("kind,k,undirected", [("variable", 26, False), ("variable", 26, True), ("fixed", 16, False),
                                               ("variable", 40, True), ("levels", 34, True), ("variable", 32, False),
                                               ("levels", 20, False), ("levels", 32, True)])
def test_scrambled_ids_match_oracle(kind, k, undirected):
    m = 30_000
    if kind == "variable":
        t = rm.rmat_build_table(*G500, k, 4096)
        ot = [oracle.Table.variable(*G500, k, 4096)]
    elif kind == "fixed":
        t = rm.rmat_build_table_fixed(*ASYM, k, 4)
        ot = [oracle.Table.fixed([ASYM], 4)]
    else:
        P = noisy_levels(k, seed=5)
        t = rm.rmat_build_table_levels(P, k, 6)
        ot = oracle.level_groups(P, k, 6)
    rm.rmat_table_set_flags(t, rm.RMAT_UNDIRECTED if undirected else 0)
    rm.rmat_table_set_scramble(t, True, 2024 + k)
    ref = oracle.generate_scrambled(ot, k, 2024 + k, 77, 5, m, undirected=undirected)
    assert_same(gpu_edges(t, k, 77, 5, m), ref)
    rm.rmat_table_set_scramble(t, False)
    assert_same(gpu_edges(t, k, 77, 5, m), oracle.generate(ot, k, 77, 5, m, undirected=undirected))


@pytest.mark.parametrize("e0,count", [((1 << 64) - 5001, 5000), ((1 << 63) + 17, 3000), ((1 << 32) - 7, 64)])
def test_edge_offsets_at_the_top_of_the_counter(e0, count):
    """Edge numbers near 2^64 (counter words 2 and 3 of the Philox block);
    edge_offset + count must fit 64 bits, so the last usable edge is 2^64 - 2."""
    k = 26
    t = rm.rmat_build_table(*G500, k, 4096)
    ot = oracle.Table.variable(*G500, k, 4096)
    assert_same(gpu_edges(t, k, 99, e0, count), oracle.generate([ot], k, 99, e0, count))
    with pytest.raises(rm.RmatError):     # e0 + count past 2^64 is refused on the host
        rm.rmat_generate(t, 99, (1 << 64) - 10, 11, rm.empty_edges(11, k))
