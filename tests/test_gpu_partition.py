"""GPU parity for partitioned graphs (Sec. 3): every PE's tiles generated by
the batched kernel with the tile levels fixed, against the CPU oracle, bit for
bit, through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_1905_03525_gb300 as rm
from paper_1905_03525_gb300.workloads import G500, SKEWED

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


def pairs(t, k):
    h = t.cpu().numpy()
    h = h.view(np.uint32) if k <= 32 else h.view(np.uint64)
    return h[:, 0].astype(np.uint64), h[:, 1].astype(np.uint64)


def assert_same(gpu, ref):
    bad = np.nonzero((gpu[0] != ref[0]) | (gpu[1] != ref[1]))[0]
    assert bad.size == 0, f"{bad.size} edges differ; first at {bad[:5]}"


@pytest.mark.parametrize("kind,params,k,t,m,seed,rows", [
    ("variable", G500, 20, 3, 300_001, 1, None),           # several tiles, ragged counts
    ("variable", ASYM, 12, 0, 70_000, 2, None),            # one tile = the plain graph
    ("fixed", ASYM, 16, 4, 200_000, 3, (5, 9)),            # one PE's rows
    ("variable", SKEWED, 30, 6, 150_000, 4, (0, 7)),       # wide path entries
    ("variable", G500, 40, 5, 60_000, 5, None),            # u64 output
    ("variable", G500, 14, 14, 5_000, 6, None),            # tiles of one cell: no draws
    ("variable", G500, 26, 2, 1, 7, None),                 # a single edge
    ("variable", G500, 26, 5, 2_000_003, 9, (3, 20)),      # the bench's tiles, one PE's rows
])
def test_partition_matches_oracle(kind, params, k, t, m, seed, rows):
    table = rm.rmat_build_table(*params, k, 4096) if kind == "variable" else rm.rmat_build_table_fixed(*params, k, 4)
    ot = oracle.Table.variable(*params, k, 4096) if kind == "variable" else oracle.Table.fixed([params], 4)
    r0, r1 = rows if rows else (0, 1 << t)
    p = rm.rmat_partition_create(table, t, m, seed, r0, r1)
    ntiles, edges = rm.rmat_partition_info(p)
    out = rm.empty_edges(max(edges, 1), k)
    rm.rmat_generate_partition(p, out)
    torch.cuda.synchronize()
    tiles, ref = oracle.generate_partitioned(ot, params, k, t, m, seed, r0, r1)
    assert ntiles == len(tiles["row"]) and edges == len(ref[0])
    assert_same(pairs(out[:edges], k), ref)
    if t == 0:
        plain = rm.empty_edges(m, k)
        rm.rmat_generate(table, seed, 0, m, plain)
        torch.cuda.synchronize()
        assert torch.equal(plain, out[:m])


def test_batch_tiles_mix_with_plain_graphs():
    """Tiles of two partitions and plain graphs in one batched launch."""
    ta = rm.rmat_build_table(*G500, 22, 2048)
    tb = rm.rmat_build_table_fixed(*ASYM, 18, 5)
    oa, ob = oracle.Table.variable(*G500, 22, 2048), oracle.Table.fixed([ASYM], 5)
    b = rm.rmat_batch_create()
    cases = [(ta, oa, 22, 4, 11, 5, 9, 40_000, 3), (tb, ob, 18, 7, 100, 27, 1, 33_333, 0),
             (ta, oa, 22, 0, 0, 0, 4, 25_000, 77)]
    outs = []
    for t, _, k, lv, R, C, seed, n, first in cases:
        o = rm.empty_edges(n, k)
        rm.rmat_batch_add_tile(b, t, seed, first, n, lv, R, C, o)
        outs.append(o)
    rm.rmat_batch_launch(b)
    torch.cuda.synchronize()
    for (t, ot, k, lv, R, C, seed, n, first), o in zip(cases, outs):
        assert_same(pairs(o, k), oracle.generate_tile(ot, k, lv, R, C, seed, first, n))


def test_partition_output_buffer_can_change():
    table = rm.rmat_build_table(*G500, 20, 4096)
    p = rm.rmat_partition_create(table, 4, 100_000, 8)
    _, edges = rm.rmat_partition_info(p)
    a, b = rm.empty_edges(edges, 20), rm.empty_edges(edges + 1, 20)
    rm.rmat_generate_partition(p, a)
    rm.rmat_generate_partition(p, b[1:])     # another (8-byte aligned) buffer
    rm.rmat_generate_partition(p, a)         # and back
    torch.cuda.synchronize()
    assert torch.equal(a, b[1:])


def test_partition_full_size_two_pes():
    """k = 26, m = 2^30 in 2^5 x 2^5 tiles, split over two PEs by tile rows:
    together they hold every edge once; sampled tiles match the oracle and
    every edge lies in its tile."""
    k, t, m, seed = 26, 5, 1 << 30, 1
    table = rm.rmat_build_table(*G500, k, 4096)
    ot = oracle.Table.variable(*G500, k, 4096)
    total = 0
    rng = np.random.default_rng(5)
    for r0, r1 in [(0, 9), (9, 32)]:
        p = rm.rmat_partition_create(table, t, m, seed, r0, r1)
        tl = rm.rmat_partition_tiles(p)
        ntiles, edges = rm.rmat_partition_info(p)
        total += edges
        out = rm.empty_edges(edges, k)
        rm.rmat_generate_partition(p, out)
        torch.cuda.synchronize()
        rows = out[:, 0].view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        assert int((rows >> (k - t)).min()) >= r0 and int((rows >> (k - t)).max()) < r1
        pos = np.concatenate([[0], np.cumsum(tl["count"])]).astype(np.int64)
        for i in rng.choice(ntiles, 12, replace=False):
            n = int(min(tl["count"][i], 1500))
            s = int(pos[i]) + int(tl["count"][i]) - n           # the tile's last n edges
            ref = oracle.generate_tile(ot, k, t, int(tl["row"][i]), int(tl["col"][i]), seed,
                                       int(tl["first"][i]) + int(tl["count"][i]) - n, n)
            assert_same(pairs(out[s:s + n], k), ref)
        del out
        torch.cuda.empty_cache()
    assert total == m


def _dedup_gpu(out, n, k):
    u = rm.rmat_dedup_edges(out, n, k)
    torch.cuda.synchronize()
    return u, pairs(out[:u], k)


@pytest.mark.parametrize("k,m", [(8, 200_000), (12, 100_003), (3, 5000), (20, 1 << 20),
                                 (12, (3 << 21) + 7), (24, (1 << 23) + 3)])   # the last two: two levels of buckets
def test_dedup_keeps_first_occurrences(k, m):
    t = rm.rmat_build_table(*G500, k, 256)
    ot = oracle.Table.variable(*G500, k, 256)
    out = rm.empty_edges(m, k)
    rm.rmat_generate(t, 3, 0, m, out)
    u, got = _dedup_gpu(out, m, k)
    ref = oracle.dedup_first(*oracle.generate([ot], k, 3, 0, m))
    assert u == len(ref[0])
    assert_same(got, ref)


def test_dedup_of_a_2p26_partition_output():
    """The partition workload's PE output at 2^26 edges (2^15 buckets): the GPU's
    duplicate removal against the oracle's first-occurrence filter of the
    same array."""
    k, t, m, seed = 26, 5, 1 << 26, 1
    table = rm.rmat_build_table(*G500, k, 4096)
    p = rm.rmat_partition_create(table, t, m, seed)
    _, edges = rm.rmat_partition_info(p)
    out = rm.empty_edges(edges, k)
    rm.rmat_generate_partition(p, out)
    torch.cuda.synchronize()
    ref = oracle.dedup_first(*pairs(out, k))
    u, got = _dedup_gpu(out, edges, k)
    assert u == len(ref[0])
    assert_same(got, ref)
    del out
    torch.cuda.empty_cache()


def test_dedup_edge_cases():
    one = rm.empty_edges(1, 10)
    one.fill_(5)
    assert rm.rmat_dedup_edges(one, 1, 10) == 1
    same = rm.empty_edges(4096, 10)
    same.fill_(7)
    assert rm.rmat_dedup_edges(same, 4096, 10) == 1
    assert rm.rmat_dedup_edges(same, 0, 10) == 0
    with pytest.raises(rm.RmatError):
        rm.rmat_dedup_edges(same, 10, 32)


def _to_device(h, out):
    out.copy_(torch.from_numpy(np.ascontiguousarray(h).view(np.int32)))


def test_dedup_heavy_repeats_use_the_overflow_table():
    """Keys repeated more often than a shared-memory bucket holds (30000,
    9000 and 7000 copies among 400000 edges) go through the device-memory
    table; the result still equals the oracle's first-occurrence filter."""
    k, m = 20, 400_000
    t = rm.rmat_build_table(*G500, k, 256)
    out = rm.empty_edges(m, k)
    rm.rmat_generate(t, 5, 0, m, out)
    torch.cuda.synchronize()
    h = out.cpu().numpy().view(np.uint32).copy()
    rng = np.random.default_rng(11)
    for (r, c), copies in (((3, 5), 30_000), ((100, 7), 9_000), ((1, 1), 7_000)):
        at = rng.choice(m, copies, replace=False)
        h[at, 0], h[at, 1] = r, c
    _to_device(h, out)
    ref = oracle.dedup_first(h[:, 0].astype(np.uint64), h[:, 1].astype(np.uint64))
    u, got = _dedup_gpu(out, m, k)
    assert u == len(ref[0])
    assert_same(got, ref)


def test_dedup_of_two_keys_in_4m_edges():
    """2^22 edges alternating between two keys: at most two buckets, each of
    about 2^21 edges, both far above the shared-memory limit."""
    k, m = 16, 1 << 22
    h = np.empty((m, 2), np.uint32)
    h[0::2] = (9, 4)
    h[1::2] = (4, 9)
    out = rm.empty_edges(m, k)
    _to_device(h, out)
    u, got = _dedup_gpu(out, m, k)
    assert u == 2
    assert got[0].tolist() == [9, 4] and got[1].tolist() == [4, 9]


def test_dedup_of_distinct_edges_keeps_all():
    """(2^21 + 5) distinct edges in a scrambled order (two levels of buckets,
    a ragged bitmap tail): nothing is removed and the order is kept."""
    k, m = 22, (1 << 21) + 5
    rng = np.random.default_rng(2)
    v = rng.permutation(1 << 22)[:m].astype(np.uint32)
    h = np.stack([v, (v * 7 + 3) & ((1 << 22) - 1)], axis=1).astype(np.uint32)
    out = rm.empty_edges(m, k)
    _to_device(h, out)
    u, got = _dedup_gpu(out, m, k)
    assert u == m
    assert np.array_equal(got[0], h[:, 0]) and np.array_equal(got[1], h[:, 1])


def test_dedup_release_and_reuse():
    """The kept scratch is freed on request; the next call allocates it again
    and gives the same result; releasing twice is harmless."""
    k, m = 14, 123_457
    t = rm.rmat_build_table(*G500, k, 256)
    out = rm.empty_edges(m, k)
    rm.rmat_generate(t, 8, 0, m, out)
    keep = out.clone()
    u1, got1 = _dedup_gpu(out, m, k)
    rm.rmat_dedup_release()
    rm.rmat_dedup_release()
    u2, got2 = _dedup_gpu(keep, m, k)
    assert u1 == u2
    assert_same(got2, got1)


def test_partitioned_dedup_is_local():
    """Duplicates only meet inside a tile, so the PEs' own duplicate removal
    gives the whole graph's distinct edges, each exactly once."""
    k, t, m, seed = 10, 2, 300_000, 4
    table = rm.rmat_build_table(*G500, k, 512)
    ot = oracle.Table.variable(*G500, k, 512)
    kept = []
    for r0, r1 in [(0, 1), (1, 4)]:
        p = rm.rmat_partition_create(table, t, m, seed, r0, r1)
        _, edges = rm.rmat_partition_info(p)
        out = rm.empty_edges(edges, k)
        rm.rmat_generate_partition(p, out)
        u, got = _dedup_gpu(out, edges, k)
        _, ref = oracle.generate_partitioned(ot, G500, k, t, m, seed, r0, r1)
        assert_same(got, oracle.dedup_first(*ref))
        kept.append(set(zip(got[0].tolist(), got[1].tolist())))
    assert not (kept[0] & kept[1])
    _, whole = oracle.generate_partitioned(ot, G500, k, t, m, seed)
    assert kept[0] | kept[1] == set(zip(whole[0].tolist(), whole[1].tolist()))
