"""The no-allocation entry point (rmat_generate_batch_noalloc), for callers
that cannot call cudaMalloc -- their device memory is reserved up front by
another allocator, or allocation would take locks on a latency-critical path.
Its scratch lives in a fixed library array, so the call must give exactly the
bytes of the ordinary entry point.  Two calls in a row check that nothing of
the first call's scratch leaks into the second; after the set-up call
(n = 0), calls take no device memory.

Collected last (file name) so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import ctypes

import pytest

import paper_1905_03525_gb300 as rm
from paper_1905_03525_gb300 import _capi
from paper_1905_03525_gb300.workloads import G500, SKEWED, batched_graphs, noisy_levels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1905_03525_gb300 import build
    build.build()


def _call_through_c_abi(tables, seeds, offsets, counts, outs, stream=0):
    n = len(tables)
    T = (ctypes.c_void_p * n)(*[t.handle.value for t in tables])
    S = (ctypes.c_uint64 * n)(*seeds)
    E = (ctypes.c_uint64 * n)(*offsets)
    C = (ctypes.c_uint64 * n)(*counts)
    O = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    _capi.check(_capi.lib().rmat_generate_batch_noalloc(T, S, E, C, O, n, stream))


def _reference(t, seed, e0, m, k):
    ref = rm.empty_edges(m, k)
    rm.rmat_generate(t, seed, e0, m, ref)
    return ref


def test_noalloc_matches_rmat_generate_twice():
    # first call: graphs of mixed table kinds and sizes (u32 output)
    gs = batched_graphs(6, seed=3, k_range=(10, 24), log2m_range=(10.0, 18.0))
    tabs = [rm.rmat_build_table(*g["abcd"], g["k"], 1 << (9 + i % 4)) for i, g in enumerate(gs)]
    tabs.append(rm.rmat_build_table(*SKEWED, 30, 1 << 13))      # wide path entries
    tabs.append(rm.rmat_build_table_fixed(*G500, 16, 4))
    tabs.append(tabs[0])                                         # the same table again: one blob, two jobs
    tabs.append(rm.rmat_build_table(*G500, 26, 1 << 14))        # 577 KiB: read from global memory
    ks = [g["k"] for g in gs] + [30, 16, gs[0]["k"], 26]
    seeds = [g["seed"] for g in gs] + [11, 1, 999, 3]
    offs = [0] * len(gs) + [12345, 0, 1 << 33, 77]
    counts = [g["m"] for g in gs] + [70_001, 1 << 20, 20_000, 90_001]
    outs = [rm.empty_edges(m, k) for m, k in zip(counts, ks)]
    _call_through_c_abi(tabs, seeds, offs, counts, outs)
    torch.cuda.synchronize()
    for t, s, e0, m, k, o in zip(tabs, seeds, offs, counts, ks, outs):
        assert torch.equal(o, _reference(t, s, e0, m, k))

    # second call right after: other graphs, fewer of them, u64 output
    P = noisy_levels(34)
    tabs2 = [rm.rmat_build_table_levels(P, 34, 6, rm.RMAT_UNDIRECTED), rm.rmat_build_table(*G500, 40, 4096)]
    seeds2, offs2, counts2 = [34, 5], [31 << 30, 7], [50_000, 33_333]
    outs2 = [rm.empty_edges(m, 34) for m in counts2]
    _call_through_c_abi(tabs2, seeds2, offs2, counts2, outs2)
    torch.cuda.synchronize()
    for t, s, e0, m, o in zip(tabs2, seeds2, offs2, counts2, outs2):
        assert torch.equal(o, _reference(t, s, e0, m, 34))

    # and the first call again gives the same bytes as before
    again = [torch.zeros_like(o) for o in outs]
    _call_through_c_abi(tabs, seeds, offs, counts, again)
    torch.cuda.synchronize()
    assert all(torch.equal(a, o) for a, o in zip(again, outs))
    rm.rmat_check_device_errors()


def test_noalloc_back_to_back_on_one_stream():
    """Two calls queued on one stream with no host synchronisation between
    them, on different graphs: the second call rebuilds the library's staging
    image while the first call's work may still be pending."""
    s = torch.cuda.Stream()
    a = [rm.rmat_build_table(*G500, 26, 4096), rm.rmat_build_table_fixed(*SKEWED, 18, 5)]
    b = [rm.rmat_build_table(*SKEWED, 22, 2048), rm.rmat_build_table(*G500, 30, 1024),
         rm.rmat_build_table(*G500, 12, 256)]
    ca, cb = [1 << 21, 300_003], [123_457, 1 << 20, 4097]
    ka, kb = [26, 18], [22, 30, 12]
    oa = [rm.empty_edges(m, k) for m, k in zip(ca, ka)]
    ob = [rm.empty_edges(m, k) for m, k in zip(cb, kb)]
    torch.cuda.synchronize()
    _call_through_c_abi(a, [5, 6], [0, 1 << 40], ca, oa, s.cuda_stream)
    _call_through_c_abi(b, [7, 8, 9], [3, 0, 1 << 20], cb, ob, s.cuda_stream)
    s.synchronize()
    for t, sd, e0, m, k, o in zip(a, [5, 6], [0, 1 << 40], ca, ka, oa):
        assert torch.equal(o, _reference(t, sd, e0, m, k))
    for t, sd, e0, m, k, o in zip(b, [7, 8, 9], [3, 0, 1 << 20], cb, kb, ob):
        assert torch.equal(o, _reference(t, sd, e0, m, k))


def test_noalloc_takes_no_device_memory_after_setup():
    """The set-up call (n = 0, NULL arrays) loads the scratch and the kernel;
    after it, calls leave the device's free memory unchanged."""
    _capi.check(_capi.lib().rmat_generate_batch_noalloc(None, None, None, None, None, 0, None))
    t = [rm.rmat_build_table(*G500, 26, 4096), rm.rmat_build_table(*G500, 40, 4096)]
    o32, o64 = rm.empty_edges(1 << 22, 26), rm.empty_edges(1 << 16, 40)
    _call_through_c_abi(t[:1], [1], [0], [1 << 22], [o32])
    _call_through_c_abi(t[1:], [2], [0], [1 << 16], [o64])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        _call_through_c_abi(t[:1], [1], [0], [1 << 22], [o32])
        _call_through_c_abi(t[1:], [2], [0], [1 << 16], [o64])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(o32, _reference(t[0], 1, 0, 1 << 22, 26))


def test_noalloc_scrambled_graphs():
    tabs = [rm.rmat_build_table(*G500, 26, 4096), rm.rmat_build_table(*SKEWED, 20, 1024)]
    rm.rmat_table_set_scramble(tabs[0], True, 9)
    counts = [100_003, 40_000]
    outs = [rm.empty_edges(m, k) for m, k in zip(counts, (26, 20))]
    _call_through_c_abi(tabs, [1, 2], [0, 5], counts, outs)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], _reference(tabs[0], 1, 0, counts[0], 26))
    assert torch.equal(outs[1], _reference(tabs[1], 2, 5, counts[1], 20))


def test_noalloc_rejects_what_does_not_fit():
    t = rm.rmat_build_table(*G500, 26, 4096)
    out = rm.empty_edges(8, 26)
    with pytest.raises(rm.RmatError) as ei:     # beyond the per-call maximum
        _call_through_c_abi([t], [1], [0], [(1 << 64) - 1], [out])
    assert ei.value.status == _capi.RMAT_ERR_INVALID_ARGUMENT
    big = 1 << 40   # needs far more unit entries than the scratch holds
    with pytest.raises(rm.RmatError) as ei:
        _call_through_c_abi([t], [1], [0], [big], [out])
    assert ei.value.status == _capi.RMAT_ERR_INVALID_ARGUMENT
    many = [t] * 65
    with pytest.raises(rm.RmatError):
        _call_through_c_abi(many, [1] * 65, [0] * 65, [8] * 65, [out] * 65)
    mixed = [t, rm.rmat_build_table(*G500, 40, 4096)]
    with pytest.raises(rm.RmatError):
        _call_through_c_abi(mixed, [1, 1], [0, 0], [8, 8], [out, rm.empty_edges(8, 40)])
