"""Serving with continuous batching: every request's result is the same
alone and in the mix -- checksums and full chunk bytes (seen through the
callback) against the CPU oracle and against the single-graph entry point --
admission backs off on memory, and host-side waits time out without
disturbing the server."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle
import paper_1905_03525_gb300 as rm
from paper_1905_03525_gb300 import _capi
from paper_1905_03525_gb300.serve import DONE, Server
from paper_1905_03525_gb300.workloads import G500, SKEWED

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M1 = np.uint64(0x9E3779B97F4A7C15)
M2 = np.uint64(0xC2B2AE3D27D4EB4F)
M3 = np.uint64(0x165667B19E3779F9)
F1 = np.uint64(0xBF58476D1CE4E5B9)
F2 = np.uint64(0x94D049BB133111EB)


def host_checksum(rows, cols, e0):
    """The checksum documented in include/rmat.h, recomputed on the host."""
    with np.errstate(over="ignore"):
        e = np.arange(e0, e0 + len(rows), dtype=np.uint64)
        x = e * M1 + rows.astype(np.uint64) * M2 + cols.astype(np.uint64) * M3
        x = (x ^ (x >> np.uint64(30))) * F1
        x = (x ^ (x >> np.uint64(27))) * F2
        x = x ^ (x >> np.uint64(31))
        return int(x.sum(dtype=np.uint64))


def alone(abcd, k, m, seed, bound=4096):
    t = rm.rmat_build_table(*abcd, k, bound)
    out = rm.empty_edges(m, k)
    rm.rmat_generate(t, seed, 0, m, out)
    torch.cuda.synchronize()
    h = out.cpu().numpy()
    h = h.view(np.uint32) if k <= 32 else h.view(np.uint64)
    return h[:, 0].astype(np.uint64), h[:, 1].astype(np.uint64)


def oracle_edges(abcd, k, m, seed, bound, undirected=False, scramble_seed=None):
    """The request's edges from the CPU oracle (table of the bound the server used)."""
    t = [oracle.Table.variable(*abcd, k, bound)]
    if scramble_seed is not None:
        return oracle.generate_scrambled(t, k, scramble_seed, seed, 0, m, undirected=undirected)
    return oracle.generate_parallel(t, k, seed, 0, m, undirected=undirected)


REQS = [(G500, 20, 100_000, 1), (SKEWED, 26, 300_001, 2), ((0.5, 0.2, 0.25, 0.05), 12, 5_000, 3),
        (G500, 30, 1 << 19, 4), (G500, 16, 70_000, 5), ((0.45, 0.22, 0.22, 0.11), 24, 250_000, 6),
        (G500, 34, 40_000, 7), (G500, 8, 1, 8), (SKEWED, 18, 200_000, 9), (G500, 22, 65_536, 10)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1905_03525_gb300 import build
    build.build()


def test_results_same_alone_and_in_the_mix():
    # small chunks and few slots: requests queue, interleave and share steps
    with Server(256 << 20, chunk_edges=1 << 16, step_edges=1 << 18, max_active=4) as srv:
        ids = [srv.submit(*p, k, m, s) for p, k, m, s in REQS]
        srv.drain(600)
        mixed = [srv.status(i) for i in ids]
        st = srv.stats()
    assert all(x["state"] == DONE and x["edges_done"] == m for x, (_, _, m, _) in zip(mixed, REQS))
    assert st["steps"] > len(REQS)  # multi-chunk requests really were split
    for x, (p, k, m, s) in zip(mixed, REQS):
        r, c = oracle_edges(p, k, m, s, x["table_bound"])
        assert x["checksum"] == host_checksum(r, c, 0), ("oracle", k, m)
        r, c = alone(p, k, m, s, x["table_bound"])
        assert x["checksum"] == host_checksum(r, c, 0), ("alone", k, m)
    # auto bounds: deep (wide-entry) tables were shrunk to fit shared memory
    assert mixed[1]["table_bound"] < mixed[0]["table_bound"] <= 8192
    # one request alone on its own server gives the same checksum
    with Server(64 << 20, chunk_edges=1 << 20, step_edges=1 << 20, max_active=1) as srv:
        p, k, m, s = REQS[1]
        assert srv.wait(srv.submit(*p, k, m, s))["checksum"] == mixed[1]["checksum"]


def _cudart():
    for name in ("libcudart.so", "libcudart.so.13", ctypes.util.find_library("cudart")):
        if not name:
            continue
        for d in ("", "/usr/local/cuda/lib64/"):
            try:
                return ctypes.CDLL(d + name)
            except OSError:
                pass
    pytest.skip("CUDA runtime library not found for the callback copy")


def test_chunk_callback_sees_every_edge():
    rt = _cudart()
    rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    got = {}

    def on_chunk(rid, off, cnt, ptr):
        eb = got[rid]["eb"]
        buf = np.empty(cnt * eb // 4, np.uint32)
        assert rt.cudaMemcpy(buf.ctypes.data, ptr, cnt * eb, 2) == 0
        got[rid]["parts"].append((off, buf))

    reqs = [(G500, 26, 50_001, 11, 0), (SKEWED, 40, 33_000, 12, 4096), (G500, 12, 777, 13, 0)]
    with Server(128 << 20, chunk_edges=8192, step_edges=1 << 15, max_active=3) as srv:
        srv.set_chunk_callback(on_chunk)
        for p, k, m, s, bound in reqs:
            rid = srv.submit(*p, k, m, s, bound)
            got[rid] = {"eb": 8 if k <= 32 else 16, "parts": [], "req": (p, k, m, s)}
        srv.drain(600)
        bounds = {rid: srv.status(rid)["table_bound"] for rid in got}
    # explicit bound kept; G500 at k = 26 needs wide 8192-column entries (too big), at k = 12 it fits
    assert sorted(bounds.values()) == [4096, 4096, 8192]
    for rid, g in got.items():
        p, k, m, s = g["req"]
        parts = sorted(g["parts"], key=lambda x: x[0])
        assert [o for o, _ in parts] == list(range(0, m, 8192))
        data = np.concatenate([b for _, b in parts])
        data = data.view(np.uint32 if k <= 32 else np.uint64).reshape(-1, 2)
        r, c = alone(p, k, m, s, bounds[rid])
        assert np.array_equal(data[:, 0].astype(np.uint64), r) and np.array_equal(data[:, 1].astype(np.uint64), c)


def test_served_bytes_match_oracle():
    """One request of each kind -- u32, u64 IDs, undirected, scrambled, and a
    skewed deep table -- served together with the server's own table bounds;
    every byte seen by the callback and every checksum against the oracle."""
    rt = _cudart()
    rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    got = {}

    def on_chunk(rid, off, cnt, ptr):
        eb = got[rid]["eb"]
        buf = np.empty(cnt * eb // 4, np.uint32)
        assert rt.cudaMemcpy(buf.ctypes.data, ptr, cnt * eb, 2) == 0
        got[rid]["parts"].append((off, buf))

    # (params, k, m, seed, flags, scramble seed)
    reqs = [(G500, 24, 300_007, 21, 0, None), (G500, 44, 120_001, 22, 0, None),
            (SKEWED, 30, 200_003, 23, rm.RMAT_UNDIRECTED, None), ((0.45, 0.22, 0.22, 0.11), 28, 150_000, 24, 0, 99),
            (G500, 36, 90_000, 25, rm.RMAT_UNDIRECTED, 7), (SKEWED, 26, 250_000, 26, 0, None)]
    with Server(256 << 20, chunk_edges=1 << 15, step_edges=1 << 17, max_active=3) as srv:
        srv.set_chunk_callback(on_chunk)
        for p, k, m, s, fl, scr in reqs:
            rid = srv.submit(*p, k, m, s, flags=fl, scramble_seed=scr)
            got[rid] = {"eb": 8 if k <= 32 else 16, "parts": [], "req": (p, k, m, s, fl, scr)}
        srv.drain(600)
        status = {rid: srv.status(rid) for rid in got}
    for rid, g in got.items():
        p, k, m, s, fl, scr = g["req"]
        st = status[rid]
        assert st["state"] == DONE and st["edges_done"] == m
        parts = sorted(g["parts"], key=lambda x: x[0])
        assert [o for o, _ in parts] == list(range(0, m, 1 << 15))
        data = np.concatenate([b for _, b in parts]).view(np.uint32 if k <= 32 else np.uint64).reshape(-1, 2)
        r, c = oracle_edges(p, k, m, s, st["table_bound"], undirected=bool(fl), scramble_seed=scr)
        bad = np.nonzero((data[:, 0] != r) | (data[:, 1] != c))[0]
        assert bad.size == 0, (k, fl, scr, st["table_bound"], bad[:5])
        assert st["checksum"] == host_checksum(r, c, 0), (k, fl, scr)


def test_large_bound_tables_built_on_the_gpu():
    """Requests with a large explicit bound get their table from the GPU
    build on the server's builder thread (parameters outside its range fall
    back to the host build); their bytes are the oracle's, and small requests
    submitted behind them are not held up."""
    reqs = [(G500, 26, 200_000, 31, 1 << 16), (SKEWED, 24, 100_003, 32, 1 << 15),
            ((0.6, 0.2, 0.2, 0.0), 20, 50_000, 33, 1 << 14),   # d = 0: host build
            (G500, 18, 30_000, 34, 0), ((0.45, 0.22, 0.22, 0.11), 22, 70_000, 35, 0)]
    with Server(256 << 20, chunk_edges=1 << 16, step_edges=1 << 18, max_active=4,
                gpu_build_min_bound=1 << 14) as srv:
        ids = [srv.submit(*p, k, m, s, bound) for p, k, m, s, bound in reqs]
        srv.drain(600)
        sts = [srv.status(i) for i in ids]
    for st, (p, k, m, s, bound) in zip(sts, reqs):
        assert st["state"] == DONE and st["edges_done"] == m, st
        if bound:
            assert st["table_bound"] == bound
        r, c = oracle_edges(p, k, m, s, st["table_bound"])
        assert st["checksum"] == host_checksum(r, c, 0), (k, bound)


def test_admission_backs_off_on_memory():
    # 1 MiB holds one request at a time (33 KiB table + 512 KiB chunk buffer)
    with Server(1 << 20, chunk_edges=1 << 16, step_edges=1 << 16, max_active=8) as srv:
        ids = [srv.submit(*G500, 20, 200_000, s) for s in range(3)]
        srv.drain(600)
        sts = [srv.status(i) for i in ids]
    assert all(x["state"] == DONE for x in sts)
    # one at a time: each admission comes after the previous completion
    spans = sorted((x["admit_s"], x["done_s"]) for x in sts)
    assert all(spans[i + 1][0] >= spans[i][1] - 1e-6 for i in range(len(spans) - 1))
    for x, s in zip(sts, range(3)):
        r, c = alone(G500, 20, 200_000, s)
        assert x["checksum"] == host_checksum(r, c, 0)


def test_rejections_and_timeouts():
    with Server(1 << 20, chunk_edges=1 << 20, step_edges=1 << 20, max_active=2) as srv:
        with pytest.raises(rm.RmatError) as ei:
            srv.submit(*G500, 26, 1 << 20, 1)      # 8 MiB chunk > 1 MiB budget: never fits
        assert ei.value.status == _capi.RMAT_ERR_OUT_OF_MEMORY
        with pytest.raises(rm.RmatError) as ei:
            srv.submit(*G500, 0, 10, 1)
        assert ei.value.status == _capi.RMAT_ERR_INVALID_ARGUMENT
    with Server(64 << 20, chunk_edges=1 << 20, step_edges=1 << 20, max_active=2) as srv:
        rid = srv.submit(*G500, 26, 1 << 26, 1)   # 64 steps of 2^20 edges
        with pytest.raises(rm.RmatError) as ei:
            srv.wait(rid, 0.0005)
        assert ei.value.status == _capi.RMAT_ERR_TIMEOUT
        assert srv.wait(rid, 600)["state"] == DONE


def test_scrambled_request_matches_scrambled_table():
    p, k, m, s = SKEWED, 26, 300_001, 2
    with Server(128 << 20, chunk_edges=1 << 16, step_edges=1 << 18, max_active=2) as srv:
        plain = srv.submit(*p, k, m, s)
        scr = srv.submit(*p, k, m, s, scramble_seed=4242)
        srv.drain(600)
        a, b = srv.status(plain), srv.status(scr)
    assert a["state"] == DONE and b["state"] == DONE and a["checksum"] != b["checksum"]
    t = rm.rmat_build_table(*p, k, b["table_bound"])
    rm.rmat_table_set_scramble(t, True, 4242)
    out = rm.empty_edges(m, k)
    rm.rmat_generate(t, s, 0, m, out)
    torch.cuda.synchronize()
    h = out.cpu().numpy().view(np.uint32)
    assert b["checksum"] == host_checksum(h[:, 0].astype(np.uint64), h[:, 1].astype(np.uint64), 0)
