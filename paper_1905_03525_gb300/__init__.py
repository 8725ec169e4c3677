"""GB300-native R-MAT generation with constant work per edge (arXiv 1905.03525).

Python binding of librmat with the same names as the C ABI in include/rmat.h.
Tables are built on the host by the library; every edge is generated by the
library's sm_103a kernels.  PyTorch, when used, only supplies device memory
and streams: ``out`` arguments accept a CUDA tensor or a raw device address,
``stream`` accepts a ``torch.cuda.Stream``, a raw handle or None.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._capi import (RMAT_UNDIRECTED, LaunchConfig, RmatError, TableInfo, check, lib)

__all__ = [
    "RMAT_UNDIRECTED", "RmatError", "Table", "rmat_build_table", "rmat_build_table_fixed",
    "rmat_build_table_levels", "rmat_table_set_flags", "rmat_table_set_scramble", "rmat_table_info", "rmat_table_group_info",
    "rmat_table_export", "rmat_table_upload", "rmat_free_table", "rmat_generate", "rmat_generate_host",
    "rmat_generate_naive", "rmat_set_launch_config", "rmat_get_launch_config",
    "rmat_check_device_errors", "rmat_version", "edge_bytes", "empty_edges", "Batch", "rmat_batch_create",
    "rmat_batch_add", "rmat_batch_prepare", "rmat_batch_launch", "rmat_batch_size", "rmat_batch_free",
    "rmat_generate_batch_noalloc", "rmat_batch_add_tile", "Partition", "rmat_partition_create",
    "rmat_partition_info", "rmat_partition_tiles", "rmat_generate_partition", "rmat_free_partition",
    "rmat_build_table_kron", "rmat_build_table_kron_fixed", "empty_edges_for", "rmat_build_table_gpu",
    "rmat_dedup_edges", "rmat_dedup_release", "rmat_selftest_bounded_wait",
]


class Table:
    """Owning handle of an ``rmat_table``; freed with the object."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @property
    def handle(self):
        if not self._h:
            raise ValueError("table already freed")
        return self._h

    def free(self):
        if self._h:
            lib().rmat_free_table(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return rmat_table_info(self)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take an address of {type(x)!r}")


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    raise TypeError(f"not a stream: {type(s)!r}")


def _new_table(call) -> Table:
    h = ctypes.c_void_p()
    check(call(ctypes.byref(h)))
    return Table(h)


def rmat_build_table(a, b, c, d, k, table_bound) -> Table:
    """Variable-length table of similar-probability paths (Sec. 2)."""
    return _new_table(lambda out: lib().rmat_build_table(a, b, c, d, k, table_bound, out))


def rmat_build_table_gpu(a, b, c, d, k, table_bound, stream=None) -> Table:
    """rmat_build_table's table, built on the current GPU (Sec. 3 parallel
    construction); identical result."""
    return _new_table(lambda out: lib().rmat_build_table_gpu(a, b, c, d, k, table_bound, _stream(stream), out))


def rmat_build_table_fixed(a, b, c, d, k, ell) -> Table:
    """All 4^ell paths of length ell (Sec. 2)."""
    return _new_table(lambda out: lib().rmat_build_table_fixed(a, b, c, d, k, ell, out))


def rmat_build_table_levels(abcd, k, ell, flags=0) -> Table:
    """Per-level parameters (k x 4), one fixed-length table per ell levels (Sec. 3)."""
    P = np.ascontiguousarray(abcd, dtype=np.float64).reshape(-1, 4)
    if P.shape[0] != k:
        raise ValueError("abcd must have k rows")
    return _new_table(lambda out: lib().rmat_build_table_levels(P.ctypes.data, k, ell, flags, out))


def rmat_build_table_kron(theta, n0, k, table_bound) -> Table:
    """Stochastic Kronecker graph with an n0 x n0 initiator (Sec. 3):
    variable-length table of similar-probability paths."""
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(n0 * n0)
    return _new_table(lambda out: lib().rmat_build_table_kron(th.ctypes.data, n0, k, table_bound, out))


def rmat_build_table_kron_fixed(theta, n0, k, ell) -> Table:
    """Stochastic Kronecker graph: all (n0^2)^ell paths of length ell."""
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(n0 * n0)
    return _new_table(lambda out: lib().rmat_build_table_kron_fixed(th.ctypes.data, n0, k, ell, out))


def rmat_table_set_flags(t: Table, flags: int) -> None:
    check(lib().rmat_table_set_flags(t.handle, flags))


def rmat_table_set_scramble(t: Table, enable: bool, scramble_seed: int = 0) -> None:
    """Relabel vertex IDs by the seeded bijection of include/rmat.h (Sec. 3 scrambling)."""
    check(lib().rmat_table_set_scramble(t.handle, int(bool(enable)), scramble_seed))


def rmat_table_info(t: Table) -> dict:
    info = TableInfo()
    check(lib().rmat_table_info(t.handle, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in TableInfo._fields_}


def rmat_table_group_info(t: Table, group: int):
    e, b, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().rmat_table_group_info(t.handle, group, ctypes.byref(e), ctypes.byref(b), ctypes.byref(m)))
    return e.value, b.value, m.value


def rmat_table_export(t: Table, group: int = 0) -> dict:
    entries, bits, max_len = rmat_table_group_info(t, group)
    N = 1 << bits
    out = {"sym": np.zeros(N, np.uint64), "len": np.zeros(N, np.uint8), "p": np.zeros(N, np.float64),
           "w": np.zeros(N, np.uint64), "thr": np.zeros(N, np.uint32), "alias": np.zeros(N, np.uint32)}
    check(lib().rmat_table_export(t.handle, group, *[out[x].ctypes.data for x in
                                                     ("sym", "len", "p", "w", "thr", "alias")]))
    out.update(entries=entries, bits=bits, max_len=max_len)
    return out


def rmat_table_upload(t: Table) -> None:
    check(lib().rmat_table_upload(t.handle))


def rmat_free_table(t: Table) -> None:
    t.free()


def edge_bytes(k: int) -> int:
    """Bytes per edge of the output layout: uint32 pairs for k <= 32, else uint64."""
    return 8 if k <= 32 else 16


def empty_edges(count: int, k: int, device="cuda", pin_memory=False):
    """Allocate an output buffer for `count` edges as a torch tensor of shape
    (count, 2), uint32 (k <= 32) or int64 holding uint64 bits (k > 32)."""
    import torch
    dt = torch.int32 if k <= 32 else torch.int64
    if device == "cpu":
        return torch.empty((count, 2), dtype=dt, pin_memory=pin_memory)
    return torch.empty((count, 2), dtype=dt, device=device)


def empty_edges_for(t: Table, count: int, device="cuda", pin_memory=False):
    """Output buffer for `count` edges of table t (its vertex-ID width)."""
    import torch
    dt = torch.int32 if rmat_table_info(t)["index_bytes"] == 4 else torch.int64
    if device == "cpu":
        return torch.empty((count, 2), dtype=dt, pin_memory=pin_memory)
    return torch.empty((count, 2), dtype=dt, device=device)


def rmat_generate(t: Table, seed: int, edge_offset: int, count: int, out, stream=None) -> None:
    """Edges edge_offset .. edge_offset+count-1 into device memory `out` (async)."""
    check(lib().rmat_generate(t.handle, seed, edge_offset, count, _ptr(out), _stream(stream)))


def rmat_generate_host(t: Table, seed: int, edge_offset: int, count: int, host_out, stream=None) -> None:
    """Edges into host memory (blocking; pinned memory gives full bandwidth)."""
    check(lib().rmat_generate_host(t.handle, seed, edge_offset, count, _ptr(host_out), _stream(stream)))


def rmat_generate_naive(abcd, k, flags, seed, edge_offset, count, out, stream=None) -> None:
    """Plain per-bit R-MAT (Sec. 1) on the GPU: k quadrant draws per edge."""
    P = np.ascontiguousarray(abcd, dtype=np.float64).reshape(-1, 4)
    if P.shape[0] == 1:
        P = np.repeat(P, k, axis=0)
    check(lib().rmat_generate_naive(P.ctypes.data, k, flags, seed, edge_offset, count, _ptr(out),
                                    _stream(stream)))


def rmat_set_launch_config(t: Table, threads: int, ctas_per_sm: int, tile_edges: int) -> None:
    cfg = LaunchConfig(threads, ctas_per_sm, tile_edges)
    check(lib().rmat_set_launch_config(t.handle, ctypes.byref(cfg)))


def rmat_get_launch_config(t: Table) -> dict:
    cfg = LaunchConfig()
    check(lib().rmat_get_launch_config(t.handle, ctypes.byref(cfg)))
    return {"threads": cfg.threads, "ctas_per_sm": cfg.ctas_per_sm, "tile_edges": cfg.tile_edges}


class Batch:
    """Owning handle of an ``rmat_batch``; keeps its tables alive."""

    def __init__(self, handle):
        self._h = handle
        self._tables = []

    @property
    def handle(self):
        if not self._h:
            raise ValueError("batch already freed")
        return self._h

    def free(self):
        if self._h:
            lib().rmat_batch_free(self._h)
            self._h = None
            self._tables = []

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rmat_batch_create() -> Batch:
    h = ctypes.c_void_p()
    check(lib().rmat_batch_create(ctypes.byref(h)))
    return Batch(h)


def rmat_batch_add(b: Batch, t: Table, seed: int, edge_offset: int, count: int, out) -> None:
    check(lib().rmat_batch_add(b.handle, t.handle, seed, edge_offset, count, _ptr(out)))
    b._tables.append(t)


def rmat_batch_add_tile(b: Batch, t: Table, seed: int, edge_offset: int, count: int, tile_levels: int,
                        tile_row: int, tile_col: int, out) -> None:
    """A tile of a partitioned graph: edges started with their top
    tile_levels levels fixed to (tile_row, tile_col)."""
    check(lib().rmat_batch_add_tile(b.handle, t.handle, seed, edge_offset, count, tile_levels, tile_row, tile_col,
                                    _ptr(out)))
    b._tables.append(t)


def rmat_batch_prepare(b: Batch, threads=None, ctas_per_sm=None, tile_edges=None) -> None:
    if threads is None and ctas_per_sm is None and tile_edges is None:
        check(lib().rmat_batch_prepare(b.handle, None))
        return
    cfg = LaunchConfig(threads or 1024, ctas_per_sm or 1, tile_edges or 256)
    check(lib().rmat_batch_prepare(b.handle, ctypes.byref(cfg)))


def rmat_batch_launch(b: Batch, stream=None) -> None:
    check(lib().rmat_batch_launch(b.handle, _stream(stream)))


def rmat_batch_size(b: Batch):
    g, e = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().rmat_batch_size(b.handle, ctypes.byref(g), ctypes.byref(e)))
    return g.value, e.value


def rmat_batch_free(b: Batch) -> None:
    b.free()


def rmat_generate_batch_noalloc(tables, seeds, edge_offsets, counts, outs, stream=None) -> None:
    """Batched generation that allocates no device memory (scratch lives in a
    fixed library array; see include/rmat.h for the limits)."""
    n = len(tables)
    if not (len(seeds) == len(edge_offsets) == len(counts) == len(outs) == n):
        raise ValueError("argument lists differ in length")
    T = (ctypes.c_void_p * max(n, 1))(*[t.handle.value for t in tables])
    S = (ctypes.c_uint64 * max(n, 1))(*seeds)
    E = (ctypes.c_uint64 * max(n, 1))(*edge_offsets)
    C = (ctypes.c_uint64 * max(n, 1))(*counts)
    O = (ctypes.c_void_p * max(n, 1))(*[_ptr(o) for o in outs])
    check(lib().rmat_generate_batch_noalloc(T, S, E, C, O, n, _stream(stream)))


def rmat_check_device_errors() -> None:
    check(lib().rmat_check_device_errors())


def rmat_version() -> str:
    return lib().rmat_version().decode()


class Partition:
    """Owning handle of an ``rmat_partition``; keeps its table alive."""

    def __init__(self, handle, table):
        self._h = handle
        self._table = table

    @property
    def handle(self):
        if not self._h:
            raise ValueError("partition already freed")
        return self._h

    def free(self):
        if self._h:
            lib().rmat_free_partition(self._h)
            self._h = None
            self._table = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rmat_partition_create(t: Table, tile_levels: int, m: int, seed: int, row_tile_begin: int = 0,
                          row_tile_end=None) -> Partition:
    """Tiles of a depth-tile_levels partition of graph (t, m, seed) that meet
    the tile rows [row_tile_begin, row_tile_end) (Sec. 3 partitioned graphs)."""
    if row_tile_end is None:
        row_tile_end = 1 << tile_levels
    h = ctypes.c_void_p()
    check(lib().rmat_partition_create(t.handle, tile_levels, m, seed, row_tile_begin, row_tile_end, ctypes.byref(h)))
    return Partition(h, t)


def rmat_partition_info(p: Partition):
    n, e = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().rmat_partition_info(p.handle, ctypes.byref(n), ctypes.byref(e)))
    return n.value, e.value


def rmat_partition_tiles(p: Partition) -> dict:
    n, _ = rmat_partition_info(p)
    out = {f: np.zeros(max(n, 1), np.uint64) for f in ("row", "col", "count", "first")}
    check(lib().rmat_partition_tiles(p.handle, _ptr(out["row"]), _ptr(out["col"]), _ptr(out["count"]),
                                     _ptr(out["first"])))
    return {f: a[:n] for f, a in out.items()}


def rmat_generate_partition(p: Partition, out, stream=None) -> None:
    check(lib().rmat_generate_partition(p.handle, _ptr(out), _stream(stream)))


def rmat_free_partition(p: Partition) -> None:
    p.free()


def rmat_dedup_edges(edges, count: int, k: int, stream=None) -> int:
    """Remove repeated edges in place (first occurrences kept, order kept);
    returns how many remain at the front of `edges` (Sec. 3)."""
    n = ctypes.c_uint64()
    check(lib().rmat_dedup_edges(_ptr(edges), count, k, ctypes.byref(n), _stream(stream)))
    return n.value


def rmat_dedup_release() -> None:
    """Free the device scratch that rmat_dedup_edges keeps for later calls on
    the current device."""
    check(lib().rmat_dedup_release())


def rmat_selftest_bounded_wait(limit: int = 4096) -> None:
    """Run the failure-path self-test (a bounded device wait that runs out);
    raises RmatError(RMAT_ERR_TIMEOUT) as a real timeout would."""
    check(lib().rmat_selftest_bounded_wait(limit))
