"""Scalar CPU oracle for the alias-path R-MAT generator (arXiv 1905.03525).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` are the only users.  The product package
never imports this module, and this module never imports the product package.

The C source (``rmat_oracle.c``) restates the paper's table construction
(Sec. 2, table-construction fragment), Walker's alias method (Sec. 2), the
sampling loop (Sec. 2, sampling-loop fragment), undirected mirroring,
scrambling and partitioned graphs (Sec. 3) and the naive per-bit R-MAT
process (Sec. 1), plus Philox4x32-10 (Salmon et al., SC'11) and binomial
sampling (inversion; BTRS, Hoermann 1993).  This file only compiles it with gcc and marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmat_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "librmat_oracle.so")

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/librmat_oracle.so`` (plain gcc,
    no fast-math, no FMA contraction) and return the library path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(os.path.join(_HERE, "rmat_oracle.h")))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load(path: str):
    """Load an oracle shared library and declare its functions."""
    L = ctypes.CDLL(path)
    _declare(L)
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def _declare(L):
    """Argument and result types of the oracle's C functions."""
    u32, u64, i32, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    vp = ctypes.c_void_p
    L.orc_philox4x32_10.argtypes = [vp, vp, vp]
    L.orc_word.argtypes = [u64, u64, u64]
    L.orc_word.restype = u32
    L.orc_table_variable.argtypes = [dbl, dbl, dbl, dbl, i32, u64]
    L.orc_table_variable.restype = vp
    L.orc_table_fixed.argtypes = [vp, i32]
    L.orc_table_fixed.restype = vp
    L.orc_table_free.argtypes = [vp]
    for name in ("orc_table_entries", "orc_table_bits", "orc_table_max_len"):
        getattr(L, name).argtypes = [vp]
        getattr(L, name).restype = i32
    L.orc_table_get.argtypes = [vp] * 7
    L.orc_draw.argtypes = [vp, u32]
    L.orc_draw.restype = u32
    L.orc_generate.argtypes = [vp, i32, i32, i32, u64, u64, u64, vp, vp]
    L.orc_generate.restype = i32
    L.orc_generate_naive.argtypes = [vp, i32, i32, u64, u64, u64, vp, vp]
    L.orc_generate_naive.restype = i32
    L.orc_edge_distribution.argtypes = [vp, i32, i32, i32, vp]
    L.orc_edge_distribution.restype = i32
    L.orc_scramble_constants.argtypes = [u64, i32, vp]
    L.orc_scramble.argtypes = [u64, i32, vp]
    L.orc_scramble.restype = u64
    L.orc_generate_scrambled.argtypes = [vp, i32, i32, i32, vp, u64, u64, u64, vp, vp]
    L.orc_generate_scrambled.restype = i32
    L.orc_kron_table_variable.argtypes = [vp, i32, i32, u64]
    L.orc_kron_table_variable.restype = vp
    L.orc_kron_table_fixed.argtypes = [vp, i32, i32]
    L.orc_kron_table_fixed.restype = vp
    L.orc_kron_table_free.argtypes = [vp]
    for name in ("orc_kron_table_entries", "orc_kron_table_bits", "orc_kron_table_max_len"):
        getattr(L, name).argtypes = [vp]
        getattr(L, name).restype = i32
    L.orc_kron_table_get.argtypes = [vp] * 7
    L.orc_kron_draw.argtypes = [vp, u32]
    L.orc_kron_draw.restype = u32
    L.orc_kron_generate.argtypes = [vp, i32, u64, u64, u64, vp, vp]
    L.orc_kron_generate.restype = i32
    L.orc_kron_edge_distribution.argtypes = [vp, i32, i32, vp]
    L.orc_kron_edge_distribution.restype = i32
    L.orc_partition_word.argtypes = [u64, i32, u64, i32, u64]
    L.orc_partition_word.restype = u32
    L.orc_binomial.argtypes = [u64, dbl, u64, i32, u64, i32]
    L.orc_binomial.restype = u64
    L.orc_partition.argtypes = [dbl, dbl, dbl, dbl, i32, u64, u64, u64, u64, u64, vp, vp, vp, vp]
    L.orc_partition.restype = ctypes.c_int64
    L.orc_generate_tile.argtypes = [vp, i32, i32, u64, u64, u64, u64, u64, vp, vp]
    L.orc_generate_tile.restype = i32


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def word(seed: int, e: int, n: int) -> int:
    return int(lib().orc_word(seed, e, n))


class Table:
    """One oracle alias table (a single table, or one level group)."""

    def __init__(self, handle):
        if not handle:
            raise ValueError("oracle rejected the table arguments")
        self._h = ctypes.c_void_p(handle)
        L = lib()
        self.entries = L.orc_table_entries(self._h)
        self.bits = L.orc_table_bits(self._h)
        self.max_len = L.orc_table_max_len(self._h)
        N = 1 << self.bits
        self.sym = np.zeros(N, np.uint64)
        self.len = np.zeros(N, np.uint8)
        self.p = np.zeros(N, np.float64)
        self.w = np.zeros(N, np.uint64)
        self.thr = np.zeros(N, np.uint32)
        self.alias = np.zeros(N, np.uint32)
        L.orc_table_get(self._h, _ptr(self.sym), _ptr(self.len), _ptr(self.p), _ptr(self.w),
                        _ptr(self.thr), _ptr(self.alias))

    @classmethod
    def variable(cls, a, b, c, d, k, bound):
        return cls(lib().orc_table_variable(a, b, c, d, k, bound))

    @classmethod
    def fixed(cls, P, ell=None):
        P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1, 4)
        if ell is None:
            ell = P.shape[0]
        if P.shape[0] == 1 and ell > 1:
            P = np.repeat(P, ell, axis=0)
        return cls(lib().orc_table_fixed(_ptr(P), ell))

    def draw(self, u: int) -> int:
        return int(lib().orc_draw(self._h, u))

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().orc_table_free(self._h)
                self._h = None
        except Exception:
            pass


def _handles(tables):
    arr = (ctypes.c_void_p * len(tables))(*[t._h.value for t in tables])
    return arr


def generate(tables, k, seed, e0, count, undirected=False):
    """Edges e0 .. e0+count-1 as (row, col) uint64 arrays."""
    tables = list(tables)
    row = np.zeros(count, np.uint64)
    col = np.zeros(count, np.uint64)
    h = _handles(tables)
    rc = lib().orc_generate(h, len(tables), k, int(undirected), seed, e0, count, _ptr(row), _ptr(col))
    if rc != 0:
        raise ValueError("oracle rejected the generate arguments")
    return row, col


def generate_parallel(tables, k, seed, e0, count, undirected=False, threads=None):
    """generate() split over host threads, each taking one consecutive run of
    the edge range.  Edge e depends only on the tables, the seed and e (the
    counter-based stream), so the split changes nothing but the wall time."""
    tables = list(tables)
    threads = max(1, min(threads or os.cpu_count() or 1, count // 4096 or 1))
    row = np.zeros(count, np.uint64)
    col = np.zeros(count, np.uint64)
    h = _handles(tables)
    per = (count + threads - 1) // threads
    rcs = [0] * threads

    def work(i):
        lo = i * per
        n = max(0, min(count, lo + per) - lo)
        if n:
            rcs[i] = lib().orc_generate(h, len(tables), k, int(undirected), seed, e0 + lo, n,
                                        row[lo:].ctypes.data_as(ctypes.c_void_p),
                                        col[lo:].ctypes.data_as(ctypes.c_void_p))

    lib()
    ts = [threading.Thread(target=work, args=(i,)) for i in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if any(rcs):
        raise ValueError("oracle rejected the generate arguments")
    return row, col


def scramble_constants(scramble_seed: int, k: int) -> np.ndarray:
    out = np.zeros(6, np.uint64)
    lib().orc_scramble_constants(scramble_seed, k, _ptr(out))
    return out


def scramble(x: int, k: int, consts) -> int:
    c = np.ascontiguousarray(consts, dtype=np.uint64)
    return int(lib().orc_scramble(x, k, _ptr(c)))


def generate_scrambled(tables, k, scramble_seed, seed, e0, count, undirected=False):
    """orc_generate followed by the vertex relabelling of scramble_seed."""
    tables = list(tables)
    consts = scramble_constants(scramble_seed, k)
    row = np.zeros(count, np.uint64)
    col = np.zeros(count, np.uint64)
    rc = lib().orc_generate_scrambled(_handles(tables), len(tables), k, int(undirected), _ptr(consts), seed, e0,
                                      count, _ptr(row), _ptr(col))
    if rc != 0:
        raise ValueError("oracle rejected the generate arguments")
    return row, col


class KronTable:
    """Oracle table of a stochastic Kronecker graph with an n0 x n0 initiator."""

    def __init__(self, handle, n0):
        if not handle:
            raise ValueError("oracle rejected the Kronecker table arguments")
        self._h = ctypes.c_void_p(handle)
        self.n0 = n0
        L = lib()
        self.entries = L.orc_kron_table_entries(self._h)
        self.bits = L.orc_kron_table_bits(self._h)
        self.max_len = L.orc_kron_table_max_len(self._h)
        N = 1 << self.bits
        self.sym = np.zeros((N, max(self.max_len, 1)), np.uint8)
        self.len = np.zeros(N, np.uint8)
        self.p = np.zeros(N, np.float64)
        self.w = np.zeros(N, np.uint64)
        self.thr = np.zeros(N, np.uint32)
        self.alias = np.zeros(N, np.uint32)
        L.orc_kron_table_get(self._h, _ptr(self.sym), _ptr(self.len), _ptr(self.p), _ptr(self.w),
                             _ptr(self.thr), _ptr(self.alias))

    @classmethod
    def variable(cls, theta, n0, k, bound):
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(n0 * n0)
        return cls(lib().orc_kron_table_variable(_ptr(th), n0, k, bound), n0)

    @classmethod
    def fixed(cls, theta, n0, ell):
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(n0 * n0)
        return cls(lib().orc_kron_table_fixed(_ptr(th), n0, ell), n0)

    def draw(self, u: int) -> int:
        return int(lib().orc_kron_draw(self._h, u))

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().orc_kron_table_free(self._h)
                self._h = None
        except Exception:
            pass


def kron_generate(table, k, seed, e0, count):
    row = np.zeros(count, np.uint64)
    col = np.zeros(count, np.uint64)
    if lib().orc_kron_generate(table._h, k, seed, e0, count, _ptr(row), _ptr(col)) != 0:
        raise ValueError("oracle rejected the Kronecker generate arguments")
    return row, col


def kron_edge_distribution(table, k, quantised=False) -> np.ndarray:
    nv = table.n0 ** k
    out = np.zeros(nv * nv, np.float64)
    if lib().orc_kron_edge_distribution(table._h, k, int(quantised), _ptr(out)) != 0:
        raise ValueError("oracle rejected the distribution arguments")
    return out.reshape(nv, nv)


def partition_word(seed, depth, node, j, n) -> int:
    return int(lib().orc_partition_word(seed, depth, node, j, n))


def binomial(n, p, seed, depth, node, j) -> int:
    return int(lib().orc_binomial(n, p, seed, depth, node, j))


def partition(abcd, t, m, seed, row_tile_begin=0, row_tile_end=None):
    """Non-empty tiles of a depth-t partition meeting the tile rows
    [row_tile_begin, row_tile_end): dict of uint64 arrays row, col, count,
    first (quadtree order)."""
    if row_tile_end is None:
        row_tile_end = 1 << t
    L = lib()
    n = L.orc_partition(*abcd, t, m, seed, row_tile_begin, row_tile_end, 0, None, None, None, None)
    if n < 0:
        raise ValueError("oracle rejected the partition arguments")
    out = {f: np.zeros(max(n, 1), np.uint64) for f in ("row", "col", "count", "first")}
    n2 = L.orc_partition(*abcd, t, m, seed, row_tile_begin, row_tile_end, n, _ptr(out["row"]), _ptr(out["col"]),
                         _ptr(out["count"]), _ptr(out["first"]))
    assert n2 == n
    return {f: a[:n] for f, a in out.items()}


def generate_tile(table, k, t, tile_row, tile_col, seed, first, count):
    row = np.zeros(count, np.uint64)
    col = np.zeros(count, np.uint64)
    rc = lib().orc_generate_tile(table._h, k, t, tile_row, tile_col, seed, first, count, _ptr(row), _ptr(col))
    if rc != 0:
        raise ValueError("oracle rejected the tile arguments")
    return row, col


def generate_partitioned(table, abcd, k, t, m, seed, row_tile_begin=0, row_tile_end=None):
    """The tiles of partition() and their edges, concatenated in tile order."""
    tiles = partition(abcd, t, m, seed, row_tile_begin, row_tile_end)
    rows, cols = [], []
    for R, C, n, f in zip(tiles["row"], tiles["col"], tiles["count"], tiles["first"]):
        r, c = generate_tile(table, k, t, int(R), int(C), seed, int(f), int(n))
        rows.append(r)
        cols.append(c)
    if not rows:
        return tiles, (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    return tiles, (np.concatenate(rows), np.concatenate(cols))


def dedup_first(row, col):
    """Duplicate removal (Sec. 3, partitioned graphs): the first occurrence of
    every (row, col) in array order, in that order.  IDs below 2^32."""
    r = np.asarray(row, np.uint64)
    c = np.asarray(col, np.uint64)
    if len(r) and (int(r.max()) >> 32 or int(c.max()) >> 32):
        raise ValueError("dedup_first takes IDs below 2^32")
    _, first = np.unique((r << np.uint64(32)) | c, return_index=True)
    keep = np.sort(first)
    return r[keep], c[keep]


def generate_naive(P_levels, k, seed, e0, count, undirected=False):
    P = np.ascontiguousarray(P_levels, dtype=np.float64).reshape(-1, 4)
    if P.shape[0] == 1:
        P = np.repeat(P, k, axis=0)
    row = np.zeros(count, np.uint64)
    col = np.zeros(count, np.uint64)
    rc = lib().orc_generate_naive(_ptr(P), k, int(undirected), seed, e0, count, _ptr(row), _ptr(col))
    if rc != 0:
        raise ValueError("oracle rejected the naive arguments")
    return row, col


def edge_distribution(tables, k, quantised=False) -> np.ndarray:
    """Exact P(row, col) as a 2^k x 2^k array."""
    tables = list(tables)
    out = np.zeros((1 << k) * (1 << k), np.float64)
    rc = lib().orc_edge_distribution(_handles(tables), len(tables), k, int(quantised), _ptr(out))
    if rc != 0:
        raise ValueError("oracle rejected the distribution arguments")
    return out.reshape(1 << k, 1 << k)


def level_groups(P_levels, k, ell):
    """Fixed-length tables for consecutive groups of ell levels (the last group
    holds the remaining k mod ell levels), level t using P_levels[t]."""
    P = np.ascontiguousarray(P_levels, dtype=np.float64).reshape(-1, 4)
    if P.shape[0] == 1:
        P = np.repeat(P, k, axis=0)
    tables = []
    for g0 in range(0, k, ell):
        n = min(ell, k - g0)
        tables.append(Table.fixed(P[g0:g0 + n], n))
    return tables
