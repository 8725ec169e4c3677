"""Autotuner: picks the table (variable-length bound or fixed path length l),
the per-level group length l, and the launch shape (threads per CTA, CTAs per
SM, edges per warp tile) by timing real launches on the current GPU.

The paper tunes the table size by hand per machine (Fig. 1: throughput
against table size; the best size tracks the cache hierarchy).  On GB300 the
table lives in shared memory, so the trade-off is levels per draw (larger
tables) against shared-memory footprint and staging cost; the tuner measures
it instead of modelling it.  Results are cached per device in a JSON file
(``$RMAT_TUNE_CACHE`` or ``~/.cache/rmat_gb300/``).

Everything here sits above the C ABI: it only builds tables, sets launch
shapes and times ``rmat_generate`` / ``rmat_batch_launch`` with CUDA events.
"""
from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

from . import (rmat_batch_add, rmat_batch_create, rmat_batch_launch, rmat_batch_prepare, rmat_build_table,
               rmat_build_table_fixed, rmat_build_table_levels, rmat_generate, rmat_set_launch_config,
               rmat_table_info, empty_edges)

LAUNCH_SHAPES = [(1024, 1, 512), (1024, 1, 256), (768, 1, 512), (512, 2, 512), (512, 1, 1024), (256, 4, 512)]
BOUNDS = [1 << b for b in range(8, 15)]
ELLS = [4, 5, 6, 7, 8]
# Shared memory the batched kernel keeps ahead of its staged table (its
# mbarrier, the current work unit and the job's 20 Philox round keys); the
# library's kBatchHeaderBytes.
BATCH_HEADER_BYTES = 96
_lock = threading.Lock()


def _cache_path() -> str:
    base = os.environ.get("RMAT_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "rmat_gb300")
    os.makedirs(base, exist_ok=True)
    import torch
    name = torch.cuda.get_device_name().replace(" ", "_")
    return os.path.join(base, f"tune_{name}.json")


def _load() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(key: str, value) -> None:
    with _lock:
        d = _load()
        d[key] = value
        tmp = _cache_path() + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, _cache_path())


def time_launches(fn, reps: int = 5, warmup: int = 2) -> float:
    """Median device time (s) of fn(stream) over `reps` back-to-back launches,
    each timed by its own pair of events: one slow launch (a clock ramping up,
    a neighbour on the GPU) cannot flip the choice between candidates whose
    rates differ by a few per cent."""
    import torch
    s = torch.cuda.Stream()
    for _ in range(warmup):
        fn(s)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(s)
        fn(s)
        b.record(s)
    s.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in ev])) / 1e3


def tune_launch(table, sample_edges: int = 1 << 26, shapes=LAUNCH_SHAPES, out=None, seed: int = 1):
    """Time `table` under each launch shape, keep the fastest (applied to the
    table with rmat_set_launch_config) and return (shape, edges_per_s)."""
    info = rmat_table_info(table)
    key = (f"launch:k{info['k']}:e{info['entries']}:b{info['bits']}:l{info['max_len']}:g{info['groups']}:"
           f"u{info['index_bytes']}:f{info['flags']}")
    cached = _load().get(key)
    if cached:
        rmat_set_launch_config(table, *cached["shape"])
        return tuple(cached["shape"]), cached["edges_per_s"]
    if out is None:
        out = empty_edges(sample_edges, info["k"])
    best = None
    for shape in shapes:
        rmat_set_launch_config(table, *shape)
        dt = time_launches(lambda s: rmat_generate(table, seed, 0, sample_edges, out, s))
        rate = sample_edges / dt
        if best is None or rate > best[1]:
            best = (shape, rate)
    rmat_set_launch_config(table, *best[0])
    _store(key, {"shape": list(best[0]), "edges_per_s": best[1]})
    return best


def _param_key(abcd) -> str:
    return ",".join(f"{x:.3f}" for x in abcd)


def tune_table(k: int, abcd, sample_edges: int = 1 << 24, bounds=BOUNDS, ells=ELLS, seed: int = 1,
               max_blob_bytes: int = 160 * 1024, batched: bool = False):
    """Fastest table for (k, a, b, c, d): a variable-length table with one of
    `bounds`, or a fixed-length table with one of `ells`, among those whose
    device blob is at most `max_blob_bytes` (what the launch can stage in
    shared memory).  batched: time each candidate in the batched kernel (a
    one-graph batch) instead of the single-graph kernel -- the two keep
    different numbers of edges in flight per lane, which can change the
    ranking.  Returns a dict {"kind": "variable"|"fixed", "bound"|"ell": ...,
    "edges_per_s": ...}."""
    key = f"table:k{k}:p{_param_key(abcd)}:s{max_blob_bytes}" + (":batched" if batched else "")
    cached = _load().get(key)
    if cached:
        return cached
    out = empty_edges(sample_edges, k)
    cands = [("variable", b) for b in bounds] + [("fixed", l) for l in ells if l <= k]
    best = None
    for kind, x in cands:
        t = rmat_build_table(*abcd, k, x) if kind == "variable" else rmat_build_table_fixed(*abcd, k, x)
        if rmat_table_info(t)["device_image_bytes"] > max_blob_bytes:
            continue  # would not fit shared memory beside the warp tiles
        if batched:
            b = rmat_batch_create()
            rmat_batch_add(b, t, seed, 0, sample_edges, out)
            rmat_batch_prepare(b)
            dt = time_launches(lambda s: rmat_batch_launch(b, s), reps=7)
            b.free()
        else:
            dt = time_launches(lambda s: rmat_generate(t, seed, 0, sample_edges, out, s))
        rate = sample_edges / dt
        if best is None or rate > best["edges_per_s"]:
            best = {"kind": kind, ("bound" if kind == "variable" else "ell"): x, "edges_per_s": rate}
    _store(key, best)
    return best


def tune_levels(k: int, P_levels, flags: int = 0, sample_edges: int = 1 << 24, ells=(3, 4, 5, 6, 7), seed: int = 1):
    """Fastest group length l for a per-level table (one table per l levels)."""
    P = np.asarray(P_levels, np.float64).reshape(-1, 4)
    key = f"levels:k{k}:f{flags}:p{_param_key(P.mean(axis=0))}"
    cached = _load().get(key)
    if cached:
        return cached
    out = empty_edges(sample_edges, k)
    best = None
    for ell in ells:
        if (k + ell - 1) // ell > 64:
            continue
        t = rmat_build_table_levels(P, k, ell, flags)
        if rmat_table_info(t)["device_image_bytes"] > 160 * 1024:
            continue
        dt = time_launches(lambda s: rmat_generate(t, seed, 0, sample_edges, out, s))
        rate = sample_edges / dt
        if best is None or rate > best["edges_per_s"]:
            best = {"ell": ell, "edges_per_s": rate}
    _store(key, best)
    return best


def tuned_table_spec(k: int, choice, m: int | None = None):
    """("variable", bound) or ("fixed", l): the table build_tuned_table makes
    for (k, choice) and a graph of m edges.  For a graph of m edges the table's
    blob is also kept below 1/8 of the graph's output bytes (staging a table
    costs about its own size in traffic per CTA)."""
    if choice["kind"] == "fixed":
        ell = min(choice["ell"], k)
        if m is not None:
            while ell > 2 and 8 * 4 ** ell > m:   # table bytes <= 1/8 of the output bytes
                ell -= 1
        return ("fixed", ell)
    bound = choice["bound"]
    if m is not None:
        while bound > 64 and 8 * bound > m:
            bound //= 2
    return ("variable", bound)


def build_tuned_table(k: int, abcd, m: int | None = None, choice=None):
    """Build the table the tuner picked for (k, params), sized for m edges
    (tuned_table_spec); the returned table carries its spec as `.spec`."""
    choice = choice or tune_table(k, abcd)
    spec = tuned_table_spec(k, choice, m)
    if spec[0] == "fixed":
        t = rmat_build_table_fixed(*abcd, k, spec[1])
    else:
        t = rmat_build_table(*abcd, k, spec[1])
    t.spec = spec
    return t


def batch_blob_budget(threads: int = 1024, tile: int = 512, u64: bool = False) -> int:
    """Shared memory the batched kernel has left for a staged table blob beside
    its default 512-edge tiles (a larger table would make a whole wave fall
    back to 256-edge tiles)."""
    import torch
    smem = torch.cuda.get_device_properties(torch.cuda.current_device()).shared_memory_per_block_optin
    per_warp = tile * (16 if u64 else 8) + 3 * tile
    return smem - BATCH_HEADER_BYTES - (threads // 32) * per_warp


def plan_batch(graphs, representative=None, sample_edges: int = 1 << 24):
    """Table choice for every graph of a batch: the tuner runs once per k on
    representative parameters (default: the mean of the graphs' parameters),
    timing the batched kernel itself on tables that it can stage in shared
    memory, then each graph gets a table of that kind sized for its edge
    count.  Returns the tables and the per-k choices."""
    P = np.asarray([g["abcd"] for g in graphs], np.float64)
    rep = tuple(float(x) for x in (representative if representative is not None else P.mean(axis=0)))
    rep = tuple(x / sum(rep) for x in rep)
    choices = {}
    tables = []
    for g in graphs:
        k = g["k"]
        if k not in choices:
            choices[k] = tune_table(k, rep, sample_edges=sample_edges, max_blob_bytes=batch_blob_budget(),
                                    batched=True)
        tables.append(build_tuned_table(k, g["abcd"], g["m"], choices[k]))
    return tables, choices


def tune_batch_shape(tables, counts, seeds, outs, shapes=((1024, 1, 256), (1024, 1, 128), (512, 2, 256),
                                                          (512, 2, 128), (768, 1, 256))):
    """Fastest launch shape of the batched kernel for this batch."""
    best = None
    for shape in shapes:
        b = rmat_batch_create()
        for t, m, s, o in zip(tables, counts, seeds, outs):
            rmat_batch_add(b, t, s, 0, m, o)
        rmat_batch_prepare(b, *shape)
        dt = time_launches(lambda s_: rmat_batch_launch(b, s_), reps=2)
        if best is None or dt < best[1]:
            best = (shape, dt)
        b.free()
    return best
