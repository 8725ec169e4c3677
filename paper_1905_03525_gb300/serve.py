"""Python side of the generation server: a thin wrapper over the C ABI
(rmat_server_*) and the replay of the served workload (Poisson arrivals,
latency percentiles).  All generation runs in librmat's worker thread and
kernels; this module only submits requests and reads their status."""
from __future__ import annotations

import ctypes
import json
import threading
import time

import numpy as np

from ._capi import (CHUNK_FN, RMAT_UNDIRECTED, Request, RequestStatus, RmatError, ServerConfig, ServerStats, check,
                    lib)
from .workloads import served_trace

QUEUED, RUNNING, DONE, FAILED = 0, 1, 2, 3


class Server:
    """A librmat generation server on the current CUDA device."""

    def __init__(self, hbm_budget_bytes: int, chunk_edges: int = 1 << 28, step_edges: int = 1 << 31,
                 max_active: int = 64, wait_timeout_s: float = 120.0, gpu_build_min_bound: int = 1 << 14):
        """gpu_build_min_bound: requests with an explicit table bound at least
        this large get their table built on the GPU by the server's builder
        thread (0: every table is built on the host when submitted)."""
        cfg = ServerConfig(hbm_budget_bytes, chunk_edges, max(step_edges, chunk_edges), max_active, wait_timeout_s,
                           gpu_build_min_bound)
        h = ctypes.c_void_p()
        check(lib().rmat_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._cb = None

    def set_chunk_callback(self, fn):
        """fn(request_id, edge_offset, count, device_ptr) on the worker thread."""
        if fn is None:
            self._cb = None
            check(lib().rmat_server_set_chunk_callback(self._h, None, None))
            return
        self._cb = CHUNK_FN(lambda user, rid, off, cnt, ptr: fn(rid, off, cnt, ptr))
        check(lib().rmat_server_set_chunk_callback(self._h, self._cb, None))

    def submit(self, a, b, c, d, k, m, seed, table_bound=0, flags=0, scramble_seed=None) -> int:
        """Queue edges 0..m-1 of one graph; scramble_seed (not None) relabels
        its vertices as rmat_table_set_scramble does."""
        req = Request(a, b, c, d, k, m, seed, table_bound, flags, int(scramble_seed is not None),
                      scramble_seed or 0)
        rid = ctypes.c_uint64()
        check(lib().rmat_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid)))
        return rid.value

    def status(self, rid: int) -> dict:
        st = RequestStatus()
        check(lib().rmat_server_status(self._h, rid, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in RequestStatus._fields_}

    def wait(self, rid: int, timeout_s: float = 600.0) -> dict:
        st = RequestStatus()
        check(lib().rmat_server_wait(self._h, rid, timeout_s, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in RequestStatus._fields_}

    def drain(self, timeout_s: float = 3600.0) -> None:
        check(lib().rmat_server_drain(self._h, timeout_s))

    def stats(self) -> dict:
        st = ServerStats()
        check(lib().rmat_server_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self) -> None:
        if self._h:
            lib().rmat_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_trace(server: Server, trace, submitters: int = 8, table_bound: int = 0):
    """Submit every request of `trace` at its arrival time (seconds after the
    start), wait for all, and return per-request records."""
    ids = [None] * len(trace)
    t0 = time.perf_counter()
    clock0 = server.stats()["clock_s"]
    nxt = [0]
    lock = threading.Lock()

    def submitter():
        while True:
            with lock:
                i = nxt[0]
                nxt[0] += 1
            if i >= len(trace):
                return
            r = trace[i]
            delay = r["arrival"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids[i] = server.submit(*r["abcd"], r["k"], r["m"], r["seed"], table_bound)

    threads = [threading.Thread(target=submitter) for _ in range(submitters)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    server.drain()
    out = []
    for r, rid in zip(trace, ids):
        st = server.status(rid)
        out.append({**r, "id": rid, "state": st["state"], "checksum": st["checksum"], "table_bound": st["table_bound"],
                    "latency_s": st["done_s"] - st["submit_s"], "queue_s": st["admit_s"] - st["submit_s"],
                    "submit_s": st["submit_s"] - clock0, "done_s": st["done_s"] - clock0})
    return out


def summarise(records) -> dict:
    lat = np.array([r["latency_s"] for r in records])
    edges = sum(r["m"] for r in records)
    span = max(r["done_s"] for r in records) - min(r["submit_s"] for r in records)
    return {"requests": len(records), "edges": edges, "edges_per_s": edges / span, "span_s": span,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_queue_s": float(np.mean([r["queue_s"] for r in records])),
            "failed": sum(r["state"] != DONE for r in records)}


def bench(args) -> None:
    """Served workload: Poisson arrivals of requests with k ~ U{12..30}, edge
    factor in {4, 8, 16, 32}, Dirichlet(57,19,19,5) parameters, admitted by a
    160 GB device-memory budget, 2^28-edge chunks.  Reports the trace at the
    given rate and at a rate the GPU sustains."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    budget = min(160 * 10 ** 9, int(free * 0.8))
    lines = []
    with Server(budget, chunk_edges=1 << 28, step_edges=1 << 31, max_active=64) as srv:
        # warm-up: one small request compiles nothing but touches every path
        srv.wait(srv.submit(0.57, 0.19, 0.19, 0.05, 16, 1 << 20, 1))
        trace = served_trace(args.requests, rate=args.rate)
        rec = run_trace(srv, trace)
        s1 = summarise(rec)
        cap = s1["edges_per_s"]
        mean_m = float(np.mean([r["m"] for r in trace]))
        sustain = 0.7 * cap / mean_m
        trace2 = served_trace(args.requests, rate=sustain, seed=2001)
        s2 = summarise(run_trace(srv, trace2))
        st = srv.stats()
    # the same offered trace with one request on the GPU at a time (FIFO, one
    # graph per launch, same chunks and consumer): what continuous batching
    # is measured against
    with Server(budget, chunk_edges=1 << 28, step_edges=1 << 31, max_active=1) as fifo:
        fifo.wait(fifo.submit(0.57, 0.19, 0.19, 0.05, 16, 1 << 20, 1))
        s3 = summarise(run_trace(fifo, trace))
    line = {"workload": "c5", "config": {"workload": "served: Poisson arrivals, k~U{12..30}, ef in {4,8,16,32}, "
                                          "m=ef*2^k, (a,b,c,d)~Dirichlet(57,19,19,5), 2^28-edge chunks",
                                          "hbm_budget_bytes": budget, "max_active": 64, "step_edges": 1 << 31},
            "metric": "edges/s", "value": s1["edges_per_s"], "offered": {"rate_per_s": args.rate, **s1},
            "sustainable": {"rate_per_s": sustain, **s2},
            "fifo_one_request_at_a_time": {"rate_per_s": args.rate, **s3},
            "speedup_vs_fifo": s1["edges_per_s"] / s3["edges_per_s"], "server_steps": st["steps"]}
    print(json.dumps(line), flush=True)
