#!/usr/bin/env python3
"""Benchmark: R-MAT edges/s on GB300 and the fraction of the HBM-write roofline.

Default workload (one step = one pass of the whole sampling path over one
graph): k = 26 (n = 2^26), m = 2^30 edges (edge factor 16), Graph 500
parameters a, b, c, d = 0.57, 0.19, 0.19, 0.05, variable-length table with
bound 2^12 (4093 entries), Philox seed 1, uint32 (row, col) pairs -- 8 GiB of
output per step, far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun, one rank per GPU) every rank generates its
own 2^30-edge range of one 2^30*N-edge graph (weak scaling; ranges are
independent, no collective on the data path).  `--impl reference` times the
CPU oracle on the host cores instead (bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

K, LOG2M, BOUND, SEED = 26, 30, 4096, 1
G500 = (0.57, 0.19, 0.19, 0.05)
METRIC = "R-MAT edges/s on 1 GB300, % of HBM-write roofline; batched vs per-graph launches"
WORKLOAD = ("R-MAT k=26 (n=2^26), m=2^30 edges (edge factor 16), a,b,c,d=0.57,0.19,0.19,0.05, "
            "variable-length similar-probability paths, table bound 2^12 (4093 entries), "
            "Philox4x32-10 seed=1, u32 (row,col) pairs")
FALLBACK_HBM_GBS = 6800.0
# DRAM traffic of the timed kernel (k_alias_fast) per 2^30-edge launch: the
# read + write bytes of one m=2^28 launch (`ncu --metrics dram__bytes_read.sum,
# dram__bytes_write.sum`, 1 pass, profiles/k_alias_fast_k26_m2p28_traffic.md)
# scaled by the edges (x4); valid only for the kernel sources whose hash is
# recorded with it.
TRAFFIC = {"kernel_sha256_16": "e2a6c8914b67d5b0", "bytes_per_launch": 4 * (123904 + 2086040064),
           "source": "m=2^28 capture scaled x4 (profiles/k_alias_fast_k26_m2p28_traffic.md)"}
# Warp instructions per edge of the same kernel (smsp__inst_executed.sum and
# smsp__inst_executed_pipe_alu.sum / 2^26 on an m=2^26 capture of this workload,
# `ncu --metrics ... -k regex:k_alias_fast -s 3 -c 1`), valid for the same hash.
INSTR = {"kernel_sha256_16": "e2a6c8914b67d5b0", "warp_instr_per_edge": 293341562 / 2 ** 26,
         "alu_warp_instr_per_edge": 149171022 / 2 ** 26}
KERNEL_SOURCES = ("paper_1905_03525_gb300/csrc/rmat_device.cuh", "paper_1905_03525_gb300/csrc/rmat_kernels.cu")


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def issue_roofline(edges_per_s: float, sm_mhz: float):
    """The bound the kernel actually meets: its integer pipes.  The ALU pipe
    (16 lanes per scheduler: half a warp instruction per clock, measured on
    this GPU) carries the most work; `frac` is the achieved ALU warp
    instructions per second against SMs x 4 schedulers x 0.5 x the SM clock
    sampled in the run.  `issue_frac` compares all instructions with one per
    scheduler per clock.  `roofline` stays the HBM-write fraction that the
    metric names."""
    import torch
    if INSTR["kernel_sha256_16"] != kernel_hash() or not INSTR["warp_instr_per_edge"] or not sm_mhz:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    issue_peak = sms * 4 * sm_mhz * 1e6
    alu = edges_per_s * INSTR["alu_warp_instr_per_edge"]
    return {"bound": "alu", "achieved": alu, "peak": 0.5 * issue_peak, "unit": "ALU warp-instr/s",
            "frac": alu / (0.5 * issue_peak), "issue_frac": edges_per_s * INSTR["warp_instr_per_edge"] / issue_peak,
            "warp_instr_per_edge": INSTR["warp_instr_per_edge"],
            "alu_warp_instr_per_edge": INSTR["alu_warp_instr_per_edge"],
            "source": "smsp__inst_executed(_pipe_alu).sum of m=2^26 ncu captures of the same kernel sources; "
                      "peak = SMs x 4 schedulers x 0.5 ALU instr/clock x median SM clock of this run"}


def measured_traffic(log2m: int):
    if kernel_hash() != TRAFFIC["kernel_sha256_16"] or log2m != LOG2M:
        return None  # kernel changed since the counters were taken
    return TRAFFIC["bytes_per_launch"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mix", action="store_true", help="c2: leave out the batched and served measurements")
    ap.add_argument("--cpu-sample-edges", type=int, default=1 << 30)
    ap.add_argument("--workload", choices=["c2", "c1", "c3", "c4", "c5", "part", "kron", "tablebuild", "fig1"],
                    default="c2",
                    help="c2 (default): the contract line; c1/c3/c4/c5: the other configurations, one JSON line each")
    ap.add_argument("--log2m", type=int, default=LOG2M,
                    help="c2: edges per GPU = 2^log2m (default 30; smaller only for profiling captures); "
                         "c3: chunk size; part, kron: edges; fig1: edges per launch (at most 2^28)")
    ap.add_argument("--graphs", type=int, default=4096, help="c4: number of graphs")
    ap.add_argument("--tile-levels", type=int, default=5, help="part: tiles of 2^(k-t) x 2^(k-t) vertices")
    ap.add_argument("--wave-gib", type=float, default=48.0, help="c4: output budget per batched launch")
    ap.add_argument("--requests", type=int, default=256, help="c5: trace length")
    ap.add_argument("--rate", type=float, default=2000.0, help="c5: mean arrivals per second")
    return ap.parse_args()


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self._t.join(timeout=2)

    def summary(self):
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons),
                "samples": len(sms)}


def cpu_baseline(total_edges: int):
    """The oracle, as it stands, over a bounded sample of the workload on all
    host cores (one thread per core, each generating consecutive edge ranges)."""
    import numpy as np
    import oracle
    cores = os.cpu_count() or 1
    t = oracle.Table.variable(*G500, K, BOUND)
    per = (total_edges + cores - 1) // cores
    chunk = 1 << 20

    def work(c):
        lo = c * per
        hi = min(total_edges, lo + per)
        L = oracle.lib()
        row = np.zeros(chunk, np.uint64)
        col = np.zeros(chunk, np.uint64)
        h = oracle._handles([t])
        e = lo
        while e < hi:
            n = min(chunk, hi - e)
            L.orc_generate(h, 1, K, 0, SEED, e, n, row.ctypes.data, col.ctypes.data)
            e += n

    threads = [threading.Thread(target=work, args=(c,)) for c in range(cores)]
    t0 = time.perf_counter()
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    dt = time.perf_counter() - t0
    return {"value": total_edges / dt, "unit": "edges/s", "cores": cores, "kind": "oracle", "seconds": dt,
            "sample": f"edges 0..{total_edges - 1} of the same graph (k=26, bound 2^12, seed 1), "
                      f"{cores} threads, {dt:.1f} s wall"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.cpu_sample_edges
    vals = []
    for _ in range(max(0, args.warmup)):
        cpu_baseline(n // 8)
    for _ in range(max(1, args.steps)):
        vals.append(cpu_baseline(n // max(1, args.steps)))
    v = statistics.median([x["value"] for x in vals])
    step_ms = 1e3 * statistics.median([x.pop("seconds") for x in vals])
    cb = dict(vals[-1])
    cb["value"] = v
    cb["sample"] = f"{args.steps} steps of {n // max(1, args.steps)} edges each: " + cb["sample"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "edges/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "k": K, "m": 1 << LOG2M, "table_bound": BOUND},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "edges/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_1905_03525_gb300 as rm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1905_03525_gb300.sharding import weak_range
    e0, m = weak_range(rank, 1 << args.log2m)
    table = rm.rmat_build_table(*G500, K, BOUND)
    rm.rmat_table_upload(table)
    out = rm.empty_edges(m, K)
    stream = torch.cuda.Stream()

    for _ in range(max(3, args.warmup)):
        rm.rmat_generate(table, SEED, e0, m, out, stream)
    stream.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_begin = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_begin.record(stream)
        for i in range(args.steps):
            starts[i].record(stream)
            rm.rmat_generate(table, SEED, e0, m, out, stream)
            ends[i].record(stream)
        t_end.record(stream)
        stream.synchronize()
    barrier()
    torch.cuda.synchronize()
    total_ms = t_begin.elapsed_time(t_end)
    per_launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * m * args.steps / (total_ms / 1e3)

    # roofline of the (only) kernel: algorithmic bytes = 8 B per edge written
    peak, peak_src = measured_peak()
    avg_launch_s = statistics.mean(per_launch_ms) / 1e3
    achieved = 8.0 * m / avg_launch_s / 1e9
    rm.rmat_check_device_errors()

    # comparator: the naive per-bit kernel (k quadrant draws per edge) on the same workload
    naive_s = _events_time(lambda: rm.rmat_generate_naive(G500, K, 0, SEED, e0, m, out, stream), stream, 2)
    # the same launch with scrambled vertex IDs (the relabelling fused into the store)
    scr_table = rm.rmat_build_table(*G500, K, BOUND)
    rm.rmat_table_set_scramble(scr_table, True, SEED)
    rm.rmat_generate(scr_table, SEED, e0, m, out, stream)
    scr_s = _events_time(lambda: rm.rmat_generate(scr_table, SEED, e0, m, out, stream), stream, 3)
    # restore this step's output of the alias kernel
    rm.rmat_generate(table, SEED, e0, m, out, stream)
    stream.synchronize()

    # end to end through the public host-buffer call: table built and uploaded
    # every step (h2d), all edges copied back into pinned host memory (d2h).
    e2e = None
    if not args.no_e2e:
        host = rm.empty_edges(m, K, device="cpu", pin_memory=True)
        img_bytes = rm.rmat_table_info(table)["device_image_bytes"]
        rm.rmat_generate_host(table, SEED, e0, m, host, stream)  # warm the staging area
        barrier()
        times = []
        for _ in range(max(1, min(args.steps, 3))):
            t0 = time.perf_counter()
            tb = rm.rmat_build_table(*G500, K, BOUND)
            rm.rmat_table_upload(tb)
            rm.rmat_generate_host(tb, SEED, e0, m, host, stream)
            times.append(time.perf_counter() - t0)
            tb.free()
        tt = torch.tensor([statistics.median(times)], dtype=torch.float64, device="cuda")
        if dist is not None:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e = {"value": world * m / float(tt.item()), "unit": "edges/s", "h2d_bytes_per_step": int(img_bytes),
               "d2h_bytes_per_step": int(8 * m), "steps": len(times),
               "path": "rmat_build_table + rmat_table_upload + rmat_generate_host into pinned host memory"}
        del host

    # the metric's second half: batched and served generation on this GPU
    batched = served = None
    if world == 1 and not args.no_mix:
        batched = measure_batched()
        served = measure_served()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cb = None
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(args.cpu_sample_edges)
        cb.pop("seconds")
    cs = clocks.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "k": K, "m_per_gpu": m, "table_bound": BOUND, "seed": SEED,
                   "l2": "no flush: each step writes 8 GiB, far larger than the 126 MiB L2",
                   "parallelism": f"edge-range sharding x{world}, no collective"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": measured_traffic(args.log2m), "traffic_source": TRAFFIC["source"],
                     "kernel": "k_alias_fast", "peak_source": f"{peak_src} hbm_gbs (copy)",
                     "algorithmic_bytes_per_launch": 8 * m, "avg_launch_ms": avg_launch_s * 1e3},
        "issue_roofline": issue_roofline(m / avg_launch_s, cs["sm_mhz"]),
        "cpu_baseline": cb,
        "comparators": {"naive_per_bit_gpu": {"value": world * m / naive_s, "unit": "edges/s",
                                              "note": "k Philox words and quadrant draws per edge, same GPU"},
                        "scrambled_ids": {"value": world * m / scr_s, "unit": "edges/s",
                                          "overhead_ns_per_edge": (scr_s - avg_launch_s) / m * 1e9,
                                          "note": "same launch with rmat_table_set_scramble on"}},
        "e2e": e2e,
        "batched": batched,
        "served": served,
        "gpu_launches": args.steps,
        "clocks": {"sm_mhz": cs["sm_mhz"], "sm_max_mhz": cs["sm_max_mhz"], "reasons": cs["reasons"]},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _events_time(fn, stream, reps):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


def run_c1(args):
    """k=16, m=2^20, fixed l=4 (256-entry table), seed 1: one launch per step."""
    import torch
    import paper_1905_03525_gb300 as rm
    k, m = 16, 1 << 20
    t = rm.rmat_build_table_fixed(*G500, k, 4)
    rm.rmat_table_upload(t)
    out = rm.empty_edges(m, k)
    s = torch.cuda.Stream()
    for _ in range(max(3, args.warmup)):
        rm.rmat_generate(t, 1, 0, m, out, s)
    dt = _events_time(lambda: rm.rmat_generate(t, 1, 0, m, out, s), s, max(args.steps, 50))
    # the same launch replayed from a CUDA graph (no host launch cost)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(20):
            rm.rmat_generate(t, 1, 0, m, out, s)
    with torch.cuda.stream(s):
        g.replay()
        dtg = _events_time(g.replay, s, 5) / 20
    print(json.dumps({"workload": "c1", "config": {"workload": "R-MAT k=16, m=2^20, fixed l=4 (256 entries), "
                      "a,b,c,d=0.57,0.19,0.19,0.05, seed=1, u32"}, "metric": "edges/s", "value": m / dt,
                      "ms_per_launch": dt * 1e3, "graph_replay_edges_per_s": m / dtg,
                      "graph_replay_us_per_launch": dtg * 1e6, "hbm_gbs": 8 * m / dtg / 1e9}), flush=True)


def run_c3(args):
    """k=34, m=2^35 in 32 chunks of 2^30 edges, u64 pairs, undirected, per-level
    noisy parameters, one table per level group (group length tuned)."""
    import torch
    import paper_1905_03525_gb300 as rm
    from paper_1905_03525_gb300 import autotune
    from paper_1905_03525_gb300.workloads import noisy_levels
    k, chunk, nchunks = 34, 1 << min(args.log2m, 30), 32  # smaller chunks only for profiling captures
    P = noisy_levels(k)
    choice = autotune.tune_levels(k, P, rm.RMAT_UNDIRECTED)
    t = rm.rmat_build_table_levels(P, k, choice["ell"], rm.RMAT_UNDIRECTED)
    shape, _ = autotune.tune_launch(t, sample_edges=1 << 26)
    out = rm.empty_edges(chunk, k)
    s = torch.cuda.Stream()
    for _ in range(max(3, args.warmup)):
        rm.rmat_generate(t, 34, 0, chunk, out, s)
    s.synchronize()
    with ClockSampler(0) as clocks:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        for c in range(nchunks):
            rm.rmat_generate(t, 34, c * chunk, chunk, out, s)
        b.record(s)
        s.synchronize()
    dt = a.elapsed_time(b) / 1e3
    peak, src = measured_peak()
    gbs = 16.0 * chunk * nchunks / dt / 1e9
    lc = chunk.bit_length() - 1
    print(json.dumps({"workload": "c3", "config": {"workload": f"R-MAT k=34, m=2^{lc + 5} streamed in 32 chunks of "
                      f"2^{lc} edges into one {16 * chunk >> 30} GiB buffer, u64 pairs, undirected, per-level noise "
                      "+-0.05 on 0.57,0.19,0.19,0.05", "ell": choice["ell"], "launch": list(shape)},
                      "metric": "edges/s", "value": chunk * nchunks / dt, "seconds": dt,
                      "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                   "peak_source": src},
                      "clocks": clocks.summary()}), flush=True)


def measure_batched(n_graphs: int = 512):
    """The first n_graphs graphs of the 4096-graph batched workload in one
    persistent launch (captured in a CUDA graph, replayed) against a
    CUDA-graph-captured loop of one rmat_generate per graph and the same loop
    launched eagerly, every graph's bytes compared between the two."""
    import torch
    import paper_1905_03525_gb300 as rm
    from paper_1905_03525_gb300 import autotune
    from paper_1905_03525_gb300.workloads import batched_graphs
    graphs = batched_graphs(4096)[:n_graphs]
    tables, choices = autotune.plan_batch(graphs)
    offs, off = [], 0
    for g in graphs:
        offs.append(off)
        off += (g["m"] + 63) // 64 * 64
    arenas = [torch.empty((off, 2), dtype=torch.int32, device="cuda") for _ in range(2)]
    outs = [[a[o:o + g["m"]] for o, g in zip(offs, graphs)] for a in arenas]
    s = torch.cuda.Stream()
    b = rm.rmat_batch_create()
    for g, t, o in zip(graphs, tables, outs[0]):
        rm.rmat_batch_add(b, t, g["seed"], 0, g["m"], o)
    rm.rmat_batch_prepare(b)

    def loop():
        for g, t, o in zip(graphs, tables, outs[1]):
            rm.rmat_generate(t, g["seed"], 0, g["m"], o, s)

    gb, gl = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(gb, stream=s):
        rm.rmat_batch_launch(b, s)
    loop()  # plans and uploads every table before capture
    with torch.cuda.graph(gl, stream=s):
        loop()
    with torch.cuda.stream(s):
        gb.replay()
        gl.replay()
        t_batch = _events_time(gb.replay, s, 3)
        t_graph = _events_time(gl.replay, s, 3)
    t_eager = _events_time(loop, s, 2)
    same = bool(torch.equal(arenas[0], arenas[1]))
    rm.rmat_check_device_errors()
    edges = sum(g["m"] for g in graphs)
    b.free()
    del gb, gl, arenas, outs
    torch.cuda.empty_cache()
    return {"graphs": n_graphs, "edges": edges,
            "workload": f"graphs 0..{n_graphs - 1} of the batched workload: k~U{{10..24}}, m=round(2^U(12,26)), "
                        "(a,b,c,d)~Dirichlet(57,19,19,5), seed=4096+i, u32; tables as the autotuner picks them",
            "batched_edges_per_s": edges / t_batch, "per_graph_cuda_graph_edges_per_s": edges / t_graph,
            "per_graph_eager_edges_per_s": edges / t_eager, "speedup_vs_graphed_loop": t_graph / t_batch,
            "speedup_vs_eager": t_eager / t_batch, "bytes_identical": same,
            "timing": "one captured persistent launch vs one captured per-graph loop, 3 replays each, CUDA events",
            "table_choice_per_k": {str(k): v for k, v in sorted(choices.items())}}


def measure_served(n_requests: int = 64, rate: float = 2000.0):
    """A short served trace: n_requests Poisson arrivals at `rate` per second
    through the continuous-batching server, against the same trace with one
    request on the GPU at a time."""
    from paper_1905_03525_gb300 import serve
    import torch
    free, _ = torch.cuda.mem_get_info()
    budget = min(160 * 10 ** 9, int(free * 0.8))
    trace = serve.served_trace(n_requests, rate=rate)
    res = {}
    for name, active in (("continuous_batching", 64), ("one_request_at_a_time", 1)):
        with serve.Server(budget, chunk_edges=1 << 28, step_edges=1 << 31, max_active=active) as srv:
            srv.wait(srv.submit(*G500, 16, 1 << 20, 1))  # warm-up request
            res[name] = serve.summarise(serve.run_trace(srv, trace))
    return {"requests": n_requests, "rate_per_s": rate, "hbm_budget_bytes": budget,
            "workload": "Poisson arrivals, k~U{12..30}, ef in {4,8,16,32}, m=ef*2^k, "
                        "(a,b,c,d)~Dirichlet(57,19,19,5), 2^28-edge chunks",
            **res, "speedup_vs_one_at_a_time": res["continuous_batching"]["edges_per_s"] /
            res["one_request_at_a_time"]["edges_per_s"],
            "p50_vs_one_at_a_time": res["one_request_at_a_time"]["p50_latency_s"] /
            res["continuous_batching"]["p50_latency_s"]}


def run_c4(args):
    """4096 graphs, k ~ U{10..24}, m = round(2^U(12,26)), parameters ~
    Dirichlet(57,19,19,5): one persistent launch per wave (captured in a CUDA
    graph) against one launch per graph."""
    import torch
    import paper_1905_03525_gb300 as rm
    from paper_1905_03525_gb300 import autotune
    from paper_1905_03525_gb300.workloads import batched_graphs
    graphs = batched_graphs(args.graphs)
    tables, choices = autotune.plan_batch(graphs)
    budget = int(args.wave_gib * (1 << 30))
    waves, cur, cur_b = [], [], 0
    for i, g in enumerate(graphs):
        nb = 8 * g["m"]
        if cur and cur_b + nb > budget:
            waves.append(cur)
            cur, cur_b = [], 0
        cur.append(i)
        cur_b += (nb + 255) // 256 * 256
    if cur:
        waves.append(cur)
    arena = torch.empty(budget // 4 + 64 * len(graphs), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    t_batch = t_loop = t_loop_graph = 0.0
    edges = 0
    checked = 0
    for w in waves:
        outs, off = [], 0
        for i in w:
            n = 2 * graphs[i]["m"]
            outs.append(arena[off:off + n].view(-1, 2))
            off += (n + 63) // 64 * 64
        b = rm.rmat_batch_create()
        for i, o in zip(w, outs):
            rm.rmat_batch_add(b, tables[i], graphs[i]["seed"], 0, graphs[i]["m"], o)
        rm.rmat_batch_prepare(b)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            rm.rmat_batch_launch(b, s)
        with torch.cuda.stream(s):
            g.replay()
            t_batch += _events_time(g.replay, s, 3)
        # reference bytes for a few graphs of the wave, then the per-graph loop
        probe = [0, len(w) // 2, len(w) - 1]
        saved = [outs[j].clone() for j in probe]
        def loop():
            for i, o in zip(w, outs):
                rm.rmat_generate(tables[i], graphs[i]["seed"], 0, graphs[i]["m"], o, s)
        loop()
        t_loop += _events_time(loop, s, 2)
        gl = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gl, stream=s):
            loop()
        with torch.cuda.stream(s):
            gl.replay()
            t_loop_graph += _events_time(gl.replay, s, 2)
        for j, ref in zip(probe, saved):
            assert torch.equal(outs[j], ref), "batched and per-graph bytes differ"
            checked += 1
        edges += sum(graphs[i]["m"] for i in w)
        b.free()
        del g, gl
    print(json.dumps({"workload": "c4", "config": {"workload": f"{len(graphs)} graphs, k~U{{10..24}}, "
                      "m=round(2^U(12,26)), (a,b,c,d)~Dirichlet(57,19,19,5), seed=4096+i, u32",
                      "waves": len(waves), "wave_budget_gib": args.wave_gib,
                      "table_choice_per_k": {str(k): v for k, v in sorted(choices.items())}},
                      "metric": "edges/s", "edges": edges,
                      "batched_edges_per_s": edges / t_batch, "per_graph_eager_edges_per_s": edges / t_loop,
                      "per_graph_cuda_graph_edges_per_s": edges / t_loop_graph,
                      "speedup_vs_eager": t_loop / t_batch, "speedup_vs_graphed_loop": t_loop_graph / t_batch,
                      "graphs_checked_bytewise": checked}), flush=True)


def run_part(args):
    """Partitioned k = 26, m = 2^30 graph (Sec. 3): host divide and conquer
    for the tile counts, then every tile in one persistent launch;
    the same graph size as the plain single launch beside it."""
    import torch
    import paper_1905_03525_gb300 as rm
    k, m, t = K, 1 << args.log2m, args.tile_levels
    table = rm.rmat_build_table(*G500, k, BOUND)
    t0 = time.perf_counter()
    p = rm.rmat_partition_create(table, t, m, SEED)
    plan_s = time.perf_counter() - t0
    ntiles, edges = rm.rmat_partition_info(p)
    out = rm.empty_edges(edges, k)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(max(3, args.warmup)):
            rm.rmat_generate_partition(p, out, s)
        part_s = _events_time(lambda: rm.rmat_generate_partition(p, out, s), s, args.steps)
        plain_s = _events_time(lambda: rm.rmat_generate(table, SEED, 0, m, out, s), s, args.steps)
        # local duplicate removal of the PE's edges (a synchronous call that
        # rewrites its input, so the output is regenerated before each call);
        # one untimed call, then the median wall time of `steps` calls
        dedup_times = []
        for it in range(1 + max(1, args.steps)):
            rm.rmat_generate_partition(p, out, s)
            s.synchronize()
            t0 = time.perf_counter()
            unique = rm.rmat_dedup_edges(out, edges, k, s)
            if it:
                dedup_times.append(time.perf_counter() - t0)
        dedup_s = sorted(dedup_times)[len(dedup_times) // 2]
    rm.rmat_check_device_errors()
    peak, peak_src = measured_peak()
    # the oracle beside it (one core): its own split, then edges of the first tiles
    import oracle
    t0 = time.perf_counter()
    tiles = oracle.partition(G500, t, m, SEED)
    ot = oracle.Table.variable(*G500, k, BOUND)
    done, sample = 0, 1 << 20
    for R, C, n, f in zip(tiles["row"], tiles["col"], tiles["count"], tiles["first"]):
        take = int(min(n, sample - done))
        oracle.generate_tile(ot, k, t, int(R), int(C), SEED, int(f), take)
        done += take
        if done >= sample:
            break
    cpu_s = time.perf_counter() - t0
    print(json.dumps({"workload": "part", "config": {"workload": f"R-MAT k={k}, m=2^{args.log2m}, G500 parameters, "
                      f"table bound {BOUND}, {1 << t}x{1 << t} tiles, one PE (all tile rows), u32", "tile_levels": t},
                      "metric": "edges/s", "edges": edges, "tiles": ntiles, "host_plan_ms": plan_s * 1e3,
                      "partitioned_edges_per_s": edges / part_s, "ms_per_launch": part_s * 1e3,
                      "hbm_frac": 8.0 * edges / part_s / 1e9 / peak, "peak_source": peak_src,
                      "plain_single_launch_edges_per_s": m / plain_s,
                      "dedup": {"unique_edges": unique, "ms": dedup_s * 1e3, "edges_per_s": edges / dedup_s,
                                "calls": len(dedup_times), "ms_first_to_last": [t * 1e3 for t in dedup_times],
                                "note": "rmat_dedup_edges on the PE's output: median wall time of a call after "
                                        "one untimed call"},
                      "cpu_baseline": {"value": done / cpu_s, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                       "sample": f"the oracle's tile split of the whole graph, then the first {done} "
                                                 "edges in tile order, one thread"}}), flush=True)


def run_kron(args):
    """Stochastic Kronecker graph with a 3 x 3 initiator (Sec. 3): k = 17
    (3^17 = 1.3e8 vertices), m = 2^30, variable table bound 4096, u32."""
    import torch
    import numpy as np
    import paper_1905_03525_gb300 as rm
    from paper_1905_03525_gb300.workloads import KRON3
    k, m = 17, 1 << args.log2m
    table = rm.rmat_build_table_kron(np.array(KRON3), 3, k, BOUND)
    out = rm.empty_edges_for(table, m)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(max(3, args.warmup)):
            rm.rmat_generate(table, SEED, 0, m, out, s)
        dt = _events_time(lambda: rm.rmat_generate(table, SEED, 0, m, out, s), s, args.steps)
    rm.rmat_check_device_errors()
    peak, peak_src = measured_peak()
    info = rm.rmat_table_info(table)
    import oracle
    ot = oracle.KronTable.variable(np.array(KRON3), 3, k, BOUND)
    sample = 1 << 20
    t0 = time.perf_counter()
    oracle.kron_generate(ot, k, SEED, 0, sample)
    cpu_s = time.perf_counter() - t0
    print(json.dumps({"workload": "kron", "config": {"workload": f"stochastic Kronecker graph, 3x3 initiator {KRON3}, "
                      f"k={k} (3^{k} vertices), m=2^{args.log2m}, table bound {BOUND} ({info['entries']} entries), "
                      "u32", "n0": 3, "k": k},
                      "metric": "edges/s", "value": m / dt, "ms_per_launch": dt * 1e3,
                      "hbm_frac": 8.0 * m / dt / 1e9 / peak, "peak_source": peak_src,
                      "roofline": {"bound": "hbm", "kernel": "k_kron_fast", "achieved": 8.0 * m / dt / 1e9,
                                   "peak": peak, "unit": "GB/s", "frac": 8.0 * m / dt / 1e9 / peak,
                                   "algorithmic_bytes_per_launch": 8 * m, "avg_launch_ms": dt * 1e3,
                                   "traffic_per_edge": 475.7e6 / 2 ** 26,
                                   "traffic_source": "dram__bytes_write.sum of the m=2^26 capture "
                                                     "(profiles/k_kron_fast_n3_k17_m2p26_full.md): stores coalesce",
                                   "measured_bound": "integer ALU pipe (68.6 % of its cycles, issue 71.9 %)"},
                      "cpu_baseline": {"value": sample / cpu_s, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                       "sample": f"edges 0..{sample - 1} of the same graph, one thread"}}),
          flush=True)


SKEWED = (0.9, 0.025, 0.025, 0.05)  # the skewed parameters of Sec. 4


def run_fig1(args):
    """The experiment of Fig. 1 on one GB300: edges/s against table size for
    variable-length tables (bounds 2^8..2^20) and fixed-length tables (l =
    4..10), with the Graph 500 and the skewed parameters of Sec. 4, n = 2^30
    vertices, 2^28 edges per launch (u32).  Tables up to ~2^14 columns are
    staged in shared memory; larger ones are read from global memory (L2)."""
    import torch
    import paper_1905_03525_gb300 as rm
    k, m = 30, 1 << min(args.log2m, 28)
    out = rm.empty_edges(m, k)
    s = torch.cuda.Stream()
    rows = []
    for pname, abcd in (("graph500", G500), ("skewed", SKEWED)):
        cases = [("variable", b, lambda b=b: rm.rmat_build_table(*abcd, k, b)) for b in
                 (1 << 8, 1 << 10, 1 << 12, 1 << 14, 1 << 16, 1 << 18, 1 << 20)]
        cases += [("fixed", ell, lambda ell=ell: rm.rmat_build_table_fixed(*abcd, k, ell)) for ell in range(4, 11)]
        for kind, x, build in cases:
            table = build()
            info = rm.rmat_table_info(table)
            with torch.cuda.stream(s):
                for _ in range(max(2, args.warmup)):
                    rm.rmat_generate(table, SEED, 0, m, out, s)
                dt = _events_time(lambda: rm.rmat_generate(table, SEED, 0, m, out, s), s, max(3, min(args.steps, 5)))
            rm.rmat_check_device_errors()
            rows.append({"params": pname, "kind": kind, ("bound" if kind == "variable" else "ell"): x,
                         "entries": info["entries"], "image_bytes": info["device_image_bytes"],
                         "edges_per_s": m / dt, "ns_per_edge_per_sm": dt / m * 1e9 * torch.cuda.get_device_properties(
                             torch.cuda.current_device()).multi_processor_count})
            table.free()
    print(json.dumps({"workload": "fig1", "config": {"workload": f"R-MAT k={k}, 2^{m.bit_length() - 1} edges per "
                      f"launch, seed {SEED}, u32; Graph 500 parameters {G500} and skewed {SKEWED}; variable bounds "
                      "2^8..2^20, fixed l = 4..10"}, "metric": "edges/s", "rows": rows}), flush=True)


def run_tablebuild(args):
    """Variable-length table construction (G500 parameters, k = 26) on the host
    (rmat_build_table) and on the GPU (rmat_build_table_gpu, identical
    tables), wall time per table for several bounds."""
    import torch
    import paper_1905_03525_gb300 as rm
    torch.cuda.synchronize()
    rows = []
    for bound in (1 << 12, 1 << 16, 1 << 20, 1 << 22):
        reps = 5 if bound <= 1 << 16 else 2
        rm.rmat_build_table_gpu(*G500, K, bound)  # warm
        times = {}
        for name, fn in (("host", lambda: rm.rmat_build_table(*G500, K, bound)),
                         ("gpu", lambda: rm.rmat_build_table_gpu(*G500, K, bound))):
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                fn().free()
                ts.append(time.perf_counter() - t0)
            times[name] = statistics.median(ts)
        row = {"bound": bound, "host_ms": times["host"] * 1e3, "gpu_ms": times["gpu"] * 1e3,
               "speedup": times["host"] / times["gpu"]}
        if bound <= 1 << 20:  # the oracle beside it (plain C, one thread)
            import oracle
            t0 = time.perf_counter()
            oracle.Table.variable(*G500, K, bound)
            row["oracle_ms"] = (time.perf_counter() - t0) * 1e3
        rows.append(row)
    # serving: a request with a large explicit bound, from the client's submit
    # call to its admission, with the table built on the submitting thread
    # (host) or by the server's builder thread (GPU), and the submit call itself
    from paper_1905_03525_gb300 import serve
    served = []
    for bound in (1 << 16, 1 << 18, 1 << 20):
        row = {"bound": bound}
        for mode, min_bound in (("host_build", 0), ("gpu_build", 1 << 14)):
            with serve.Server(1 << 30, chunk_edges=1 << 20, step_edges=1 << 22, max_active=4,
                              gpu_build_min_bound=min_bound) as srv:
                srv.wait(srv.wait(srv.submit(*G500, K, 1 << 16, 1, bound))["id"])  # warm: caches, kernels
                clock0 = srv.stats()["clock_s"]
                t0 = time.perf_counter()
                rid = srv.submit(*G500, K, 1 << 20, 2, bound)
                call_ms = (time.perf_counter() - t0) * 1e3
                st = srv.wait(rid)
            row[mode] = {"submit_call_ms": call_ms, "admission_ms": (st["admit_s"] - clock0) * 1e3,
                         "latency_ms": (st["done_s"] - clock0) * 1e3}
        served.append(row)
    print(json.dumps({"workload": "tablebuild", "config": {"workload": "variable-length table, G500 parameters, "
                      "k=26; wall time of one build call including copies back to the host; served: one request of "
                      "2^20 edges with that bound, from the client's submit call"},
                      "metric": "ms per table", "rows": rows, "served": served}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c1":
        run_c1(args)
    elif args.workload == "c3":
        run_c3(args)
    elif args.workload == "c4":
        run_c4(args)
    elif args.workload == "part":
        run_part(args)
    elif args.workload == "kron":
        run_kron(args)
    elif args.workload == "tablebuild":
        run_tablebuild(args)
    elif args.workload == "fig1":
        run_fig1(args)
    elif args.workload == "c5":
        from paper_1905_03525_gb300 import serve
        serve.bench(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
