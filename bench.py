"""Benchmark of the compressed-table PFAC matcher on GB300.

Default workload: the DNA-shaped configuration (alphabet 4, 10,000 patterns
of length U[8,64], 256 MiB input as one segment, 0.1% of positions planted).
A step is one pfac_match_async over the whole input with the table resident
and the input already in HBM: the scan kernel, the key-count scan, the
overflow re-scan and the key expansion (all kernels of the path).  The input
(256 MiB) is larger than L2 (129 MB), so no flush is needed between steps.

Printed (rank 0, one JSON line): scan throughput in Gbps (8 * input bytes /
device time, whole job over all ranks), the same metric end to end through
the C ABI with host buffers (pinned H2D of the input, D2H of count and keys),
the uncompressed-table kernel's Gbps and both tables' bytes, p50/p99 step
latency, the scan kernel's roofline against the measured HBM peak (its
algorithmic bytes over the time of both of its launches, the scan pass and the
emit pass), the CPU oracle timed on a bounded sample, clocks sampled during the
timed region, and the number of kernels launched.  The line also carries
``sweep_256_1000``: the same measurements on the alphabet-256 cell with 1,000
patterns and 512 MiB of input, timed after the main workload, and
``serving``: one level of the serving loop (50,000 resident patterns, Poisson
arrivals of packet batches offered at 100 Gbps for 2 s) with request p50/p99.

``--impl reference`` times the CPU oracle (Aho-Corasick with failure links,
all host cores) on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

SCAN_KERNELS_PER_STEP = 5  # scan, key-count reduce, offsets, overflow re-scan, key expansion
# (plus the resolver kernel where the plan hands queues over)


# dram__bytes_read.sum + dram__bytes_write.sum of one scan launch from ncu
# captures (summaries under profiles/), per workload and scan plan (the
# autotuner settles on one of near-equal plans), with the digest of the
# kernel sources they were taken on; reported only while the sources match
MEASURED_TRAFFIC = {
    "dna": [(310759680, "d100e0d9e6ba3865",
             {"variant": 1, "prefix_depth": 10, "bitmap_copies": 1, "child_masks": 1,
              "gram_filter": 1, "prefix_bytes": 1, "warps_per_cta": 16, "scan_kernel": 1,
              "records_per_slice": 512, "resolver": 2}),
            (311110912, "d100e0d9e6ba3865",
             {"variant": 1, "prefix_depth": 10, "bitmap_copies": 1, "child_masks": 1,
              "gram_filter": 1, "prefix_bytes": 1, "warps_per_cta": 16, "scan_kernel": 1,
              "records_per_slice": 32, "resolver": 2})],
    "sweep-256-1000": [(550563584, "d100e0d9e6ba3865",
                        {"variant": 1, "prefix_depth": 2, "bitmap_copies": 1, "child_masks": 1,
                         "gram_filter": 2, "prefix_bytes": 1, "warps_per_cta": 16,
                         "scan_kernel": 2, "records_per_slice": 32, "resolver": 2}),
                       (553913344, "d100e0d9e6ba3865",
                        {"variant": 2, "prefix_depth": 2, "bitmap_copies": 1, "child_masks": 2,
                         "gram_filter": 2, "prefix_bytes": 1, "warps_per_cta": 16,
                         "scan_kernel": 2, "records_per_slice": 32, "resolver": 1})],
}
KERNEL_SOURCES = ["kernels_q.cuh", "kernels_r.cuh", "kernels.cuh", "table.h"]
TUNE_SAMPLE = 128 << 20
E2E_CHUNK = 32 << 20


def kernel_digest():
    """Digest of the kernel sources with comments and blank lines removed
    (comment edits do not invalidate a capture)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1704_02272_gb300", "csrc", f)) as fh:
            src = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in src.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_traffic(workload, plan):
    digest = kernel_digest()
    for traffic, dg, pl in MEASURED_TRAFFIC.get(workload, []):
        if dg == digest and all(plan.get(k) == v for k, v in pl.items()):
            return traffic
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_workload(name, rank):
    seed_shift = 1000 * rank
    if name == "dna":
        return workloads.config2(seed=workloads.seed_for(2) + seed_shift)
    if name == "plain":
        return workloads.config1(seed=workloads.seed_for(1) + seed_shift)
    if name == "ids":
        return workloads.config3(seed=workloads.seed_for(3) + seed_shift)
    if name.startswith("letters-"):
        n = int(name.split("-")[1])
        return workloads.letters(n, seed=workloads.seed_for(6, 52, n) + seed_shift)
    if name.startswith("sweep-"):
        _, s, n = name.split("-")
        return workloads.config4(int(s), int(n), seed=workloads.seed_for(4, int(s), int(n)) + seed_shift)
    raise SystemExit(f"unknown workload {name}")


WORKLOAD_DESC = {
    "dna": "DNA-shaped: alphabet 4, 10,000 patterns U[8,64], 256 MiB one segment, 0.1% planted",
    "plain": "alphabet 256, 1,000 patterns U[4,32], 1 MiB, 2,000 planted",
    "ids": "IDS-shaped: alphabet 256, 20,000 log-normal patterns, 1 GiB of 64-1500 B packets",
}


METRIC = ("scan Gbps (1xGB300) compressed vs uncompressed PFAC, bit-exact; table bytes; "
          "p99 latency")


def base_config(w, args):
    return {"workload": WORKLOAD_DESC.get(args.workload, args.workload),
            "n_bytes": w.n_bytes, "segments": len(w.seg_offsets) - 1,
            "patterns": len(w.patterns), "alphabet": w.sigma,
            "l2": "input larger than L2, no flush"}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, budget_s=12.0, sample_mib=128, threads=None):
    """The oracle (AC with failure links, all host cores) on the first
    sample_mib MiB of the workload; scaled down until it fits the budget."""
    import oracle
    threads = threads or oracle.default_threads()
    ac = oracle.ACOracle(w.patterns)
    nb = min(w.n_bytes, sample_mib << 20)
    seg = w.seg_offsets
    t0 = time.perf_counter()
    ac.match(w.text, seg, lo=0, hi=nb, threads=threads)
    dt = time.perf_counter() - t0
    reps = max(1, int(budget_s / max(dt, 1e-3)))
    reps = min(reps, 5)
    t0 = time.perf_counter()
    for _ in range(reps):
        ac.match(w.text, seg, lo=0, hi=nb, threads=threads)
    dt = (time.perf_counter() - t0) / reps
    ac.close()
    return {"value": round(8 * nb / dt / 1e9, 4), "unit": "Gbps", "cores": threads,
            "kind": "oracle",
            "sample": f"start positions [0, {nb >> 20} MiB) of the workload, Aho-Corasick with "
                      f"failure links in C on {threads} threads, mean of {reps} runs"}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        # NCCL's own log (rank count, transport) stays on, on stderr
        os.environ.setdefault("NCCL_DEBUG", "INFO")
        dist.init_process_group("nccl")
    return rank, world, local


def run_reference(args):
    # the CPU oracle runs on rank 0 alone; the other ranks leave without
    # work (no process group: nothing is exchanged)
    if int(os.environ.get("RANK", "0")) != 0:
        return
    w = load_workload(args.workload, 0)
    import oracle
    threads = oracle.default_threads()
    ac = oracle.ACOracle(w.patterns)
    nb = min(w.n_bytes, args.ref_sample_mib << 20)
    for _ in range(args.warmup):
        ac.match(w.text, w.seg_offsets, lo=0, hi=nb, threads=threads)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ac.match(w.text, w.seg_offsets, lo=0, hi=nb, threads=threads)
        t.append(time.perf_counter() - t0)
    ac.close()
    ms = 1e3 * sum(t) / len(t)
    v = 8 * nb / (ms / 1e3) / 1e9
    sample = (f"start positions [0, {nb >> 20} MiB) of the workload per step, Aho-Corasick with "
              f"failure links in C on {threads} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "Gbps",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": base_config(w, args),
        "cpu_baseline": {"value": round(v, 4), "unit": "Gbps", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 4), "unit": "Gbps", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def user_options(args):
    user_opt = {}
    for key, val in (("variant", args.variant), ("prefix_depth", args.prefix_depth),
                     ("bitmap_copies", args.copies), ("child_masks", args.masks),
                     ("gram_filter", args.gram), ("prefix_bytes", args.bytes),
                     ("warps_per_cta", args.warps), ("scan_kernel", args.kernel),
                     ("records_per_slice", args.records), ("resolver", args.resolver)):
        if val:
            user_opt[key] = val
    return user_opt


def time_cell(pfac, torch, w, dev, stream, args, user_opt, workload_name, graph_steps=True,
              gpu_index=0, barrier=None, call_opt=None):
    """Times one workload: K steps of one pfac_match_async over the whole
    input (the captured graph of the call, replayed), the scan kernel's two
    launches (scan pass, emit pass) by events on their stream, and the
    uncompressed table on the same input.  Returns the measurements and the
    objects the caller needs for the end-to-end leg."""
    N = w.n_bytes
    S = len(w.seg_offsets) - 1
    # the bytes this call's walks start at (a shard's own share; the rest of
    # its text is the read halo)
    n_starts = call_opt["starts_end"] if call_opt and call_opt.get("starts_end") else N
    text = torch.from_numpy(w.text).to(dev)
    seg = torch.from_numpy(w.seg_offsets.astype(np.int64)).to(dev)
    t0 = time.perf_counter()
    table = pfac.Table(w.patterns, w.sigma, truncate_depth=args.truncate)
    build_s = time.perf_counter() - t0
    info = table.info()
    t0 = time.perf_counter()
    dense = pfac.Table(w.patterns, w.sigma, layout=pfac.LAYOUT_DENSE, truncate_depth=args.truncate)
    dense_build_s = time.perf_counter() - t0
    dinfo = dense.info()

    tune = dense_tune = None
    if not args.no_autotune and not user_opt:
        # the autotuner on a bounded prefix sample of the input (whole
        # segments, at most TUNE_SAMPLE bytes); untimed
        nb = max(16, min(N, TUNE_SAMPLE) & ~15)
        offs = w.seg_offsets.astype(np.int64)
        cut = int(np.searchsorted(offs, nb, side="left"))  # offsets below nb
        s_offs = torch.from_numpy(np.concatenate([offs[:cut], [nb]])).to(dev)
        tune = pfac.autotune(table, text[:nb], s_offs)
        # the uncompressed table gets the same search over the same kernels
        dense_tune = pfac.autotune(dense, text[:nb], s_offs)
    call_opt = call_opt or {}
    # the untimed reference call runs the plan the steps run
    with torch.cuda.stream(stream):
        keys = pfac.match(table, text, seg, stream=stream, **user_opt, **call_opt)
        stream.synchronize()
    n_match = keys.numel()
    cap = n_match + 1024
    out = torch.empty(cap, dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)

    K, W = args.steps, args.warmup
    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_b, ev_e, sc_b, sc_e, em_b, em_e = mk(), mk(), mk(), mk(), mk(), mk()
    with torch.cuda.stream(stream):
        for e in ev_b + ev_e + sc_b + sc_e + em_b + em_e:  # creates the CUDA events
            e.record(stream)
    stream.synchronize()

    plan = pfac.plan(table, **user_opt)
    ws = torch.empty(max(pfac.workspace_bytes(table, N, S, **user_opt),
                         pfac.workspace_bytes(dense, N, S),
                         pfac.workspace_bytes(dense, N, S, scan_kernel=pfac.binding.KERNEL_SERIAL)),
                     dtype=torch.uint8, device=dev)

    def step(i=None, tbl=table):
        opt = dict(user_opt) if tbl is table else {}
        opt.update(call_opt)
        if i is not None:
            opt["scan_events"] = (sc_b[i], sc_e[i])
            opt["emit_events"] = (em_b[i], em_e[i])
        pfac.match_async(tbl, text, seg, out, cnt, st, ws, stream=stream, **opt)

    graph = None
    if graph_steps:
        # the whole call (workspace clear, segment pass, scan, ordering kernels)
        # captured once and replayed per step
        for _ in range(2):
            step()
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            step()
        stream.synchronize()

    for _ in range(W):
        step()
    stream.synchronize()
    if barrier is not None:
        barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    for i in range(K):
        ev_b[i].record(stream)
        if graph is not None:
            with torch.cuda.stream(stream):
                graph.replay()
        else:
            step(i)
        ev_e[i].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    if graph is not None:
        # kernel times of the graph steps: one more eager pass with events
        for i in range(K):
            step(i)
        stream.synchronize()
    clk = clocks.stop()
    if barrier is not None:
        barrier()
    step_ms = [ev_b[i].elapsed_time(ev_e[i]) for i in range(K)]
    scan_ms = [sc_b[i].elapsed_time(sc_e[i]) for i in range(K)]
    emit_ms = [em_b[i].elapsed_time(em_e[i]) for i in range(K)]
    total_ms = ev_b[0].elapsed_time(ev_e[K - 1])
    assert int(st.item()) == 0, f"device status {int(st.item())}"
    assert int(cnt.item()) == n_match

    # uncompressed table on the same GPU, same input
    dk = pfac.match(dense, text, seg, stream=stream, **call_opt)
    stream.synchronize()
    exact = bool(torch.equal(dk, keys))
    del dk

    def timed(tbl, opt=None):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        o = dict(call_opt)
        o.update(opt or {})
        for _ in range(W):
            pfac.match_async(tbl, text, seg, out, cnt, st, ws, stream=stream, **o)
        e0.record(stream)
        for _ in range(K):
            pfac.match_async(tbl, text, seg, out, cnt, st, ws, stream=stream, **o)
        e1.record(stream)
        stream.synchronize()
        return 8.0 * n_starts * K / (e0.elapsed_time(e1) / 1e3) / 1e9

    dense_gbps = timed(dense)
    dense_plan = pfac.plan(dense)
    # the thread-serial kernel (one thread walks its positions in turn)
    serial = {"scan_kernel": pfac.binding.KERNEL_SERIAL}
    dk = pfac.match(dense, text, seg, stream=stream, **call_opt, **serial)
    stream.synchronize()
    serial_exact = bool(torch.equal(dk, keys))
    del dk
    serial_gbps = timed(dense, serial)
    merged = None if args.no_suffix_merge or args.truncate else time_merged(
        pfac, torch, w, text, seg, keys, stream, args, call_opt, n_starts)

    hbm_peak, peak_kind = peaks()
    # algorithmic bytes of the scan kernel's launches in one step: every input
    # byte read once and one 8-byte record per matched position written (the
    # 16-byte halo of each 512-byte slice is re-read from L2 and not counted);
    # charged to the time of both launches (scan pass and emit pass), which
    # between them read the input and write those bytes
    pos = keys >> 24
    matched_positions = int(torch.unique_consecutive(pos).numel()) if n_match else 0
    alg_bytes = n_starts + 8 * matched_positions
    scan_avg_ms = sum(scan_ms) / K
    emit_avg_ms = sum(emit_ms) / K
    kern_ms = scan_avg_ms + emit_avg_ms
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": args.traffic if (args.traffic is not None and graph_steps) else (
                    measured_traffic(workload_name, plan) if not user_opt else None),
                "kernel": "k_scanq (compressed-table scan: scan pass + emit pass)",
                "alg_bytes_per_launch": alg_bytes,
                "scan_pass_ms": round(scan_avg_ms, 4), "emit_pass_ms": round(emit_avg_ms, 4)}
    cell = {
        "value": round(8.0 * n_starts * K / (total_ms / 1e3) / 1e9, 3), "unit": "Gbps",
        "ms_per_step": round(total_ms / K, 4),
        "p50_ms": round(statistics.median(step_ms), 4),
        "p99_ms": round(float(np.percentile(step_ms, 99)), 4),
        "matches": n_match, "matched_position_frac": round(matched_positions / N, 6),
        "table_bytes": {"compressed": info["device_bytes"], "dense": dinfo["device_bytes"],
                        "paper_model": info["paper_bytes"], "trie_nodes": info["trie_nodes"],
                        "records": info["records"], "merged_leaves": info["merged_leaves"]},
        "dense": {"value": round(dense_gbps, 3), "unit": "Gbps", "bit_exact_vs_compressed": exact,
                  "kernel": "the compressed table's kernels over the dense transition table",
                  "scan_plan": dense_plan, "autotuned": dense_tune,
                  "thread_serial": {"value": round(serial_gbps, 3), "unit": "Gbps",
                                    "bit_exact_vs_compressed": serial_exact}},
        "suffix_merge": merged,
        "build_s": {"compressed": round(build_s, 3), "dense": round(dense_build_s, 3)},
        "roofline": roofline,
        "scan_plan": plan, "autotuned": tune, "cuda_graph": bool(graph is not None),
        "wall_s_timed": round(wall, 4),
        "clocks": clk,
    }
    ctx = {"table": table, "dense": dense, "text": text, "seg": seg, "keys": keys,
           "cap": cap, "total_ms": total_ms, "n_match": n_match}
    return cell, ctx


def time_merged(pfac, torch, w, text, seg, keys, stream, args, call_opt, n_starts):
    """The merged trie (reduction step 2, Section 3.2) on the same input: its
    table sizes against the tree's, whether its keys equal the plain table's,
    and its throughput over K eager calls with the library's default plan."""
    N, S, K = w.n_bytes, len(w.seg_offsets) - 1, args.steps
    t0 = time.perf_counter()
    mt = pfac.Table(w.patterns, w.sigma, suffix_merge=True)
    m_build = time.perf_counter() - t0
    try:
        mi = mt.info()
        with torch.cuda.stream(stream):
            mk = pfac.match(mt, text, seg, stream=stream, **call_opt)
            stream.synchronize()
        exact = bool(torch.equal(mk, keys))
        out = torch.empty(keys.numel() + 1024, dtype=torch.int64, device=text.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=text.device)
        st = torch.zeros(1, dtype=torch.int32, device=text.device)
        ws = torch.empty(pfac.workspace_bytes(mt, N, S), dtype=torch.uint8, device=text.device)
        del mk

        def step():
            pfac.match_async(mt, text, seg, out, cnt, st, ws, stream=stream, **call_opt)

        for _ in range(args.warmup):
            step()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            step()
        e1.record(stream)
        stream.synchronize()
        assert int(st.item()) == 0, f"device status {int(st.item())}"
        gbps = 8.0 * n_starts * K / (e0.elapsed_time(e1) / 1e3) / 1e9
        per_node = (w.sigma + 7) // 8 + 4
        return {"value": round(gbps, 3), "unit": "Gbps", "bit_exact_vs_compressed": exact,
                "device_bytes": mi["device_bytes"], "records": mi["records"],
                "merged_trie_nodes": mi["merged_trie_nodes"], "side_entries": mi["side_entries"],
                "paper_model": mi["merged_trie_nodes"] * per_node,
                "node_reduction": round(1.0 - mi["merged_trie_nodes"] / mi["trie_nodes"], 4),
                "build_s": round(m_build, 3), "plan": "library default, eager calls"}
    finally:
        mt.close()


def shard_workload(full, world, rank):
    """One job split by start position: every rank builds the same workload,
    keeps its share plus a read halo of max_len - 1 bytes, and reports global
    positions (starts_end / position_base).  Returns the rank's workload, its
    match options and its shard."""
    from paper_1704_02272_gb300 import shard as shard_mod
    sh = shard_mod.plan(full.n_bytes, full.seg_offsets, world, full.max_len)[rank]
    if sh.stop <= sh.start:
        raise SystemExit(f"rank {rank} has no share of a {full.n_bytes}-byte input")
    w = workloads.Workload(f"{full.name}-shard{rank}", full.sigma, full.patterns,
                           np.ascontiguousarray(full.text[sh.start:sh.read_end]), sh.seg)
    return w, {"starts_end": sh.stop - sh.start, "position_base": sh.start}, sh


def run_ours(args):
    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1704_02272_gb300 as pfac

    from paper_1704_02272_gb300 import shard as shard_mod
    strong = world > 1 and args.scaling == "strong"
    call_opt, sh = None, None
    if strong:
        full = load_workload(args.workload, 0)
        w, call_opt, sh = shard_workload(full, world, rank)
        N_job, N_rank = full.n_bytes, sh.stop - sh.start
    else:
        w = load_workload(args.workload, rank)
        N_job, N_rank = w.n_bytes * world, w.n_bytes
    N = w.n_bytes
    S = len(w.seg_offsets) - 1
    stream = torch.cuda.Stream(device=dev)
    user_opt = user_options(args)
    K, W = args.steps, args.warmup

    barrier = torch.distributed.barrier if world > 1 else None
    cell, ctx = time_cell(pfac, torch, w, dev, stream, args, user_opt, args.workload,
                          gpu_index=local, barrier=barrier, call_opt=call_opt)
    clk = cell.pop("clocks")
    total_ms = ctx["total_ms"]
    if world > 1:
        tt = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    value = 8.0 * N_job * K / (total_ms / 1e3) / 1e9
    shard_line = None
    if strong:
        # after the timed region: the merge (one gather of counts and lists,
        # concatenated in rank order), checked on rank 0 against one
        # unsharded call over the whole input
        merged = shard_mod.gather(ctx["keys"])
        shard_line = {"ranks": world, "share_bytes": N_rank, "halo_bytes": N - N_rank,
                      "merged_matches": int(merged.numel())}
        if rank == 0:
            ft = torch.from_numpy(full.text).to(dev)
            fs = torch.from_numpy(full.seg_offsets.astype(np.int64)).to(dev)
            whole = pfac.match(ctx["table"], ft, fs, **user_opt)
            torch.cuda.synchronize()
            shard_line["bit_exact_vs_unsharded"] = bool(torch.equal(whole, merged))
            del ft, fs, whole
        del merged
    table, keys, n_match, cap = ctx["table"], ctx["keys"], ctx["n_match"], ctx["cap"]
    text, seg = ctx["text"], ctx["seg"]

    # prefix matching: the timed steps gave candidates; time their
    # verification (pfac_verify) and report the exact count
    prefix_line = None
    if args.truncate:
        cand = keys
        vout = torch.empty(max(cand.numel(), 1), dtype=torch.int64, device=dev)
        vcnt = torch.zeros(1, dtype=torch.int64, device=dev)
        v0 = torch.cuda.Event(enable_timing=True)
        v1 = torch.cuda.Event(enable_timing=True)
        for _ in range(2):
            pfac.verify_into(table, text, seg, cand, vout, vcnt, stream=stream)
        v0.record(stream)
        for _ in range(K):
            pfac.verify_into(table, text, seg, cand, vout, vcnt, stream=stream)
        v1.record(stream)
        stream.synchronize()
        vms = v0.elapsed_time(v1) / K
        exact_keys = vout[:int(vcnt.item())]
        prefix_line = {"truncate_depth": args.truncate, "candidates": n_match,
                       "exact_matches": int(exact_keys.numel()),
                       "verify_ms": round(vms, 4),
                       "match_and_verify_gbps": round(8.0 * N / ((total_ms / K + vms) / 1e3) / 1e9, 3)}

    # end to end through the C ABI from host buffers: pfac_match_host copies
    # the pinned text in and the keys out, chunk by chunk, overlapped with the
    # matching
    host_in = torch.from_numpy(w.text).pin_memory()
    host_seg = torch.from_numpy(w.seg_offsets.astype(np.int64)).pin_memory()
    host_out = torch.empty(cap, dtype=torch.int64).pin_memory()
    chunk = E2E_CHUNK
    n_chunks = (N + chunk - 1) // chunk

    def e2e_step():
        n = pfac.match_host(table, host_in, host_seg, host_out, chunk_bytes=chunk,
                            stream=stream, **user_opt)
        if sh is not None:
            # the shard's own starts, at global positions (its halo's starts
            # belong to the next rank)
            return int(shard_mod.own(host_out[:n].numpy().view(np.uint64), sh).size)
        return n

    for _ in range(max(1, W)):
        e2e_step()
    if world > 1:
        torch.distributed.barrier()
    e0 = time.perf_counter()
    e2e_n = 0
    for _ in range(K):
        e2e_n = e2e_step()
    e2e_s = (time.perf_counter() - e0) / K
    if world > 1:
        # the slowest rank sets the job's end-to-end time
        tt = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(tt.item())
    halo = (n_chunks - 1) * max(w.max_len - 1, 0)
    e2e = {"value": round(8.0 * N_job / e2e_s / 1e9, 3), "unit": "Gbps",
           "h2d_bytes_per_step": int(N + halo + 8 * (S + 1 + 2 * n_chunks)),
           "d2h_bytes_per_step": int(8 * e2e_n + 16 * n_chunks),
           "call": "pfac_match_host", "chunk_bytes": chunk}
    assert e2e_n == n_match
    table.close()
    ctx["dense"].close()
    del ctx, text, seg, keys, host_in, host_out

    # the alphabet-256 cell (1,000 patterns, 512 MiB), where a scan over few
    # survivors should come closest to the HBM bound (timed the same way, on
    # rank 0's GPU only)
    extra = {}
    if not args.no_sweep_cell and args.workload != "sweep-256-1000" and world == 1:
        wc = load_workload("sweep-256-1000", 0)
        c2, cx2 = time_cell(pfac, torch, wc, dev, stream, args, user_opt, "sweep-256-1000")
        c2["config"] = {"workload": "sweep cell: alphabet 256, 1,000 patterns U[4,64], 512 MiB "
                                    "uniform, one segment",
                        "n_bytes": wc.n_bytes, "patterns": len(wc.patterns), "alphabet": 256,
                        "l2": "input larger than L2, no flush"}
        cx2["table"].close()
        cx2["dense"].close()
        extra["sweep_256_1000"] = c2
        del cx2, wc

    # one short serving level (100 Gbps offered, 2 s of arrivals) with the
    # request latency the serving loop reports
    if not args.no_serving and world == 1:
        extra["serving"] = serving_levels(args, [100.0], 2.0, 30, 2000, verbose=False)[0]

    roofline = cell.pop("roofline")
    # this library's launches per step: the five of every call, the resolver
    # kernel where the plan hands queues to it, the segment pass for several
    # segments
    per_step = SCAN_KERNELS_PER_STEP + (1 if cell["scan_plan"].get("resolver") == 2 else 0) + \
        (1 if S > 1 else 0)
    line = {
        "metric": METRIC,
        "value": round(value, 3), "unit": "Gbps", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(total_ms / K, 4), "higher_is_better": True,
        "scaling": "strong" if strong else "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": dict(base_config(w if not strong else full, args),
                       parallelism=(f"{world} start-range shards of one input" if strong else
                                    f"{world} independent inputs" if world > 1 else "1 GPU"),
                       prefix_depth=cell["scan_plan"]["prefix_depth"],
                       variant=args.variant or "default", bitmap_copies=args.copies or "auto",
                       autotuned=cell.pop("autotuned"), scan_plan=cell.pop("scan_plan"),
                       cuda_graph=cell.pop("cuda_graph")),
        "p50_ms": cell["p50_ms"], "p99_ms": cell["p99_ms"],
        "matches": cell["matches"], "matched_position_frac": cell["matched_position_frac"],
        "table_bytes": cell["table_bytes"], "dense": cell["dense"],
        "suffix_merge": cell["suffix_merge"],
        "prefix_matching": prefix_line,
        "shards": shard_line,
        "build_s": cell["build_s"],
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": per_step * K,
        "clocks": clk,
        "wall_s_timed": cell["wall_s_timed"],
    }
    line.update(extra)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w if not strong else full)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def serving_levels(args, loads, seconds, n_min, n_max, verbose=True):
    """Serving loop: Poisson arrivals of packet batches (1-4096 packets of
    64-9000 bytes, 50,000 IDS-shaped patterns resident) at each offered load;
    each level runs `seconds` of arrivals (at least n_min, at most n_max
    batches).  Per level: p50/p99 latency (completion minus scheduled
    arrival), its parts (how late the load generator submitted, the wait for
    admission, the host time of the admission's calls, the time on the GPU),
    the results whose keys went through a staging copy instead of the result
    arena, and the sustained throughput.  The load generator consumes each
    result as it is polled (a view of the server's memory) and releases it at
    once, as a client that keeps up does."""
    import gc
    import threading
    import torch
    import paper_1704_02272_gb300 as pfac
    torch.cuda.set_device(0)
    pats = workloads.config5_patterns()
    rs = np.random.RandomState(workloads.seed_for(5) + 1)
    batches = [workloads.serving_batch(rs, pats) for _ in range(args.serve_batches)]
    pinned = [(torch.from_numpy(t).pin_memory(), torch.from_numpy(s.view(np.int64)).pin_memory())
              for t, s in batches]
    mean_bytes = float(np.mean([t.size for t, _ in batches]))
    table = pfac.Table(pats, 256)
    t0, s0 = batches[0]
    pfac.autotune(table, torch.from_numpy(t0).cuda(), torch.from_numpy(s0.view(np.int64)).cuda())
    biggest = max(t.size for t, _ in batches)
    out = []
    with pfac.Server(table, n_slots=args.serve_slots, device_bytes=args.serve_pool << 20,
                     max_request_bytes=biggest) as srv:
        for _ in range(3):  # warm-up
            rid = srv.submit(*pinned[0])
            srv.wait(rid, 60)
            srv.release(rid)
        for load in loads:
            # the load generator's own garbage collection would stall both of
            # its threads mid-level: collect between levels, not during them
            gc.collect()
            gc.disable()
            rate = load * 1e9 / 8.0 / mean_bytes  # batches per second
            n = int(min(max(n_min, rate * seconds), n_max))
            arr = workloads.poisson_arrivals(np.random.RandomState(int(load)), rate, n)
            ids, sched, sizes, late = [], [], [], []
            start = time.monotonic() + 0.05

            def submitter():
                for k in range(n):
                    at = start + arr[k]
                    dt = at - time.monotonic()
                    if dt > 0:
                        time.sleep(dt)
                    t, s = pinned[k % len(pinned)]
                    late.append(time.monotonic() - at)
                    ids.append(srv.submit(t, s))
                    sched.append(at)
                    sizes.append(t.numel())

            th = threading.Thread(target=submitter)
            th.start()
            # a client that consumes each result as it comes: keep the
            # stamps, release the request (its keys' block) at once
            done = {}
            while len(done) < n:
                r = srv.poll(copy=False)
                if r is None:
                    time.sleep(0.0002)
                    continue
                r["n_keys"] = r.pop("keys").size
                srv.release(r["id"])
                done[r["id"]] = r
            th.join()
            lat, wait_adm, service, issue = [], [], [], []
            staged = 0  # results whose keys went through a staging copy
            for rid, at in zip(ids, sched):
                r = done[rid]
                assert r["status"] == 0
                lat.append(r["t_done"] - at)
                wait_adm.append(r["t_admit"] - r["t_submit"])
                service.append(r["t_done"] - r["t_admit"])
                issue.append(r["t_issued"] - r["t_admit"])
                staged += 0 if r["in_arena"] or not r["n_keys"] else 1
            gc.enable()
            t_end = max(done[i]["t_done"] for i in ids)
            ms = lambda xs, q: round(1e3 * float(np.percentile(xs, q)), 3)
            line = {"impl": "ours", "mode": "serving", "offered_gbps": load,
                    "sustained_gbps": round(8.0 * sum(sizes) / (t_end - start) / 1e9, 3),
                    "p50_ms": ms(lat, 50), "p99_ms": ms(lat, 99),
                    "p99_submit_late_ms": ms(late, 99), "p99_admission_wait_ms": ms(wait_adm, 99),
                    "p99_on_gpu_ms": ms(service, 99), "p99_issue_ms": ms(issue, 99),
                    "max_issue_ms": round(1e3 * max(issue), 3), "staged_results": staged,
                    "requests": n, "mean_request_bytes": int(mean_bytes),
                    "slots": args.serve_slots}
            out.append(line)
            if verbose:
                print(json.dumps(line), flush=True)
    table.close()
    return out


def run_serving(args):
    """The serving sweep: one JSON line per offered load."""
    loads = [float(x) for x in args.loads.split(",")]
    return serving_levels(args, loads, args.serve_seconds, args.serve_min, args.serve_max)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dna")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per scan launch from an ncu capture of the current kernel sources")
    # the reference arm's sample: the same 128 MiB of start positions as the
    # cpu_baseline leg of the default line
    ap.add_argument("--ref-sample-mib", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-suffix-merge", action="store_true",
                    help="skip the merged-trie table (reduction step 2) beside the plain one")
    ap.add_argument("--scaling", default="strong", choices=["strong", "weak"],
                    help="with several GPUs: strong = one input split by start position "
                         "(shards with a read halo, merged after the timed region); weak = "
                         "an input of the full size per GPU")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the short serving level timed after the main workload")
    ap.add_argument("--no-sweep-cell", action="store_true",
                    help="skip the alphabet-256 x 1,000-pattern cell timed after the main "
                         "workload")
    ap.add_argument("--variant", type=int, default=0, help="1: entries via L2, 2: entries in smem")
    ap.add_argument("--prefix-depth", type=int, default=0)
    ap.add_argument("--copies", type=int, default=0, help="prefix-bitmap copies in smem")
    ap.add_argument("--masks", type=int, default=0, help="child masks: 1 off, 2 on")
    ap.add_argument("--gram", type=int, default=0, help="gram filter first stage: 1 off, 2 on")
    ap.add_argument("--bytes", type=int, default=0, help="prefix bytes first stage: 1 off, 2 on")
    ap.add_argument("--warps", type=int, default=0, help="scan-kernel warps per CTA: 16 or 24")
    ap.add_argument("--records", type=int, default=0, help="records per slice: 32 or 512")
    ap.add_argument("--resolver", type=int, default=0,
                    help="queues of survivors: 1 resolved by the scan, 2 by the resolver kernel")
    ap.add_argument("--kernel", type=int, default=0,
                    help="scan kernel: 1 queued (input staged in shared memory), 2 register-staged "
                         "(alphabets of 129-256 symbols)")
    ap.add_argument("--truncate", type=int, default=0,
                    help="prefix matching (Section 2.4): tables hold the patterns cut to this "
                         "many symbols; the timed step yields candidates, verified after")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip pfac_autotune on a sample of the input (it runs by default "
                         "when no scan option is given)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every step's kernels directly instead of replaying the "
                         "captured CUDA graph of one call")
    ap.add_argument("--loads", default="10,25,50,100,200,300,400")
    ap.add_argument("--serve-batches", type=int, default=48)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-pool", type=int, default=4096, help="MiB")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-min", type=int, default=30)
    ap.add_argument("--serve-max", type=int, default=10000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "serving":
        run_serving(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
