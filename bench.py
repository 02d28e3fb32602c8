"""Benchmark of the PFAC scan on one GB300 (or N GPUs, one process each).

Workload (one step = one scan of the whole text): the genome-scale single scan —
256 Mi bases of a 41 %-GC order-2 Markov text with 5 % planted repeats, 2-bit packed
and resident in HBM, against 20,000 patterns of length 20-100 (70 % text substrings
with 1 % point mutations). Output: one int32 longest-pattern id per base.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). ``value`` is Gbases/s over all ranks; each rank scans
its own text of the same size (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gbases/s PFAC scan at 1 GB300 (% of HBM roofline); batched vs per-call; p99 ms"
UNIT = "Gbases/s"
N_BASES = 256 << 20
N_PATTERNS = 20_000
BYTES_PER_BASE = 4.25          # 2-bit packed text in (0.25 B) + int32 id out (4 B)
HBM_FALLBACK_GBS = 6800.0


def workload_name(n_bases=N_BASES, n_patterns=N_PATTERNS):
    return (f"genome-scale single scan: {n_bases} bases order-2 Markov 41% GC + 5% repeats, "
            f"2-bit packed; {n_patterns} patterns len 20-100 (70% substrings w/ 1% mutations)")


def measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every `interval_ms` (default 50)
    in the background from start() to stop(); each sample carries its host time, so the
    samples inside a window (the timed steps) can be picked out."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 50):
        self.gpu = gpu_index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []          # (host time, csv line)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.proc = None

    def __enter__(self):
        return self.start()

    def __exit__(self, *a):
        self.stop()

    def summary(self, t0: float | None = None, t1: float | None = None):
        """Median SM clock over the samples taken under load (GPU utilisation > 0),
        between host times t0 and t1 when given, and every throttle reason seen active
        in them."""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in list(self.lines):
            if (t0 is not None and ts < t0) or (t1 is not None and ts > t1):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                clk, cmax, util = float(parts[1]), float(parts[2]), float(parts[4])
            except ValueError:
                continue
            mx = cmax
            if util > 0:
                sm.append(clk)
                for name, v in zip(names, parts[6:10]):
                    if v.lower() == "active":
                        reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples_under_load": len(sm)}


def kernel_source_hash():
    """SHA-256 (first 16 hex digits) of the scan kernels' sources: pfac_kernels.cu, then
    pfac_device.cuh."""
    h = hashlib.sha256()
    for f in ("pfac_kernels.cu", "pfac_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1811_10498_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_fields(txt: str) -> dict:
    """The "- key: value" lines of an ncu summary."""
    vals = {}
    for line in txt.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    return vals


def profiled_traffic(path: str | None = None):
    """DRAM bytes per launch of the scan kernel from the committed ncu summary (or the
    summary at `path`), if it was taken on the current kernel source; else None."""
    p = path or os.path.join(ROOT, "profiles", "scan_kernel_genome_scan.md")
    try:
        txt = open(p).read()
    except OSError:
        return None
    vals = profile_fields(txt)
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def job_throughput(local_s: float, n_per_rank: int, steps: int, world: int, device=None):
    """Whole-job Gbases/s under weak scaling: every rank scans its own text of
    `n_per_rank` bases `steps` times; the job takes as long as its slowest rank (max of
    the ranks' timed totals over the process group, which must be initialised when
    world > 1). Returns (slowest total seconds, Gbases/s)."""
    total_s = local_s
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([local_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    return total_s, world * n_per_rank * steps / total_s / 1e9


def make_workload(rank: int, n_bases: int, n_patterns: int):
    from paper_1811_10498_gb300 import datagen
    return datagen.genome_scan(seed=2 + rank, n_bases=n_bases, n_patterns=n_patterns)


def cpu_baseline(w, got_prefix: np.ndarray | None, seconds: float = 8.0, single_seconds: float = 2.0):
    """The CPU oracle (scan only) on the first bases of the text: on all host threads,
    and (``single_core``) the same scan on one thread over a shorter prefix."""
    import oracle
    threads = os.cpu_count() or 1
    trie = oracle.Trie((w.blob, w.offsets))
    n = w.text.size
    sample = min(n, 1 << 20)
    t0 = time.perf_counter()
    trie.scan_threads(w.text, threads, 0, sample)
    dt = time.perf_counter() - t0
    rate = sample / max(dt, 1e-9)
    sample = int(min(n, max(1 << 20, rate * seconds)))
    sample -= sample % 64
    t0 = time.perf_counter()
    ref = trie.scan_threads(w.text, threads, 0, sample)
    dt = time.perf_counter() - t0
    out = {"value": sample / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"first {sample} offsets of the same text (walks may read past the sample), "
                     f"{threads} threads, scan only"}
    if got_prefix is not None:
        out["parity_on_sample"] = bool(np.array_equal(ref[:sample], got_prefix[:sample]))
    one = int(min(n, max(1 << 18, sample / dt / threads * single_seconds)))
    t0 = time.perf_counter()
    trie.scan(w.text, 0, one)
    dt1 = time.perf_counter() - t0
    out["single_core"] = {"value": one / dt1 / 1e9, "unit": UNIT, "cores": 1,
                          "sample": f"first {one} offsets of the same text, 1 thread, scan only"}
    return out


def batched_measure(steps: int, tune: bool = True):
    """The batched workload: 4,096 reads (log-normal lengths, median 1,500) against 64
    resident tables; one captured CUDA graph per batch vs one launch per read. tune=False
    keeps the library's default launch shape (no autotuner launches before the graph)."""
    import torch
    from paper_1811_10498_gb300 import _binding as b
    from paper_1811_10498_gb300 import datagen
    from paper_1811_10498_gb300.batched import BatchedScanner, PerReadGraph, scan_per_read
    w = datagen.read_batch(seed=4)
    t0 = time.perf_counter()
    tables = [b.Table(s) for s in w.sets]
    build_s = time.perf_counter() - t0
    n = int(w.reads.size)
    sc = BatchedScanner(tables, max_bases=n, max_reads=len(w.read_set), graph=False)
    sc.load(w.reads, w.read_offsets, w.read_set)
    if tune:
        tuned = sc.tune(use_cache=False)      # picks the launch shape, then captures the graph
    else:
        sc.capture()
        tuned = {}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        sc.run()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        with torch.cuda.stream(sc.stream):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(sc.stream)
        sc.run()
        with torch.cuda.stream(sc.stream):
            e1.record(sc.stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    batched_out = sc.out[:n].clone()
    ms = statistics.median(times)
    d_text = sc.texts[:n]
    # the baseline as device work: one pfac_match per read, captured in one CUDA graph
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    pg = PerReadGraph(tables, d_text, w.read_offsets, w.read_set, out)
    for _ in range(2):
        pg.run()
    torch.cuda.synchronize()
    per_times = []
    for _ in range(max(3, steps // 4)):
        with torch.cuda.stream(pg.stream):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(pg.stream)
        pg.run()
        with torch.cuda.stream(pg.stream):
            e1.record(pg.stream)
        e1.synchronize()
        per_times.append(e0.elapsed_time(e1))
    per_ms = statistics.median(per_times)
    same = bool(torch.equal(out, batched_out))
    # and as a host loop issuing the same calls one by one (context: host cost per call)
    out2 = torch.zeros(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    scan_per_read(tables, d_text, w.read_offsets, w.read_set, out2)
    torch.cuda.synchronize()
    loop_ms = 1e3 * (time.perf_counter() - t0)
    same = same and bool(torch.equal(out2, batched_out))
    for t in tables:
        t.close()
    return {"workload": w.name, "bases": n, "reads": int(len(w.read_set)), "tables": len(w.sets),
            "table_build_s": build_s, "graph_replay_ms": ms, "gbases_s": n / ms / 1e6,
            "per_read_graph_ms": per_ms, "per_read_gbases_s": n / per_ms / 1e6,
            "batched_vs_per_read": per_ms / ms,
            "per_read_host_loop_ms": loop_ms, "batched_vs_per_read_host_loop": loop_ms / ms,
            "same_output": same,
            "autotune": {k: tuned.get(k) for k in ("lane_offsets", "threads", "ctas_per_sm", "walk_loads",
                                                   "ms", "default_ms", "candidates")},
            "launches_per_batch": 1 if len(w.read_set) <= 8192 else 4, "launches_per_read_pass": pg.launches,
            "per_read_baseline": "one pfac_match (scan + tail kernel) per read, all captured in one CUDA graph "
                                 "and replayed; L2 flushed before each replay"}


def large_dict_measure(steps: int):
    """The large-dictionary workload: 2^30 i.i.d. bases at 41 % GC against 10^6 patterns
    of 16-64 bases (a trie of tens of millions of states, held in HBM); dense ids and
    the compacted (offset, id) list, each timed over `steps` launches with the L2
    flushed before each."""
    import torch
    from paper_1811_10498_gb300 import _binding as b
    from paper_1811_10498_gb300 import datagen
    w = datagen.large_dict_scan(seed=3)
    n = int(w.text.size)
    t0 = time.perf_counter()
    table = b.Table((w.blob, w.offsets))
    build_s = time.perf_counter() - t0
    info = table.info
    d_text = torch.from_numpy(w.text).cuda()
    packed, status, _ = b.pack(d_text)
    del d_text
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cap = 1 << 24
    d_off = torch.empty(cap, dtype=torch.int64, device="cuda")
    d_ids = torch.empty(cap, dtype=torch.int32, device="cuda")
    d_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    assert int(status.item()) == 0

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    dense_ms = timed(lambda: b.pfac_match_packed(table.h, packed, n, out))
    compact_ms = timed(lambda: b.pfac_match_compact(table.h, packed, n, d_off, d_ids, d_cnt))
    matches = int(d_cnt.item())
    same = matches <= cap and int((out != 0).sum().item()) == matches
    # the same table built on the GPU from the patterns in device memory (after one small
    # build that loads the construction kernels), and a scan with it
    d_blob = torch.from_numpy(w.blob).cuda()
    d_offs = torch.from_numpy(w.offsets.astype(np.int64)).cuda()
    b.Table.from_device(d_blob[:64], torch.tensor([0, 16, 32], dtype=torch.int64, device="cuda")).close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tdev = b.Table.from_device(d_blob, d_offs)
    dev_build_s = time.perf_counter() - t0
    keys = ("n_states", "n_duplicates", "filter_b", "filter_set", "table_bytes", "sample_q")
    same_info = all(tdev.info[k] == info[k] for k in keys)
    out2 = torch.empty_like(out)
    b.pfac_match_packed(tdev.h, packed, n, out2)
    torch.cuda.synchronize()
    same_dev_ids = bool(torch.equal(out, out2))
    tdev.close()
    del out2, d_blob, d_offs
    peak, _ = measured_hbm()
    res = {"workload": w.name, "bases": n, "n_states": info["n_states"], "filter_b": info["filter_b"],
           "table_bytes": info["table_bytes"], "table_build_s": build_s,
           "dense_ms": dense_ms, "dense_gbases_s": n / dense_ms / 1e6,
           "dense_roofline_frac": BYTES_PER_BASE * n / (dense_ms * 1e-3) / (peak * 1e9),
           "compact_ms": compact_ms, "compact_gbases_s": n / compact_ms / 1e6, "matches": matches,
           "compact_count_equals_dense_nonzeros": same,
           "device_build_s": dev_build_s, "device_build_same_counts": same_info,
           "device_build_same_ids": same_dev_ids, "sample_q": info["sample_q"],
           "config": b.pfac_get_config(table.h, n)}
    table.close()
    return res


def serving_measure(seconds: float):
    """The serving workload: Poisson arrivals at 2,000 requests/s, 16 resident tables of
    1,000-200,000 patterns, texts of 1 kb-10 Mb.

    * served: the continuous-batching server on the stream in real time (p50/p99
      latency, Gbases/s; at this offered load it keeps up, so its Gbases/s is the
      offered load);
    * per_request: the same stream in real time served one request at a time with one
      pfac_match launch each (serving.serve_per_request);
    * capacity: both again with every request arriving at time 0 (saturation): the
      Gbases/s each can serve, and their ratio."""
    from paper_1811_10498_gb300 import _binding as b
    from paper_1811_10498_gb300 import datagen
    from paper_1811_10498_gb300.serving import Server, requests_from_stream, serve_per_request
    st = datagen.request_stream(seed=5, duration=seconds)
    tables = [b.Table(s) for s in st.sets]
    srv = Server(tables, slot_bases=1 << 24, n_slots=3, max_reads=4096)
    reqs = requests_from_stream(st)
    _, _, stats = srv.run(reqs, realtime=True)
    stats["workload"] = st.name
    stats["offered_gbases_s"] = stats["bases"] / seconds / 1e9
    _, _, per = serve_per_request(tables, reqs, realtime=True)
    _, _, cap = srv.run(reqs, realtime=False)
    _, _, per_cap = serve_per_request(tables, reqs, realtime=False)
    stats["per_request"] = {k: per[k] for k in ("gbases_s", "p50_ms", "p99_ms", "wall_s", "launches")}
    stats["capacity"] = {"all_requests_at_t0": True, "batched": {k: cap[k] for k in
                                                                 ("gbases_s", "p50_ms", "p99_ms", "wall_s",
                                                                  "batches")},
                         "per_request": {k: per_cap[k] for k in ("gbases_s", "p50_ms", "p99_ms", "wall_s")}}
    stats["capacity_gbases_s"] = cap["gbases_s"]
    stats["per_request_gbases_s"] = per_cap["gbases_s"]
    stats["served_vs_per_request"] = cap["gbases_s"] / per_cap["gbases_s"] if per_cap["gbases_s"] else None
    for t in tables:
        t.close()
    return stats


def paper_suite(args):
    """The paper's experiments re-run on GB300 with synthetic stand-ins for its files:
    input data sets of 0.75-3.75 M newline-separated 100-base lines (Table IV) and
    pattern sets of 1,000-5,000 100-base patterns (Table III), scanned as ASCII.

    * placement (Figs. 6-8) on input set 5 for every pattern set: the paper's kernel
      structure (one thread per offset, kernel 1) with the transition table as its two
      arrays (nextState, matchedPatternId) or merged into one array of pairs, the text in
      global memory or staged per block in shared memory, table loads through the
      default L1-cached path, the read-only (texture) path, or with L1 bypassed (the
      paper's L1-off setting); kernel 1 over 16-byte rows; and this design's pipelined
      kernel (prefix filter in shared memory, rank index in shared or global memory, an
      L2 access-policy window on the skip entries);
    * patterns: Fig. 9's sweep (pattern sets 1-5 on input set 5), the same points;
    * inputs: Fig. 10's sweep (input sets 1-5 with pattern set 5), the paper's best
      placement (one array, text in shared memory, texture path) vs this design.
    Prints one JSON line per point: median kernel time over the timed launches (L2
    flushed before each), Gbases/s counting every input byte as an offset, and the HBM
    roofline fraction at 5 bytes per offset (1 in, 4 out)."""
    import torch
    from paper_1811_10498_gb300 import _binding as b
    from paper_1811_10498_gb300 import build_ext, datagen
    build_ext.build()
    peak, peak_kind = measured_hbm()
    src = datagen.paper_source()
    lines = [750_000 * k for k in range(1, 6)]
    n_pats = [1000 * k for k in range(1, 6)]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    texts = {}

    def text(n_lines):
        if n_lines not in texts:
            texts.clear()
            texts[n_lines] = torch.from_numpy(datagen.paper_input(src, n_lines)).cuda()
        return texts[n_lines]

    # Fig. 6: {two arrays, one merged array} x {GM only, GM + text in SM, GM + SM + table
    # through the texture path}; Figs. 7-8: L1 on (default global loads) vs L1 bypassed;
    # then this design's kernel 1 (16-byte rows) and kernel 2 placements.
    placements = {
        "GM, two arrays": dict(kernel=1, table_layout=1, row_loads=1, text_smem=0),
        "GM+SM, two arrays": dict(kernel=1, table_layout=1, row_loads=1, text_smem=1),
        "GM+SM+Tex, two arrays": dict(kernel=1, table_layout=1, row_loads=0, text_smem=1),
        "GM, one array": dict(kernel=1, table_layout=2, row_loads=1, text_smem=0),
        "GM+SM, one array": dict(kernel=1, table_layout=2, row_loads=1, text_smem=1),
        "GM+SM+Tex, one array": dict(kernel=1, table_layout=2, row_loads=0, text_smem=1),
        "GM+SM, two arrays, L1 off": dict(kernel=1, table_layout=1, row_loads=2, text_smem=1),
        "GM+SM, one array, L1 off": dict(kernel=1, table_layout=2, row_loads=2, text_smem=1),
        "global (kernel 1)": dict(kernel=1),
        "smem text + smem filter, rank in global": dict(kernel=2, rank_in_smem=-1),
        "smem text + smem filter and rank (default)": dict(kernel=0),
        "default + L2 window on skip entries": dict(kernel=2, l2_persist=1),
    }

    ref_ids = {}

    def point(fig, n_lines, n_p, label, cfg):
        d_text = text(n_lines)
        blob, offs = datagen.paper_patterns(src, n_p)
        t = b.Table((blob, offs))
        b.pfac_set_config(t.h, cfg)
        out = torch.empty(d_text.numel(), dtype=torch.int32, device="cuda")
        for _ in range(3):
            t.match(d_text, out)
        torch.cuda.synchronize()
        # every placement must give the same ids as the first one timed on this input
        key = (n_lines, n_p)
        if key not in ref_ids:
            ref_ids[key] = out.clone()
        same = bool(torch.equal(out, ref_ids[key]))
        ts = []
        for _ in range(min(args.steps, 20)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            t.match(d_text, out)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        n = d_text.numel()
        line = {"suite": "paper", "figure": fig, "input_lines": n_lines, "input_bytes": n, "patterns": n_p,
                "placement": label, "config": b.pfac_get_config(t.h, n), "ms": ms, "gbases_s": n / ms / 1e6,
                "roofline_frac": 5.0 * n / (ms * 1e-3) / (peak * 1e9), "peak_gbs": peak, "peak_source": peak_kind,
                "matches": int((out != 0).sum().item()), "filter_b": t.info["filter_b"], "states": t.info["n_states"],
                "same_ids_as_first_placement": same}
        print(json.dumps(line), flush=True)
        b.pfac_set_config(t.h, None)
        t.close()

    for n_p in n_pats:                                 # Figs. 6-8 and 9
        for label, cfg in placements.items():
            point("6-9", lines[-1], n_p, label, cfg)
    for n_l in lines[:-1]:                             # Fig. 10 (input set 5 is above)
        for label in ("GM+SM+Tex, one array", "smem text + smem filter and rank (default)"):
            point("10", n_l, n_pats[-1], label, placements[label])

    # the paper's host program from files (Figs. 4-5): pattern set 5 and input set 5 written
    # to files, read back, the table built from its file, the text scanned from host memory
    import tempfile
    from paper_1811_10498_gb300.hoststream import HostScanner
    blob, offs = datagen.paper_patterns(src, n_pats[-1])
    text = datagen.paper_input(src, lines[-1])
    with tempfile.TemporaryDirectory() as d:
        pf, tf = os.path.join(d, "patterns.txt"), os.path.join(d, "input.txt")
        with open(pf, "wb") as f:
            f.write(b"\n".join(datagen.pattern_list(blob, offs)) + b"\n")
        text.tofile(tf)
        t0 = time.perf_counter()
        h_text = torch.from_numpy(b.read_text_file(tf)).pin_memory()
        read_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        t = b.Table.from_file(pf)
        build_s = time.perf_counter() - t0
    h_out = torch.empty(h_text.numel(), dtype=torch.int32).pin_memory()
    hs = HostScanner(t, chunk_bases=1 << 24, ascii=True)
    hs.scan(h_text, h_out)
    hs.synchronize()
    runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs.scan(h_text, h_out)
        hs.synchronize()
        runs.append(time.perf_counter() - t0)
    scan_s = statistics.median(runs)
    ref = b.Table((blob, offs))
    same = bool(torch.equal(h_out, ref.match(torch.from_numpy(text).cuda()).cpu()))
    n = h_text.numel()
    print(json.dumps({"suite": "paper", "figure": "4-5 (files)", "input_lines": lines[-1], "input_bytes": n,
                      "patterns": n_pats[-1], "read_s": read_s, "read_gb_s": n / read_s / 1e9,
                      "build_from_file_s": build_s, "scan_from_host_s": scan_s,
                      "scan_from_host_gbases_s": n / scan_s / 1e9, "same_as_in_memory": same}), flush=True)
    t.close()
    ref.close()


def large_suite(args):
    """The large-dictionary workload at `--n-bases` bases (10^6 patterns of 16-64 bases),
    scanned `--steps` times (dense ids, L2 flushed before each), with the table built
    the default way (order-14 filter, sampled 13-gram screen) or in the earlier
    structure (`--large-structure order12`: order-12 filter behind the order-10
    first-level filter). One JSON line."""
    import torch
    from paper_1811_10498_gb300 import _binding as b
    from paper_1811_10498_gb300 import build_ext, datagen
    build_ext.build()
    w = datagen.large_dict_scan(seed=3, n_bases=args.n_bases)
    n = int(w.text.size)
    kw = dict(filter_b=12, sample=-1) if args.large_structure == "order12" else {}
    if args.large_filter_b:
        kw["filter_b"] = args.large_filter_b
    table = b.Table((w.blob, w.offsets), **kw)
    if args.large_config:
        b.pfac_set_config(table.h, json.loads(args.large_config))
    d = torch.from_numpy(w.text).cuda()
    packed, _, _ = b.pack(d)
    del d
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    b.pfac_match_packed(table.h, packed, n, out)
    ts = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.pfac_match_packed(table.h, packed, n, out)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    peak, _ = measured_hbm()
    info = table.info
    print(json.dumps({"suite": "large", "workload": w.name, "structure": args.large_structure,
                      "config": b.pfac_get_config(table.h, n), "bases": n,
                      "filter_b": info["filter_b"], "sample_q": info["sample_q"], "n_states": info["n_states"],
                      "ms": ms, "gbases_s": n / ms / 1e6,
                      "roofline_frac": BYTES_PER_BASE * n / (ms * 1e-3) / (peak * 1e9),
                      "matches": int((out != 0).sum().item()), "device_status": b.pfac_device_status(table.h),
                      "launches": 1 + args.steps}), flush=True)
    table.close()


def ceilings_suite():
    """The hardware ceilings behind the kernels' design (csrc/ceilings.cu, built here with
    nvcc for sm_103a): store bandwidth for 1 GiB of ids by several store paths, and random
    4-byte lookup rates from L1/L2/HBM, shared memory and cluster distributed shared
    memory. Prints the program's JSON lines."""
    from paper_1811_10498_gb300 import build_ext
    src = os.path.join(build_ext.CSRC, "ceilings.cu")
    os.makedirs(build_ext.BUILD, exist_ok=True)
    exe = os.path.join(build_ext.BUILD, "ceilings")
    subprocess.run([build_ext.nvcc(), "-O3", *build_ext.ARCH, "-o", exe, src], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    for line in r.stdout.splitlines():
        if line.startswith("{"):
            print(json.dumps({"suite": "ceilings", **json.loads(line)}), flush=True)
    if r.returncode != 0:
        raise SystemExit(r.returncode)


def configs_suite(steps: int):
    """Kernel-2 launch configurations on the genome-scale workload (the benchmark's
    table and text): the default, the shared-memory 10-gram screen, the zero-writer
    warp, stages, walk depth, rank index placement. One JSON line each: median step time
    (L2 flushed before each step) and whether the ids equal the default's."""
    import torch
    from paper_1811_10498_gb300 import _binding as b
    from paper_1811_10498_gb300 import build_ext
    build_ext.build()
    w = make_workload(0, N_BASES, N_PATTERNS)
    n = w.text.size
    table = b.Table((w.blob, w.offsets))
    d = torch.from_numpy(w.text).cuda()
    packed, _, _ = b.pack(d)
    del d
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    peak, _ = measured_hbm()
    ref = None
    # the same table built with the 10-gram screen too (pfac_build_opts.sample = 1)
    table10 = b.Table((w.blob, w.offsets), sample=1)
    cfgs = [dict(), dict(screen=2, sample=1), dict(screen=2, walk_loads=1, sample=1),
            dict(screen=2, rank_in_smem=-1, sample=1), dict(zero_writer=2), dict(zero_writer=3), dict(zero_writer=4),
            dict(zero_writer=4, walk_loads=1), dict(zero_writer=4, stages=4), dict(stages=2),
            dict(stages=4), dict(walk_loads=1), dict(rank_in_smem=-1), dict(lane_offsets=16, stages=4)]
    for cfg in cfgs:
        cfg = dict(cfg)
        t = table10 if cfg.pop("sample", 0) else table
        b.pfac_set_config(t.h, dict(kernel=2, **cfg))
        for _ in range(3):
            b.pfac_match_packed(t.h, packed, n, out)
        torch.cuda.synchronize()
        if ref is None:
            ref = out.clone()
        ts = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.pfac_match_packed(t.h, packed, n, out)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        print(json.dumps({"suite": "configs", "workload": workload_name(), "config": cfg,
                          "table": "with the 10-gram screen" if t is table10 else "default", "ms": ms,
                          "roofline_frac": BYTES_PER_BASE * n / (ms * 1e-3) / (peak * 1e9),
                          "same_ids_as_default": bool(torch.equal(out, ref)),
                          "device_status": b.pfac_device_status(t.h)}), flush=True)
    table.close()
    table10.close()


def run_reference(args):
    """The oracle, as it stands, on the host cores: each step scans a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1811_10498_gb300 import datagen
    w = make_workload(0, args.n_bases, args.n_patterns)
    threads = os.cpu_count() or 1
    trie = oracle.Trie((w.blob, w.offsets))
    n = w.text.size
    probe = min(n, 1 << 20)
    t0 = time.perf_counter()
    trie.scan_threads(w.text, threads, 0, probe)
    rate = probe / max(time.perf_counter() - t0, 1e-9)
    per_step = max(64, int(rate * min(1.0, 90.0 / max(1, args.steps + args.warmup))))
    per_step = min(per_step, n)
    for i in range(args.warmup):
        lo = (i * per_step) % max(1, n - per_step)
        trie.scan_threads(w.text, threads, lo, lo + per_step)
    times = []
    for i in range(args.steps):
        lo = ((args.warmup + i) * per_step) % max(1, n - per_step)
        t0 = time.perf_counter()
        trie.scan_threads(w.text, threads, lo, lo + per_step)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * args.steps / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": workload_name(args.n_bases, args.n_patterns), "n_bases": int(n),
                       "n_patterns": args.n_patterns,
                       "inputs": {"seed": 2, "text_sha256": datagen.sha256(w.text),
                                  "patterns_sha256": datagen.sha256(w.blob)}},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} consecutive offsets per step, {threads} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-bases", type=int, default=N_BASES)
    ap.add_argument("--n-patterns", type=int, default=N_PATTERNS)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-chunk", type=int, default=1 << 25)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the large-dictionary (10^6 patterns) leg")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--no-tune", action="store_true", help="use the library's default launch configuration")
    ap.add_argument("--large-structure", default="default", choices=["default", "order12"],
                    help="--suite large: the table's filter structure")
    ap.add_argument("--large-config", default="", help="--suite large: a launch configuration (JSON of pfac_config "
                                                        "fields) applied to the table")
    ap.add_argument("--large-filter-b", type=int, default=0, help="--suite large: the table's filter order (0 = automatic)")
    ap.add_argument("--suite", default=None, choices=["paper", "batched", "ceilings", "configs", "large"],
                    help="paper: the paper's placement, pattern-set and input-size experiments (many lines); "
                         "batched: the batched workload alone; ceilings: store and lookup rates of the GPU; "
                         "configs: kernel-2 launch configurations on the benchmark's workload; "
                         "large: the large-dictionary workload at --n-bases")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.suite == "paper":
        paper_suite(args)
        return
    if args.suite == "large":
        large_suite(args)
        return
    if args.suite == "ceilings":
        ceilings_suite()
        return
    if args.suite == "configs":
        configs_suite(min(args.steps, 60))
        return
    if args.suite == "batched":
        from paper_1811_10498_gb300 import build_ext
        build_ext.build()
        print(json.dumps({"suite": "batched", **batched_measure(min(args.steps, 20), tune=not args.no_tune)}),
              flush=True)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1811_10498_gb300 import _binding as b
    from paper_1811_10498_gb300 import build_ext, datagen
    build_ext.build()

    w = make_workload(rank, args.n_bases, args.n_patterns)
    n = w.text.size
    t0 = time.perf_counter()
    table = b.Table((w.blob, w.offsets))
    build_s = time.perf_counter() - t0
    info = table.info

    stream = torch.cuda.current_stream(dev)
    d_text = torch.from_numpy(w.text).to(dev)
    packed, status, bad = b.pack(d_text)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(max(4 * l2, 256 << 20), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    assert int(status.item()) == 0

    # launch configuration: the autotuner's pick for this table and text size
    tuned = {}
    if not args.no_tune:
        from paper_1811_10498_gb300 import autotune
        tuned = autotune.tune_scan(table, packed, n, packed=True, use_cache=False)

    # pack throughput (not part of a step: the text is packed once)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        b.pfac_pack(d_text, packed, None, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    pack_gbs = 5 * n / (e0.elapsed_time(e1) * 1e-3) / 1e9

    def step():
        b.pfac_match_packed(table.h, packed, n, out, stream)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    # clocks sampled every 50 ms from here to the end of the run (the timed steps, then
    # the other legs, all of them GPU load)
    clocks = ClockSampler(local, interval_ms=50).start()
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                      # L2 flushed between timed steps (outside the events)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    wall = wall1 - wall0
    if world > 1:
        dist.barrier()
    # a bounded wait that ran out inside a timed step would leave ids unwritten: the
    # run is void unless every kernel of the timed steps reported PFAC_OK
    device_status = b.pfac_device_status(table.h, stream)
    if device_status != 0:
        clocks.stop()
        print(f"bench: device status {device_status} ({b.lib().pfac_error_string(device_status).decode()}) "
              "after the timed steps; no result", file=sys.stderr, flush=True)
        sys.exit(3)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s, value = job_throughput(sum(step_ms) * 1e-3, n, args.steps, world, dev)
    ms_per_step = 1e3 * total_s / args.steps

    # roofline of the scan kernel (the only kernel of a step)
    peak, peak_kind = measured_hbm()
    t_launch = statistics.median(step_ms) * 1e-3
    achieved = BYTES_PER_BASE * n / t_launch / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(), "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": BYTES_PER_BASE * n,
                "kernel": "scan_kernel<packed> (kernel 2; plus tail_kernel, both inside each step)"
                if b.pfac_get_config(table.h, n)["kernel"] == 2 else "walk_rows_kernel<packed> (kernel 1)"}

    # end to end through the public API with host buffers: the ASCII text in pinned host
    # memory, chunks copied in, packed, scanned and their ids copied out on three streams
    # (hoststream.HostScanner), every step; wall clock from the first copy to the last id
    # on the host.
    from paper_1811_10498_gb300.hoststream import HostScanner
    h_text = torch.from_numpy(w.text).pin_memory()
    h_out = torch.empty(n, dtype=torch.int32).pin_memory()
    hs = HostScanner(table, chunk_bases=args.e2e_chunk)
    n_chunks = (n + hs.chunk - 1) // hs.chunk
    h2d_bytes = n + (n_chunks - 1) * (info["max_len"] - 1)
    # (a) the match list: every offset with a pattern and its id; only the matches cross
    # the host link
    nz = torch.nonzero(out).flatten()
    want_off, want_ids = nz.cpu().numpy(), out[nz].cpu().numpy()
    h_moff = torch.empty(want_off.size + 1024, dtype=torch.int64).pin_memory()
    h_mids = torch.empty(want_off.size + 1024, dtype=torch.int32).pin_memory()
    for _ in range(2):
        n_match = hs.scan_matches(h_text, h_moff, h_mids)
    list_same = bool(n_match == want_off.size and np.array_equal(h_moff.numpy()[:n_match], want_off)
                     and np.array_equal(h_mids.numpy()[:n_match], want_ids))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        hs.scan_matches(h_text, h_moff, h_mids)
    list_s = time.perf_counter() - t0
    e2e = {"value": world * n * args.e2e_steps / list_s / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": 12 * n_match + 8 * n_chunks,
           "steps": args.e2e_steps, "matches": n_match, "same_as_device": list_same,
           "path": f"pinned host ASCII -> hoststream.HostScanner.scan_matches ({hs.chunk}-base chunks: H2D, "
                   "pfac_pack, pfac_match_compact, D2H count then pairs, on three overlapped streams) -> pinned "
                   "host (offset, id) list of every offset with a pattern, ascending"}
    # (b) one id per base: 4 bytes per base cross the host link
    for _ in range(2):
        hs.scan(h_text, h_out)
        assert hs.synchronize() == 0
    e2e_same = bool(torch.equal(h_out, out.cpu()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        hs.scan(h_text, h_out)
        hs.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_dense = {"value": world * n * args.e2e_steps / e2e_s / 1e9, "unit": UNIT,
                 "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": 4 * n,
                 "steps": args.e2e_steps, "same_as_device": e2e_same,
                 "path": f"pinned host ASCII -> hoststream.HostScanner ({hs.chunk}-base chunks: H2D, pfac_pack, "
                         "pfac_match_packed, D2H ids on three overlapped streams) -> pinned host ids"}

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            got = out.cpu().numpy()
            cpu = cpu_baseline(w, got)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload_name(args.n_bases, args.n_patterns), "n_bases": n,
                       "n_patterns": args.n_patterns, "n_states": info["n_states"], "filter_b": info["filter_b"],
                       "l2": "flushed between timed steps (memset of 4x L2 outside the events)",
                       "input_resident": "packed text in HBM",
                       "inputs": {"seed": 2 + rank, "text_sha256": datagen.sha256(w.text),
                                  "patterns_sha256": datagen.sha256(w.blob)}},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "e2e_dense_ids": e2e_dense,
            "gpu_launches": 2 * args.steps,
            "device_status": device_status,
            "clocks": None,
            "wall_s_timed_region": wall,
            "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
            "autotune": {k: tuned.get(k) for k in ("lane_offsets", "threads", "stages", "walk_loads",
                                                   "rank_in_smem", "zero_writer", "ms", "default_ms", "candidates")}
            if tuned else None,
            "extra": {"pack_gbases_s": pack_gbs, "build_s": build_s,
                      "frac_of_roofline_gbases": value / world / (peak / BYTES_PER_BASE)},
        }
        if not args.no_large:
            line["large_dictionary"] = large_dict_measure(10)
        if not args.no_batched:
            line["batched"] = batched_measure(20)
        if not args.no_serving:
            line["serving"] = serving_measure(args.serve_seconds)
        clocks.stop()
        line["clocks"] = clocks.summary()
        line["clocks"]["timed_region"] = clocks.summary(wall0, wall1)
        line["clocks"]["sampled"] = "every 50 ms from the warm-up to the end of the run (all legs)"
        print(json.dumps(line), flush=True)
    else:
        clocks.stop()
    table.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
