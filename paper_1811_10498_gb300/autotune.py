"""Launch-configuration autotuner for the scan kernels.

The knobs are those of ``pfac_config`` (include/pfac.h):

* single scans (kernel 2): offsets per consumer lane and threads per CTA (together the
  tile length, 32 x lane_offsets x consumer warps), text stages in the shared-memory
  ring, dependent table loads a walk may take before it is deferred to the tail kernel,
  shared memory or L2 for the prefix filter's rank index, and who stores the zero ids
  (the consumer warps, or a writer warp with 16-byte or TMA bulk stores);
* batched passes: offsets per lane (the work-item length, 32 x lane_offsets), threads per
  SM of the persistent scan kernel, and the in-kernel walk depth.

Every configuration computes the same integers, so a candidate is accepted only if its
output is bit-identical to the output of the library's default configuration on the same
input; a mismatch raises. Candidates are timed on the device with CUDA events (median of
``reps`` launches). The search is a coordinate descent from the default: one knob at a
time, keeping a value only if it is faster by more than ``rel_gain``, until a whole pass
brings nothing. The winner is written to a JSON cache (``PFAC_TUNE_CACHE``, else
``~/.cache/pfac_gb300/tune.json``) keyed by the device (name, SM count, L2 size) and the
size class of the workload, and applied with ``pfac_set_config``.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import tempfile
import time

from . import _binding as b

SCAN_KNOBS = [
    ("lane_offsets", (16, 32)),
    ("threads", (1024, 512, 256)),
    ("stages", (2, 3, 4, 6)),
    ("walk_loads", (1, 2, 3, 4)),
    ("rank_in_smem", (0, -1)),
    ("zero_writer", (1, 2, 3, 4)),
]
# l2_persist is not searched: the persisting set-aside is a limit of the whole context,
# and on the genome-scale workload (skip entries 17 MB, already L2-resident) the window
# halved the scan's throughput.

# threads x ctas_per_sm = threads per SM of the batched scan kernel (256-thread blocks)
BATCH_KNOBS = [
    ("lane_offsets", (16, 32)),
    ("threads", (256, 512, 1024)),
    ("ctas_per_sm", (1, 2)),
    ("walk_loads", (1, 2, 3, 4)),
]


def cache_path() -> str:
    return os.environ.get("PFAC_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "pfac_gb300",
                                                             "tune.json")


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(entries: dict, path: str | None = None) -> None:
    """Merge ``entries`` into the cache file (written atomically)."""
    path = path or cache_path()
    d = load_cache(path)
    d.update(entries)
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _bucket(x: int) -> int:
    """Power-of-two size class (0 for x <= 1)."""
    return int(round(math.log2(x))) if x > 1 else 0


def device_key(props) -> str:
    """``props``: an object or dict with name, multi_processor_count and L2_cache_size
    (torch.cuda.get_device_properties)."""
    get = (lambda k: props[k]) if isinstance(props, dict) else (lambda k: getattr(props, k))
    return f"{get('name')}|sm{get('multi_processor_count')}|l2={get('L2_cache_size')}"


def scan_key(dev_key: str, info: dict, n_bases: int, packed: bool) -> str:
    return (f"scan|{dev_key}|states=2^{_bucket(int(info['n_states']))}|b={int(info['filter_b'])}"
            f"|n=2^{_bucket(int(n_bases))}|{'packed' if packed else 'ascii'}")


def batch_key(dev_key: str, n_sets: int, n_bases: int, n_reads: int) -> str:
    return f"batch|{dev_key}|sets=2^{_bucket(n_sets)}|n=2^{_bucket(n_bases)}|reads=2^{_bucket(n_reads)}"


def coordinate_search(measure, start: dict, knobs, max_passes: int = 3, rel_gain: float = 0.01):
    """Minimise ``measure(cfg)`` (a time; ``math.inf`` = cannot run) one knob at a time.
    Returns (best config, its time, [(config, time), ...] in the order measured)."""
    best = dict(start)
    best_t = measure(best)
    history = [(dict(best), best_t)]
    for _ in range(max_passes):
        improved = False
        for name, values in knobs:
            for v in values:
                if best.get(name) == v:
                    continue
                cand = dict(best)
                cand[name] = v
                t = measure(cand)
                history.append((dict(cand), t))
                if t < best_t * (1.0 - rel_gain):
                    best, best_t, improved = cand, t, True
        if not improved:
            break
    return best, best_t, history


def _events_median(torch, run, reps: int, flush=None) -> float:
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


# What a 0 ("automatic") field of pfac_config means for the knobs tuned here.
_AUTO = {"walk_loads": 2, "lane_offsets": 16, "l2_persist": -1, "zero_writer": 1}


def _start(h: int, n_bases: int, knobs, packed: bool = True) -> dict:
    """The library's default configuration for ``n_bases`` (the handle's configuration
    must have been reset), with automatic fields replaced by the values they stand for.
    ``pfac_get_config`` describes packed-text launches; an ASCII scan or a batched pass
    with no configuration set uses 2 stages and 16 offsets per lane instead."""
    d = b.pfac_get_config(h, n_bases)
    if not packed:
        d = dict(d, stages=2, lane_offsets=16)
    cfg = {"kernel": d["kernel"]}
    for k, _ in knobs:
        v = d[k]
        cfg[k] = _AUTO.get(k, v) if v == 0 else v
    return cfg


def tune_scan(table, d_input, n_bases: int, packed: bool = True, sample_bases: int = 1 << 26, reps: int = 9,
              use_cache: bool = True, cache: str | None = None, knobs=None, log=None) -> dict:
    """Tune the single-scan configuration of ``table`` (a ``Table``) for texts of about
    ``n_bases`` bases, on the first ``sample_bases`` bases of ``d_input`` (packed words
    or ASCII bytes on the device). Applies and returns the chosen configuration."""
    import torch
    h = table.h
    props = torch.cuda.get_device_properties(d_input.device)
    key = scan_key(device_key(props), b.pfac_info_ex(h), n_bases, packed)
    if use_cache:
        hit = load_cache(cache).get(key)
        if hit:
            b.pfac_set_config(h, hit["config"])
            return dict(hit["config"], cached=True)
    n = min(int(n_bases), int(sample_bases))
    src = d_input[:(n + 15) // 16] if packed else d_input[:n]
    out = torch.empty(n, dtype=torch.int32, device=d_input.device)
    l2 = props.L2_cache_size
    flush = torch.empty(2 * l2, dtype=torch.uint8, device=d_input.device) if 4 * n < 2 * l2 else None

    def run():
        if packed:
            b.pfac_match_packed(h, src, n, out)
        else:
            b.pfac_match(h, src, out, length=n)

    b.pfac_set_config(h, None)
    start = _start(h, n, knobs or SCAN_KNOBS, packed)
    if start["kernel"] != 2:
        return {"kernel": start["kernel"], "cached": False}
    run()
    torch.cuda.synchronize()
    ref = out.clone()

    def measure(cfg):
        try:
            b.pfac_set_config(h, cfg)
        except b.PfacError:
            return math.inf
        out.fill_(-1)
        run()
        torch.cuda.synchronize()
        if not torch.equal(out, ref):
            raise RuntimeError(f"configuration {cfg} changed the scan's output")
        t = _events_median(torch, run, reps, flush)
        if log:
            log(f"  {cfg} -> {t:.4f} ms")
        return t

    t0 = time.perf_counter()
    best, best_t, hist = coordinate_search(measure, start, knobs or SCAN_KNOBS)
    default_t = hist[0][1]
    b.pfac_set_config(h, best)
    entry = {"config": best, "ms": best_t, "default_ms": default_t, "sample_bases": n,
             "candidates": len(hist), "tune_s": time.perf_counter() - t0}
    save_cache({key: entry}, cache)
    return dict(best, cached=False, ms=best_t, default_ms=default_t, candidates=len(hist))


def tune_batched(tables, d_texts, d_read_offsets, d_read_set, d_out, reps: int = 9, use_cache: bool = True,
                 cache: str | None = None, knobs=None, log=None) -> dict:
    """Tune the launch shape of ``pfac_match_batched`` for this batch (the shape is taken
    from the configuration of ``tables[0]``). Applies and returns the chosen
    configuration. Call it before capturing the batched call into a CUDA graph."""
    import torch
    handles = [t.h for t in tables]
    h0 = handles[0]
    props = torch.cuda.get_device_properties(d_texts.device)
    key = batch_key(device_key(props), len(handles), d_texts.numel(), d_read_set.numel())
    if use_cache:
        hit = load_cache(cache).get(key)
        if hit:
            b.pfac_set_config(h0, hit["config"])
            return dict(hit["config"], cached=True)

    def run():
        b.pfac_match_batched(handles, d_texts, d_read_offsets, d_read_set, d_out)

    b.pfac_set_config(h0, None)
    start = _start(h0, 0, knobs or BATCH_KNOBS, packed=False)
    # offsets outside every read are never written: -1 marks them on both sides
    d_out.fill_(-1)
    run()
    torch.cuda.synchronize()
    ref = d_out.clone()

    def measure(cfg):
        try:
            b.pfac_set_config(h0, cfg)
        except b.PfacError:
            return math.inf
        d_out.fill_(-1)
        run()
        torch.cuda.synchronize()
        if not torch.equal(d_out, ref):
            raise RuntimeError(f"configuration {cfg} changed the batched output")
        t = _events_median(torch, run, reps)
        if log:
            log(f"  {cfg} -> {t:.4f} ms")
        return t

    t0 = time.perf_counter()
    best, best_t, hist = coordinate_search(measure, start, knobs or BATCH_KNOBS)
    default_t = hist[0][1]
    b.pfac_set_config(h0, best)
    d_out.copy_(ref)
    entry = {"config": best, "ms": best_t, "default_ms": default_t, "candidates": len(hist),
             "tune_s": time.perf_counter() - t0}
    save_cache({key: entry}, cache)
    return dict(best, cached=False, ms=best_t, default_ms=default_t, candidates=len(hist))
